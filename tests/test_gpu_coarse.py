"""The dense coarse inverse ((A_c)^{-1} of Eq. (11)) element by element
against the oracle's Cholesky factorisation and substitution (columns of the
identity), for the blocked sweep in FP64 (CUDA cores) and in FP32 on the
tensor cores: random SPD matrices of ragged sizes around the 32-row pivot
blocks and 128-row tensor tiles, and the Galerkin operators of geomodels as
the stages build them.  Tolerances from the arithmetic: FP64 error of an SPD
inverse ~ cond * 1e-16, FP32 (TF32 split operands, FP32 accumulation) ~
cond * 1e-7, both relative to the largest entry."""
import numpy as np
import pytest

import oracle as O
from paper_2001_01624_gb300 import geomodel as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2001_01624_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(ms):
    c = ms.ms_create(0, torch.cuda.current_stream())
    yield c
    ms.ms_destroy(c)


def _oracle_inverse(A):
    L = O.cholesky(A)
    M = A.shape[0]
    return np.column_stack([O.cholesky_solve(L, np.eye(M)[:, j]) for j in range(M)])


def _spd(M, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((M, M)))
    lam = np.logspace(0, np.log10(cond), M)
    d = np.exp(rng.uniform(-3, 3, M))            # unequal diagonal: exercises the equilibration
    A = (Q * lam) @ Q.T
    A = d[:, None] * A * d[None, :]
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("M", [1, 5, 31, 32, 33, 100, 127, 128, 129, 257, 700])
def test_spd_inverse_matches_oracle(ms, ctx, M):
    A = _spd(M, 100.0, seed=M)
    ref = _oracle_inverse(A)
    scale = np.abs(ref).max()
    X64 = ms.ms_spd_inverse(ctx, A, ms.MS_PREC_FP64)
    assert np.abs(X64 - ref).max() <= 1e-11 * scale
    X32 = ms.ms_spd_inverse(ctx, A, ms.MS_PREC_MIXED)
    # equilibrated condition number <= cond(A) here; 100 * 6e-8 with margin
    assert np.abs(X32 - ref).max() <= 2e-4 * scale


def test_spd_inverse_rejects_indefinite(ms, ctx):
    A = _spd(40, 10.0, seed=3)
    A[17, 17] = -1.0
    for prec in (ms.MS_PREC_FP64, ms.MS_PREC_MIXED):
        with pytest.raises(ms.MsError) as e:
            ms.ms_spd_inverse(ctx, A, prec)
        assert e.value.status == ms.MS_ERR_COARSE_SINGULAR


@pytest.mark.parametrize("case", ["3d_lognormal", "faulted"])
def test_stage_inverse_matches_oracle(ms, ctx, case):
    gm = (G.lognormal_box(40, 36, 10, seed=4, block=(4, 4, 2), kz_ratio=0.1) if case == "3d_lognormal"
          else G.faulted(30, 28, 10, seed=6, n_fault_x=1, n_fault_y=1, block=(3, 4, 2)))
    s = ms.ms_system_create(ctx, gm.grid, 0)
    ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    assert M > 128   # several tensor tiles and pivot blocks
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block)
    c64 = ms.ms_galerkin(ctx, s, b, ms.MS_PREC_FP64)
    Ac = ms.ms_coarse_get(ctx, c64)
    ref = _oracle_inverse(Ac)
    inv = ms.ms_coarse_get_inverse(ctx, c64)
    assert inv["fp64"]
    d = 1.0 / np.sqrt(np.diag(Ac))
    cond = np.linalg.cond(Ac * d[:, None] * d[None, :])
    scale = np.abs(ref).max()
    assert np.abs(inv["X"] - ref).max() <= max(1e-11, 1e-15 * cond) * scale
    bm, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=ms.MS_PREC_MIXED)
    cm = ms.ms_galerkin(ctx, s, bm, ms.MS_PREC_MIXED)
    Acm = ms.ms_coarse_get(ctx, cm)
    refm = _oracle_inverse(Acm)
    invm = ms.ms_coarse_get_inverse(ctx, cm)
    print(case, "M", M, "equilibrated cond", cond, "FP32 check", invm["inv_error"], "FP64 used", invm["fp64"],
          "refinement steps", invm["refine_steps"])
    assert not invm["fp64"]          # well-conditioned: the tensor-core inverse is kept
    assert invm["inv_error"] <= 0.03
    assert np.abs(invm["X"] - refm).max() <= max(2e-4, 2e-7 * cond) * np.abs(refm).max()
    for h in (c64, cm):
        ms.ms_coarse_release(h)
    ms.ms_basis_release(b)
    ms.ms_basis_release(bm)
    ms.ms_system_release(s)
