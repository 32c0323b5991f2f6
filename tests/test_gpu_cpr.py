"""CPR pressure stage (Sec. 4, quasi-IMPES) through the C ABI against the
oracle: the pressure matrix J*, right-hand side and weights of a compressible
two-phase step, and the predictor solve on J* (non-symmetric Galerkin
stages inverted by Gauss-Jordan elimination)."""
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


CASES = {
    "3d_10x10x4": lambda: G.lognormal_box(10, 10, 4, seed=2, block=(5, 5, 2), kz_ratio=0.1),
    "faulted_18x14x7": lambda: G.faulted(18, 14, 7, seed=5, n_fault_x=1, n_fault_y=1, block=(5, 4, 3)),
    "ragged_13x11x5": lambda: G.lognormal_box(13, 11, 5, seed=21, block=(4, 4, 2), kz_ratio=0.1),
}


def _state(n, seed):
    rng = np.random.default_rng(seed)
    p = 2e7 + 1e6 * rng.standard_normal(n)
    m = len(p[1::7])
    p[0:7 * m:7] = p[1::7]                                     # some equal pressures: upstream ties
    s = rng.uniform(0.0, 1.0, n)
    s[::11] = 0.0                                              # clipped mobility derivatives
    p0 = p - 1e5 * rng.uniform(0.0, 1.0, n)
    s0 = np.clip(s - 0.05 * rng.uniform(0, 1, n), 0.0, 1.0)
    qw, qo = np.zeros(n), np.zeros(n)
    qw[0], qo[n - 1], qw[n - 1] = 0.5, -0.4, -0.1
    return p, s, p0, s0, qw, qo


def _dense_ell(col, val, diag):
    n = len(diag)
    A = np.diag(diag).astype(float)
    for w in range(col.shape[0]):
        for i in range(n):
            if col[w, i] != i:
                A[i, col[w, i]] += val[w, i]
    return A


@pytest.mark.parametrize("case", list(CASES))
def test_cpr_pressure_system_matches_oracle(ms, ctx, case):
    gm = CASES[case]()
    g = gm.grid
    vol, dt = g.dx * g.dy * g.dz, 86400.0
    s = ms.ms_system_create(ctx, g, 0)
    n = ms.ms_system_get_info(s)["n"]
    p, sw, p0, s0, qw, qo = _state(n, 7)
    w = np.empty(2 * n)
    rhs = ms.ms_cpr_pressure_system(ctx, s, gm.perm.ravel(), ms.cpr_fluid(), p, sw, p0, s0, qw, qo, dt, weights=w)
    sysr = O.assemble_tpfa(g, gm.perm)
    out = O.cpr_pressure(sysr, vol, p, sw, p0, s0, qw, qo, dt)
    Jr = out["Jstar"].dense()
    for pinned in (True, False):     # no reference-cell pinning for a CPR system
        col, val, diag = ms.ms_system_get_matrix(ctx, s, pinned)
        np.testing.assert_allclose(_dense_ell(col, val, diag), Jr, rtol=0, atol=1e-12 * np.abs(Jr).max())
    np.testing.assert_allclose(rhs, -out["rstar"], rtol=0, atol=1e-12 * np.abs(out["rstar"]).max())
    np.testing.assert_allclose(w[:n], out["ww"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(w[n:], out["wo"], rtol=1e-12, atol=1e-15)
    ms.ms_system_release(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["3d_10x10x4", "faulted_18x14x7"])
def test_cpr_predictor_solve_matches_oracle(ms, ctx, precision, case):
    """Basis smoothed on the TPFA matrix, Galerkin stage of J* (not
    symmetrised, Gauss-Jordan inverse), GMRES(30) on J* dp = -r*."""
    gm = CASES[case]()
    g = gm.grid
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    vol, dt = g.dx * g.dy * g.dz, 86400.0
    s = ms.ms_system_create(ctx, g, 0)
    n = ms.ms_system_get_info(s)["n"]
    ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
    p, sw, p0, s0, qw, qo = _state(n, 9)
    rhs = ms.ms_cpr_pressure_system(ctx, s, gm.perm.ravel(), ms.cpr_fluid(), p, sw, p0, s0, qw, qo, dt)
    c = ms.ms_galerkin(ctx, s, b, prec)
    Ac = ms.ms_coarse_get(ctx, c)
    dp = np.zeros(n)
    info = ms.ms_solve(ctx, s, [c], rhs, dp, tol=1e-8, max_iter=500, precision=prec, outer=ms.MS_OUTER_GMRES)
    sysr, Ap, qp, B, _, _ = O.setup_general(gm)
    out = O.cpr_pressure(sysr, vol, p, sw, p0, s0, qw, qo, dt)
    J = out["Jstar"]
    Acr = O.galerkin(J, B)
    atol = (1e-12 if precision == "fp64" else 1e-5) * np.abs(Acr).max()   # mixed: the basis is FP32
    np.testing.assert_allclose(Ac, Acr, rtol=0, atol=atol)
    assert np.abs(Ac - Ac.T).max() > 1e-9 * np.abs(Ac).max()            # not symmetrised
    r = O.ms_gmres(J, [(B, O.coarse_lu(J, B))], -out["rstar"], tol=1e-8, max_iter=500, restart=30)
    assert info["converged"] and r.converged
    assert abs(info["iters"] - r.iters) <= 1, (info["iters"], r.iters)
    tol = 1e-6 if precision == "fp64" else 1e-5
    assert np.linalg.norm(dp - r.x) <= tol * np.linalg.norm(r.x)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


def test_tpfa_assembly_after_cpr_restores_pinned_symmetric_system(ms, ctx):
    gm = CASES["3d_10x10x4"]()
    s = ms.ms_system_create(ctx, gm.grid, 0)
    n = ms.ms_system_get_info(s)["n"]
    p, sw, p0, s0, qw, qo = _state(n, 3)
    ms.ms_cpr_pressure_system(ctx, s, gm.perm.ravel(), ms.cpr_fluid(), p, sw, p0, s0, qw, qo, 3600.0)
    ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block)
    c = ms.ms_galerkin(ctx, s, b)
    Ac = ms.ms_coarse_get(ctx, c)
    assert np.array_equal(Ac, Ac.T)
    q = gm.q_active()
    x = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, x, tol=1e-8, max_iter=3000)
    sysr, Ap, qp, B, _, L = O.setup_general(gm)
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-8, max_iter=3000)
    assert info["converged"] and abs(info["iters"] - r.iters) <= 1
    assert np.linalg.norm(x - r.x) <= 1e-6 * np.linalg.norm(r.x)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


def test_cpr_rejects_bad_input(ms, ctx):
    gm = CASES["3d_10x10x4"]()
    s = ms.ms_system_create(ctx, gm.grid, 0)
    n = ms.ms_system_get_info(s)["n"]
    p, sw, p0, s0, qw, qo = _state(n, 1)
    with pytest.raises(ms.MsError) as e:
        ms.ms_cpr_pressure_system(ctx, s, gm.perm.ravel(), ms.cpr_fluid(), p, sw, p0, s0, qw, qo, 0.0)
    assert e.value.status == ms.MS_ERR_INVALID_ARG
    with pytest.raises(ms.MsError):
        ms.ms_cpr_pressure_system(ctx, s, gm.perm.ravel(), ms.cpr_fluid(mu_w=0.0), p, sw, p0, s0, qw, qo, 1.0)
    ms.ms_system_release(s)
