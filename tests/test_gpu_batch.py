"""Batched basis smoothing (one persistent launch over (member, tile) work
items from a device queue) computes bitwise what smoothing each member alone
computes: basis values, iteration counts and the stopping decision, for FP64
and mixed-precision bases of uneven systems and several work-item shapes;
and one member against the oracle (iterations exact, values to 1e-12)."""
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


MODELS = [lambda: G.lognormal_box(30, 26, 9, seed=31, block=(5, 5, 3), kz_ratio=0.1),
          lambda: G.lognormal_box(17, 40, 6, seed=32, block=(4, 8, 2), kz_ratio=0.1),
          lambda: G.lognormal_box(64, 48, 12, seed=33, block=(8, 8, 4), kz_ratio=0.1),
          lambda: G.lognormal_box(9, 9, 3, seed=34, block=(3, 3, 3), kz_ratio=0.1),
          lambda: G.config1(1)]


def _members(ms, ctx, prec):
    out = []
    for mk in MODELS:
        gm = mk()
        s = ms.ms_system_create(ctx, gm.grid, 0)
        ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
        part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
        b, it = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
        out.append((gm, s, b, it, ms.ms_basis_get(ctx, b)))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_smoothing_is_bitwise_the_single_smoothing(ms, ctx, prec):
    P = ms.MS_PREC_FP64 if prec == "fp64" else ms.MS_PREC_MIXED
    mem = _members(ms, ctx, P)
    for tile, cps in ((1024, 4), (256, 1), (4096, 2)):
        ms.ms_set_batch_tuning(ctx, tile, cps)
        its = ms.ms_basis_rebuild_batch(ctx, [m[1] for m in mem], [m[2] for m in mem])
        for (gm, s, b, it, (cptr, cells, val)), bit in zip(mem, its):
            assert bit == it, (tile, cps, bit, it)
            c2, cl2, v2 = ms.ms_basis_get(ctx, b)
            assert np.array_equal(c2, cptr) and np.array_equal(cl2, cells)
            assert np.array_equal(v2, val), (tile, cps, np.abs(v2 - val).max())
    ms.ms_set_batch_tuning(ctx, 1024, 4)
    if prec == "fp64":   # one member against the oracle
        gm, s, b, it, (cptr, cells, val) = mem[0]
        sysr, Ap, qp, B, Ac, L = O.setup_general(gm)
        assert it == B.iters
        np.testing.assert_allclose(val, B.pval, rtol=0, atol=1e-12)
    for gm, s, b, it, _ in mem:
        ms.ms_basis_release(b)
        ms.ms_system_release(s)


def test_batch_tuning_rejects_bad_shapes(ms, ctx):
    for t, c in ((100, 4), (256, 0), (32768, 2), (512, 9)):
        with pytest.raises(ms.MsError) as e:
            ms.ms_set_batch_tuning(ctx, t, c)
        assert e.value.status == ms.MS_ERR_INVALID_ARG
