"""Failure detection on the GPU without a GPU fault: every device-side wait of
the ILU(0) sweeps is bounded.  Withholding the first segments of a segment
sweep (host-side set-up: the sweep's first ticket is moved past them, so
nothing reads or writes out of bounds) leaves the segments that need them
waiting on values nothing publishes; the wait runs out after the system's
bound, the call returns MS_ERR_TIMEOUT, and the same context and system then
sweep and solve correctly."""
import time

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


def test_withheld_segments_time_out_and_context_recovers(ms, ctx):
    gm = G.faulted(18, 14, 7, seed=5, n_fault_x=1, n_fault_y=1, block=(5, 4, 3))
    s = ms.ms_system_create(ctx, gm.grid, 0)
    ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(ref.A, gm.q_active(), 0)
    n = Ap.n
    r = np.random.default_rng(4).standard_normal(n)
    want = O.ilu0_apply(Ap, O.ilu0(Ap), r)
    z = np.empty(n)
    ms.ms_set_wait_limit(ctx, s, 0.05)
    for prec, tol in ((ms.MS_PREC_FP64, 1e-10), (ms.MS_PREC_MIXED, 1e-5)):
        ms.ms_ilu_apply(ctx, s, r, z, precision=prec)          # factors and packed segments
        np.testing.assert_allclose(z, want, rtol=0, atol=tol * np.abs(want).max())
        ms.ms_debug_withhold_segments(ctx, s, 1, precision=prec)
        t0 = time.perf_counter()
        with pytest.raises(ms.MsError) as e:
            ms.ms_ilu_apply(ctx, s, r, z, precision=prec)
        dt = time.perf_counter() - t0
        assert e.value.status == ms.MS_ERR_TIMEOUT
        # the 50 ms bound, not the default 2 s, ended the wait
        assert 0.04 <= dt < 1.5, dt
        # the next sweep on the same system is whole again
        z[:] = np.nan
        ms.ms_ilu_apply(ctx, s, r, z, precision=prec)
        np.testing.assert_allclose(z, want, rtol=0, atol=tol * np.abs(want).max())
    ms.ms_set_wait_limit(ctx, s, 0.0)
    # and the context still solves: Richardson against the oracle
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block)
    c = ms.ms_galerkin(ctx, s, b)
    p = np.zeros(n)
    info = ms.ms_solve(ctx, s, [c], gm.q_active(), p, tol=1e-6, max_iter=2000)
    sysr, Ap2, qp2, B, Ac, L = O.setup_general(gm)
    rr = O.ms_solve(Ap2, [(B, L)], qp2, tol=1e-6, max_iter=2000)
    assert info["converged"] and abs(info["iters"] - rr.iters) <= 1
    assert np.linalg.norm(p - rr.x) <= 1e-6 * np.linalg.norm(rr.x)
    # argument checks
    for bad in (-1.0, 61.0, float("nan")):
        with pytest.raises(ms.MsError) as e:
            ms.ms_set_wait_limit(ctx, s, bad)
        assert e.value.status == ms.MS_ERR_INVALID_ARG
    for bad in (0, 10 ** 8):
        with pytest.raises(ms.MsError) as e:
            ms.ms_debug_withhold_segments(ctx, s, bad)
        assert e.value.status == ms.MS_ERR_INVALID_ARG
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


def test_withholding_needs_segment_sweeps(ms, ctx):
    gm = G.lognormal_box(10, 10, 4, seed=2, block=(5, 5, 2), kz_ratio=0.1)
    s = ms.ms_system_create(ctx, gm.grid, 0)
    ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
    n = gm.grid.N
    z = np.empty(n)
    ms.ms_ilu_apply(ctx, s, np.ones(n), z)
    with pytest.raises(ms.MsError) as e:        # structured grid: line sweeps, no segments
        ms.ms_debug_withhold_segments(ctx, s, 1)
    assert e.value.status == ms.MS_ERR_STATE
    ms.ms_system_release(s)
