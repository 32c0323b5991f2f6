"""Allocation-free ILU(0) application (ms_ilu_apply_noalloc).

Some callers cannot allocate device memory when they apply the smoother --
an application that gave all free memory to its own pool allocator, or a
latency-critical loop that cannot take an allocation's implicit device
synchronisation.  This entry point keeps its scratch in a fixed device array
inside the library.  Its output must equal ms_ilu_apply's (the tolerance of
the other ILU(0) tests, 1e-10 relative) on two calls in a row, the
library's own count of device allocations must not change across a call, and
it must reject what it cannot serve without allocating.  Collected last on
purpose.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("case", ["structured", "faulted"])
def test_noalloc_matches_ilu_apply_twice(ms, case):
    dev = torch.device("cuda:0")
    ctx = ms.ms_create(0, torch.cuda.current_stream())
    try:
        gm = (G.lognormal_box(24, 30, 9, seed=41, block=(6, 6, 3), kz_ratio=0.1) if case == "structured"
              else G.faulted(20, 18, 8, seed=42, n_fault_x=1, n_fault_y=1, block=(5, 6, 4)))
        s = ms.ms_system_create(ctx, gm.grid, 0)
        ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
        n = ms.ms_system_get_info(s)["n"]
        rng = np.random.default_rng(5)
        for _ in range(2):   # two calls in a row, each against the allocating entry point
            r = torch.from_numpy(rng.standard_normal(n)).to(dev)
            zref = torch.empty_like(r)
            ms.ms_ilu_apply(ctx, s, r, zref)           # also computes the factors on first use
            z = torch.full_like(r, float("nan"))
            torch.cuda.synchronize()
            before = ms.ms_allocation_stats()["allocations"]
            ms.ms_ilu_apply_noalloc(ctx, s, r, z)
            torch.cuda.synchronize()
            # the property the entry point exists for: the library allocated nothing
            assert ms.ms_allocation_stats()["allocations"] == before
            a, b = z.cpu().numpy(), zref.cpu().numpy()
            np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12 * np.abs(b).max())
        # host arrays would need staging buffers: rejected
        with pytest.raises(ms.MsError) as e:
            ms.ms_ilu_apply_noalloc(ctx, s, np.zeros(n), np.zeros(n))
        assert e.value.status == ms.MS_ERR_INVALID_ARG
        ms.ms_system_release(s)
    finally:
        ms.ms_destroy(ctx)


def test_noalloc_rejects_missing_factors_and_oversize(ms):
    dev = torch.device("cuda:0")
    ctx = ms.ms_create(0, torch.cuda.current_stream())
    try:
        gm = G.lognormal_box(10, 10, 4, seed=43, block=(5, 5, 2))
        s = ms.ms_system_create(ctx, gm.grid, 0)
        ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
        r = torch.ones(400, dtype=torch.float64, device=dev)
        z = torch.empty_like(r)
        with pytest.raises(ms.MsError) as e:          # factors not computed yet: would need allocation
            ms.ms_ilu_apply_noalloc(ctx, s, r, z)
        assert e.value.status == ms.MS_ERR_STATE
        ms.ms_system_release(s)
        big = G.Grid(128, 128, 65, 1.0, 1.0, 1.0)     # 1,064,960 cells > 1,048,576
        s2 = ms.ms_system_create(ctx, big, 0)
        r2 = torch.ones(big.N, dtype=torch.float64, device=dev)
        with pytest.raises(ms.MsError) as e:
            ms.ms_ilu_apply_noalloc(ctx, s2, r2, torch.empty_like(r2))
        assert e.value.status == ms.MS_ERR_INVALID_ARG and "1048576" in str(e.value)
        ms.ms_system_release(s2)
    finally:
        ms.ms_destroy(ctx)
