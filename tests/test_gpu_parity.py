"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Same seeded inputs on both sides.  Integer results (partitions, supports,
iteration counts of the basis) must match exactly; floating-point results
within the tolerances stated per test: assembly and SpMV to rounding
(1e-13), ILU(0) and basis values to 1e-10 / 1e-12, Galerkin operators to
1e-12 of their largest entry, FP64 solves to relative pressure error 1e-6
with Richardson cycle counts within +/-1, mixed-precision solves to 1e-5.
"""
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
    "2d_12x8": lambda: G.lognormal_box(12, 8, 1, seed=1, block=(4, 4, 1)),
    "3d_10x10x4": lambda: G.lognormal_box(10, 10, 4, seed=2, block=(5, 5, 2), kz_ratio=0.1),
    "ragged_13x11x5": lambda: G.lognormal_box(13, 11, 5, seed=21, block=(4, 4, 2), kz_ratio=0.1),
    "faulted_18x14x7": lambda: G.faulted(18, 14, 7, seed=5, n_fault_x=1, n_fault_y=1, block=(5, 4, 3)),
}


def _dense_ell(col, val, diag):
    n = len(diag)
    A = np.diag(diag).astype(float)
    W = col.shape[0]
    for w in range(W):
        for i in range(n):
            if col[w, i] != i:
                A[i, col[w, i]] += val[w, i]
    return A


def _system(ms, ctx, gm):
    s = ms.ms_system_create(ctx, gm.grid, 0)
    ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel())
    return s


# ------------------------------------------------------------------ assembly
@pytest.mark.parametrize("case", list(CASES))
def test_assembly_matches_oracle(ms, ctx, case):
    gm = CASES[case]()
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, _ = O.pin(ref.A, None, 0)
    for pinned, R in ((False, ref.A), (True, Ap)):
        col, val, diag = ms.ms_system_get_matrix(ctx, s, pinned)
        A = _dense_ell(col, val, diag)
        D = R.dense()
        np.testing.assert_allclose(A, D, rtol=1e-13, atol=1e-13 * np.abs(D).max())
    info = ms.ms_system_get_info(s)
    assert info["n"] == ref.A.n and info["n_faces"] == len(ref.faces[0])
    ms.ms_system_release(s)


def test_assembly_with_upstream_mobility(ms, ctx):
    gm = CASES["3d_10x10x4"]()
    s = ms.ms_system_create(ctx, gm.grid, 0)
    rng = np.random.default_rng(0)
    lam = rng.uniform(0.2, 3.0, gm.grid.n_active())
    pp = rng.standard_normal(gm.grid.n_active())
    pp[1::5] = pp[0::5][: len(pp[1::5])]     # equal pressures across some faces: mean mobility
    ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel(), lam, pp)
    ref = O.assemble_tpfa(gm.grid, gm.perm, lam=lam, p_prev=pp)
    col, val, diag = ms.ms_system_get_matrix(ctx, s, False)
    np.testing.assert_allclose(_dense_ell(col, val, diag), ref.A.dense(), rtol=1e-13,
                               atol=1e-13 * np.abs(ref.A.val).max())
    ms.ms_system_release(s)


def test_invalid_permeability_rejected(ms, ctx):
    gm = CASES["2d_12x8"]()
    s = ms.ms_system_create(ctx, gm.grid, 0)
    bad = gm.perm.copy()
    bad[5, 1] = -1.0
    with pytest.raises(ms.MsError) as e:
        ms.ms_assemble_tpfa(ctx, s, bad.ravel())
    assert e.value.status == ms.MS_ERR_INVALID_ARG
    bad[5, 1] = np.nan
    with pytest.raises(ms.MsError):
        ms.ms_assemble_tpfa(ctx, s, bad.ravel())
    ms.ms_system_release(s)


# -------------------------------------------------------------- SpMV, ILU(0)
@pytest.mark.parametrize("case", ["2d_12x8", "faulted_18x14x7"])
def test_spmv_and_ilu_match_oracle(ms, ctx, case):
    gm = CASES[case]()
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, _ = O.pin(ref.A, None, 0)
    x = np.random.default_rng(1).standard_normal(Ap.n)
    y = np.empty(Ap.n)
    ms.ms_spmv(ctx, s, x, y)
    yr = Ap.to_scipy() @ x
    np.testing.assert_allclose(y, yr, rtol=1e-12, atol=1e-13 * np.abs(yr).max())
    z = np.empty(Ap.n)
    ms.ms_ilu_apply(ctx, s, x, z)
    zr = O.ilu0_apply(Ap, O.ilu0(Ap), x)
    np.testing.assert_allclose(z, zr, rtol=1e-10, atol=1e-12 * np.abs(zr).max())
    # FP32 factors: single-precision rounding only
    ms.ms_ilu_apply(ctx, s, x, z, ms.MS_PREC_MIXED)
    assert np.abs(z - zr).max() <= 1e-4 * np.abs(zr).max()
    ms.ms_system_release(s)


# ---------------------------------------------------------------- partitions
@pytest.mark.parametrize("case", list(CASES))
def test_partitions_match_oracle(ms, ctx, case):
    gm = CASES[case]()
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    rp, rM = O.partition_cartesian(gm.grid, ref.cells, gm.block)
    assert M == rM and np.array_equal(part, rp)
    fac = (np.log(gm.perm[ref.cells, 0]) > np.median(np.log(gm.perm[ref.cells, 0]))).astype(np.int32)
    cls = part * 2 + fac
    out = np.empty(ref.A.n, np.int32)
    Ms = ms.ms_partition_components(ctx, s, cls, out)
    sp, sM = O.components(ref.A, cls)
    assert Ms == sM and np.array_equal(out, sp)
    rng = np.random.default_rng(7)
    dp = rng.standard_normal(ref.A.n) * 10.0 ** rng.uniform(-9, 0, ref.A.n)
    dp[::11] = 0.0
    Md = ms.ms_partition_dynamic(ctx, s, dp, out, 8, 1e-8)
    dpart, dM = O.partition_dynamic(ref.A, dp, 8, 1e-8)
    assert Md == dM and np.array_equal(out, dpart)
    ms.ms_system_release(s)


# -------------------------------------------------------------------- basis
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("rule", ["box", "hop"])
def test_basis_matches_oracle(ms, ctx, case, rule):
    gm = CASES[case]()
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    sup = ms.MS_SUPPORT_BOX if rule == "box" else ms.MS_SUPPORT_HOP
    b, it = ms.ms_build_basis(ctx, s, part, M, support=sup, block=gm.block)
    if rule == "box":
        sp, sc = O.support_box(gm.grid, ref.cells, ref.A, part, M, gm.block)
    else:
        sp, sc = O.support_hop(gm.grid, ref.cells, ref.A, part, M)
    B = O.msrsb_basis(ref.A, part, M, sp, sc)
    cptr, cells, val = ms.ms_basis_get(ctx, b)
    assert np.array_equal(cptr, sp) and np.array_equal(cells, sc)
    assert it == B.iters
    np.testing.assert_allclose(val, B.pval, rtol=0, atol=1e-12)
    # Galerkin coarse operator with the pinned A (Eq. (10))
    c = ms.ms_galerkin(ctx, s, b)
    Ac = ms.ms_coarse_get(ctx, c)
    Ap, _ = O.pin(ref.A, None, 0)
    Acr = O.galerkin(Ap, B)
    np.testing.assert_allclose(Ac, Acr, rtol=0, atol=1e-12 * np.abs(Acr).max())
    assert np.array_equal(Ac, Ac.T)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


def test_basis_update_continues_smoothing(ms, ctx):
    gm = CASES["3d_10x10x4"]()
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, it = ms.ms_build_basis(ctx, s, part, M, block=gm.block, tol=0.0, max_iter=3)
    assert it == 3
    assert ms.ms_basis_update(ctx, s, b, 0.0, 4) == 4
    sp, sc = O.support_box(gm.grid, ref.cells, ref.A, part, M, gm.block)
    B = O.msrsb_basis(ref.A, part, M, sp, sc, tol=0.0, max_iter=7)
    _, _, val = ms.ms_basis_get(ctx, b)
    np.testing.assert_allclose(val, B.pval, rtol=0, atol=1e-12)
    assert ms.ms_basis_rebuild(ctx, s, b) == 3
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


@pytest.mark.parametrize("rule", ["box", "hop"])
def test_basis_cell_order_windows(ms, ctx, monkeypatch, rule):
    """The FP64 smoothing takes its cells by slot count within windows of
    4096 cells: 41x23x9 spans two full windows and a ragged one.  The values
    and the iteration count are those of the natural cell order, bit for bit,
    and those of the oracle."""
    gm = G.lognormal_box(41, 23, 9, seed=33, block=(5, 4, 3), kz_ratio=0.1)
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    sup = ms.MS_SUPPORT_BOX if rule == "box" else ms.MS_SUPPORT_HOP
    got = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("MSGB_SMOOTH_ORDER", flag)
        b, it = ms.ms_build_basis(ctx, s, part, M, support=sup, block=gm.block)
        got[flag] = (it, ms.ms_basis_get(ctx, b))
        ms.ms_basis_release(b)
    monkeypatch.delenv("MSGB_SMOOTH_ORDER")
    (it1, (cp1, ce1, v1)), (it0, (cp0, ce0, v0)) = got["1"], got["0"]
    assert it1 == it0
    assert np.array_equal(cp1, cp0) and np.array_equal(ce1, ce0)
    assert np.array_equal(v1.view(np.int64), v0.view(np.int64))
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    if rule == "box":
        sp, sc = O.support_box(gm.grid, ref.cells, ref.A, part, M, gm.block)
    else:
        sp, sc = O.support_hop(gm.grid, ref.cells, ref.A, part, M)
    B = O.msrsb_basis(ref.A, part, M, sp, sc)
    assert it1 == B.iters
    np.testing.assert_allclose(v1, B.pval, rtol=0, atol=1e-12)
    ms.ms_system_release(s)


# -------------------------------------------------------------------- solve
def _oracle_general(gm, rule="box"):
    return O.setup_general(gm, support=rule)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("smoother", ["ilu0", "jacobi"])
def test_solve_matches_oracle(ms, ctx, case, smoother):
    gm = CASES[case]()
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block)
    c = ms.ms_galerkin(ctx, s, b)
    q = gm.q_active()
    p = np.zeros_like(q)
    sm = ms.MS_SMOOTHER_ILU0 if smoother == "ilu0" else ms.MS_SMOOTHER_JACOBI
    maxit = 3000 if smoother == "ilu0" else 20000
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-6, max_iter=maxit, smoother=sm)
    sysr, Ap, qp, B, Ac, L = _oracle_general(gm)
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-6, max_iter=maxit, smoother=smoother)
    assert info["converged"] == r.converged
    assert abs(info["iters"] - r.iters) <= 1
    assert np.linalg.norm(p - r.x) <= 1e-6 * np.linalg.norm(r.x)
    k = min(len(info["history"]), len(r.hist), 6)
    np.testing.assert_allclose(info["history"][:k], r.hist[:k], rtol=1e-8)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["3d_10x10x4", "faulted_18x14x7"])
@pytest.mark.parametrize("restart", [30, 5])
def test_gmres_matches_oracle(ms, ctx, precision, case, restart):
    gm = CASES[case]()
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
    c = ms.ms_galerkin(ctx, s, b, prec)
    q = gm.q_active()
    p = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-8, max_iter=500, precision=prec, outer=ms.MS_OUTER_GMRES,
                       restart=restart)
    sysr, Ap, qp, B, Ac, L = _oracle_general(gm)
    r = O.ms_gmres(Ap, [(B, L)], qp, tol=1e-8, max_iter=500, restart=restart)
    assert info["converged"] and r.converged
    assert abs(info["iters"] - r.iters) <= 1, (info["iters"], r.iters)
    tol = 1e-6 if precision == "fp64" else 1e-5
    assert np.linalg.norm(p - r.x) <= tol * np.linalg.norm(r.x)
    k = min(len(info["history"]), len(r.hist), 4)
    np.testing.assert_allclose(info["history"][:k], r.hist[:k], rtol=1e-6 if precision == "fp64" else 1e-2)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["3d_10x10x4", "faulted_18x14x7"])
def test_graph_cycles_match_host_cycles(ms, ctx, monkeypatch, precision, case):
    """Cycles run as one CUDA graph with a device-side while loop give the
    same iterates, residual history and cycle count as cycles driven from the
    host (the same kernels in the same order, deterministic reductions)."""
    gm = CASES[case]()
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
    c = ms.ms_galerkin(ctx, s, b, prec)
    q = gm.q_active()
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("MSGB_SOLVE_GRAPH", mode)
        p = np.zeros_like(q)
        info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-8, max_iter=3000, precision=prec)
        out[mode] = (p, info)
    (p0, i0), (p1, i1) = out["0"], out["1"]
    assert i0["converged"] and i1["converged"]
    assert i0["iters"] == i1["iters"]
    np.testing.assert_array_equal(i0["history"], i1["history"])
    np.testing.assert_array_equal(p0, p1)
    # the cycle cap stops the device loop exactly
    monkeypatch.setenv("MSGB_SOLVE_GRAPH", "1")
    p = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-14, max_iter=7, precision=prec)
    assert info["iters"] == 7 and not info["converged"]
    np.testing.assert_array_equal(info["history"], i0["history"][:8])
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gmres_mid_size_grid(ms, ctx, precision):
    """A 40x40x20 grid (32,000 cells): the kernels that end in a reduction
    (residual, norm, the last Gram-Schmidt pass with the new vector's norm)
    launch at most one block per 256 rows, the size of the partial-sum
    buffer; the solve reaches the direct solution."""
    import scipy.sparse.linalg as spla
    gm = G.lognormal_box(40, 40, 20, seed=5, block=(10, 10, 5), kz_ratio=0.1)
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
    c = ms.ms_galerkin(ctx, s, b, prec)
    q = gm.q_active()
    p = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-8, max_iter=500, precision=prec, outer=ms.MS_OUTER_GMRES)
    assert info["converged"]
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(ref.A, q, 0)
    xd = spla.spsolve(Ap.to_scipy().tocsc(), qp)
    assert np.linalg.norm(p - xd) <= 1e-5 * np.linalg.norm(xd)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("restart", [30, 5])
def test_graph_gmres_matches_host_gmres(ms, ctx, monkeypatch, precision, restart):
    """Flexible GMRES run as one CUDA graph (a while node over restarts, one
    conditional node per Arnoldi step, the Hessenberg column, Givens rotations
    and convergence test computed on the device) takes exactly the steps of
    the host-driven loop: the same kernels in the same order, and the small
    least-squares arithmetic in one fma-explicit form on both sides, so step
    counts, iterates and residual histories are bitwise equal."""
    gm = CASES["faulted_18x14x7"]()
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
    c = ms.ms_galerkin(ctx, s, b, prec)
    q = gm.q_active()
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("MSGB_GMRES_GRAPH", mode)
        p = np.zeros_like(q)
        info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-9, max_iter=500, precision=prec, outer=ms.MS_OUTER_GMRES,
                           restart=restart)
        out[mode] = (p, info)
    (p0, i0), (p1, i1) = out["0"], out["1"]
    assert i0["converged"] and i1["converged"]
    assert i0["iters"] == i1["iters"]
    np.testing.assert_array_equal(i1["history"], i0["history"])
    np.testing.assert_array_equal(p1, p0)
    # the step cap stops the device loop exactly, inside a restart cycle
    monkeypatch.setenv("MSGB_GMRES_GRAPH", "1")
    p = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-30, max_iter=7, precision=prec, outer=ms.MS_OUTER_GMRES,
                       restart=restart)
    assert info["iters"] == 7 and not info["converged"]
    np.testing.assert_array_equal(info["history"][:7], i0["history"][:7])
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_batch_matches_individual_solves(ms, ctx, precision):
    """Members of uneven size (structured and faulted) solved concurrently on
    worker streams give exactly what each gives alone: basis re-smoothed,
    Galerkin operator re-formed, then solved."""
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    models = [G.lognormal_box(24, 18, 9, seed=41, block=(8, 6, 3), kz_ratio=0.1),
              G.lognormal_box(10, 30, 4, seed=42, block=(5, 10, 2)),
              G.faulted(18, 14, 7, seed=5, n_fault_x=1, n_fault_y=1, block=(5, 4, 3)),
              G.lognormal_box(40, 12, 16, seed=43, block=(8, 4, 4), kz_ratio=0.1),
              G.lognormal_box(7, 9, 3, seed=44, block=(4, 3, 3))]
    mem = []
    for gm in models:
        s = _system(ms, ctx, gm)
        part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
        b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
        c = ms.ms_galerkin(ctx, s, b, prec)
        mem.append(dict(sys=s, basis=b, coarse=c, q=gm.q_active()))
    ref = []
    for m in mem:
        it = ms.ms_basis_rebuild(ctx, m["sys"], m["basis"])
        ms.ms_coarse_refresh(ctx, m["sys"], m["coarse"])
        p = np.zeros_like(m["q"])
        info = ms.ms_solve(ctx, m["sys"], [m["coarse"]], m["q"], p, tol=1e-8, max_iter=3000, precision=prec)
        ref.append((p, info, it))
    for workers in (3, 1):
        ps = [np.zeros_like(m["q"]) for m in mem]
        out = ms.ms_solve_batch(ctx, [dict(sys=m["sys"], stages=[m["coarse"]], q=m["q"], p=p, rebuild=m["basis"])
                                      for m, p in zip(mem, ps)], tol=1e-8, max_iter=3000, precision=prec,
                                n_workers=workers)
        for (pr, ir, itr), p, o in zip(ref, ps, out):
            assert o["status"] == ms.MS_OK and o["converged"]
            assert o["basis_iters"] == itr
            assert o["iters"] == ir["iters"]
            np.testing.assert_array_equal(o["history"], ir["history"])
            np.testing.assert_array_equal(p, pr)
    for m in mem:
        ms.ms_coarse_release(m["coarse"])
        ms.ms_basis_release(m["basis"])
        ms.ms_system_release(m["sys"])


def test_solve_device_pointers_and_initial_guess(ms, ctx):
    gm = CASES["3d_10x10x4"]()
    dev = torch.device("cuda:0")
    s = ms.ms_system_create(ctx, gm.grid, 0)
    ms.ms_assemble_tpfa(ctx, s, torch.from_numpy(gm.perm.ravel().copy()).to(dev))
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block)
    c = ms.ms_galerkin(ctx, s, b)
    q = torch.from_numpy(gm.q_active()).to(dev)
    p = torch.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-9, max_iter=3000)
    torch.cuda.synchronize()
    assert info["converged"]
    sysr, Ap, qp, B, Ac, L = _oracle_general(gm)
    x = np.linalg.solve(Ap.dense(), qp)
    assert np.linalg.norm(p.cpu().numpy() - x) <= 1e-6 * np.linalg.norm(x)
    # restarting from the converged iterate takes no cycle
    info2 = ms.ms_solve(ctx, s, [c], q, p, tol=1e-6, max_iter=10, use_x0=True)
    assert info2["iters"] == 0 and info2["converged"]
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


def test_not_converged_returns_last_iterate(ms, ctx):
    gm = CASES["2d_12x8"]()
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block)
    c = ms.ms_galerkin(ctx, s, b)
    q = gm.q_active()
    p = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-12, max_iter=3)
    assert info["status"] == ms.MS_ERR_NOT_CONVERGED and info["iters"] == 3 and not info["converged"]
    sysr, Ap, qp, B, Ac, L = _oracle_general(gm)
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-12, max_iter=3)
    assert np.linalg.norm(p - r.x) <= 1e-9 * np.linalg.norm(r.x)
    with pytest.raises(ms.MsError):
        ms.ms_solve(ctx, s, [c], q, p, tol=1e-12, max_iter=3, raise_not_converged=True)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


def test_multistage_static_and_adaptive_match_oracle(ms, ctx):
    gm = G.faulted(20, 16, 8, seed=9, n_fault_x=1, n_fault_y=1, block=(5, 4, 4))
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    fac = gm.facies[ref.cells].astype(np.int32)
    ps = np.empty(ref.A.n, np.int32)
    Ms = ms.ms_partition_components(ctx, s, part * 2 + fac, ps)
    b1, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block)
    b2, _ = ms.ms_build_basis(ctx, s, ps, Ms, support=ms.MS_SUPPORT_HOP)
    c1, c2 = ms.ms_galerkin(ctx, s, b1), ms.ms_galerkin(ctx, s, b2)
    q = gm.q_active()
    sysr, Ap, qp, B, Ac, L = _oracle_general(gm)
    rps, rMs = O.partition_static(ref.A, B.part, gm.facies[ref.cells])
    assert rMs == Ms and np.array_equal(rps, ps)
    sp, sc = O.support_hop(gm.grid, ref.cells, ref.A, rps, rMs)
    B2 = O.msrsb_basis(ref.A, rps, rMs, sp, sc)
    L2 = O.cholesky(O.galerkin(Ap, B2))
    for sched, smoothed in ((0, 0), (2, 0), (1, 0), (2, 1)):
        p = np.zeros_like(q)
        info = ms.ms_solve(ctx, s, [c1, c2], q, p, tol=1e-6, max_iter=3000, adapt_schedule=sched,
                           adapt=dict(smoothed=smoothed))
        ad = None if sched == 0 else dict(schedule=sched, smoothed=smoothed, grid=gm.grid, cells=ref.cells,
                                          A_unpinned=ref.A)
        r = O.ms_solve(Ap, [(B, L), (B2, L2)], qp, tol=1e-6, max_iter=3000, adapt=ad)
        assert info["converged"] and r.converged
        assert abs(info["iters"] - r.iters) <= 1, (sched, smoothed, info["iters"], r.iters)
        assert np.linalg.norm(p - r.x) <= 1e-6 * np.linalg.norm(r.x)
        if sched:
            # Dp(Inf) partitions come from the large early updates and must match
            # exactly.  Dp(1) rebuilds from ever smaller updates; once |dp| nears
            # the rounding level of the iterates its log-binning is not determined
            # (the paper notes these late partitions are dominated by noise), so
            # only the first 10 cycles are compared there.
            k = min(len(info["dyn_blocks"]), len(r.md_hist), 10 if sched == 1 else 10 ** 9)
            assert np.array_equal(info["dyn_blocks"][:k], r.md_hist[:k])
    for h in (c1, c2):
        ms.ms_coarse_release(h)
    for h in (b1, b2):
        ms.ms_basis_release(h)
    ms.ms_system_release(s)


def test_adaptive_basis_entry_point(ms, ctx):
    gm = CASES["faulted_18x14x7"]()
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    dp = np.random.default_rng(3).standard_normal(ref.A.n) * 10.0 ** np.linspace(-6, 0, ref.A.n)
    for smoothed in (0, 1):
        b = ms.ms_add_adaptive_basis(ctx, s, dp, smoothed=smoothed)
        part, M = O.partition_dynamic(ref.A, dp)
        if smoothed:
            sp, sc = O.support_hop(gm.grid, ref.cells, ref.A, part, M)
            B = O.msrsb_basis(ref.A, part, M, sp, sc)
        else:
            B = O.constant_basis(part, M)
        cptr, cells, val = ms.ms_basis_get(ctx, b)
        assert np.array_equal(cptr, B.sptr) and np.array_equal(cells, B.scells)
        np.testing.assert_allclose(val, B.pval, rtol=0, atol=1e-12)
        ms.ms_basis_release(b)
    ms.ms_system_release(s)


# -------------------------------------------------------------- mixed form
@pytest.mark.parametrize("case", ["3d_10x10x4", "faulted_18x14x7"])
def test_mixed_precision_solve(ms, ctx, case):
    gm = CASES[case]()
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=ms.MS_PREC_MIXED)
    c = ms.ms_galerkin(ctx, s, b, ms.MS_PREC_MIXED)
    q = gm.q_active()
    p = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-6, max_iter=3000, precision=ms.MS_PREC_MIXED)
    sysr, Ap, qp, B, Ac, L = _oracle_general(gm)
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-6, max_iter=3000)
    assert info["converged"]
    assert abs(info["iters"] - r.iters) <= 1, (info["iters"], r.iters)
    assert np.linalg.norm(p - r.x) <= 1e-5 * np.linalg.norm(r.x)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


# ------------------------------------------------- tiled wavefront ILU(0)
def _check_ilu_sweeps(ms, ctx, gm):
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, _ = O.pin(ref.A, None, 0)
    lu = O.ilu0(Ap)
    rng = np.random.default_rng(2)
    for _ in range(3):   # repeated sweeps reuse the progress counters
        x = rng.standard_normal(Ap.n)
        z = np.empty(Ap.n)
        ms.ms_ilu_apply(ctx, s, x, z)
        zr = O.ilu0_apply(Ap, lu, x)
        np.testing.assert_allclose(z, zr, rtol=1e-10, atol=1e-12 * np.abs(zr).max())
        ms.ms_ilu_apply(ctx, s, x, z, ms.MS_PREC_MIXED)
        assert np.abs(z - zr).max() <= 1e-4 * np.abs(zr).max()
    ms.ms_system_release(s)


@pytest.mark.parametrize("kernel", ["lines", "pencil"])
@pytest.mark.parametrize("tile", ["4x2", "8x1", "3x3", "32x8", "1x4"])
@pytest.mark.parametrize("shape", [(9, 13, 7), (6, 40, 1), (17, 5, 11), (300, 7, 3)])
def test_tiled_ilu_sweeps_across_tiles(ms, ctx, monkeypatch, kernel, tile, shape):
    """Tiled wavefront sweeps (x-line scans over CTA tiles, or x-pencils, the
    only form for lines longer than 256 cells); small tiles force many CTAs,
    ragged last tiles and cross-tile hand-overs."""
    monkeypatch.setenv("MSGB_ILU_KERNEL", kernel)
    monkeypatch.setenv("MSGB_ILU_TILE", tile)
    monkeypatch.setenv("MSGB_LINE_TILE", tile)
    _check_ilu_sweeps(ms, ctx, G.lognormal_box(*shape, seed=31, block=(3, 4, 2), kz_ratio=0.1))


@pytest.mark.parametrize("kern", ["seg", "seg_pp1", "seg_pp2", "cluster"])
@pytest.mark.parametrize("tk", ["", "3", "1"])
@pytest.mark.parametrize("lines", ["y", "x"])
@pytest.mark.parametrize("shape", [(9, 13, 1), (9, 13, 7), (70, 6, 17), (33, 20, 40), (200, 5, 11),
                                   (60, 9, 85), (12, 4, 200), (256, 3, 5), (20, 60, 17), (7, 256, 9),
                                   (13, 100, 33), (129, 5, 6)])
def test_cluster_ilu_sweeps(ms, ctx, monkeypatch, shape, lines, tk, kern):
    """Line scans pipelined across thread-block clusters: k-rows split over up
    to 16 CTAs per cluster (rows per CTA from 1 to 13, ragged last CTA), on
    y-lines of transposed vectors (y) or on x-lines, one-layer and single-CTA
    grids.  With few rows per CTA (tk) the rows span several clusters, which
    hand lines over through the global ring in ticket order (up to 13
    clusters).  seg: lines cut into 1 to 4 segments of 64 cells (full,
    ragged and single-cell last segments), one warp each (pp1) or two warps
    taking the lines in turn (pp2), passing the value that leaves a segment to
    the next; cluster: one warp per line, 2, 4 and 8 cells per lane."""
    monkeypatch.setenv("MSGB_ILU_KERNEL", "cluster")
    if kern.startswith("seg"):
        monkeypatch.delenv("MSGB_ILU_SEG", raising=False)   # both precisions segmented (the default)
        if kern != "seg":
            monkeypatch.setenv("MSGB_SEG_PP", kern[-1])
        monkeypatch.setenv("MSGB_SEG_LINES", lines)
        if tk:
            monkeypatch.setenv("MSGB_SEG_TK", tk)
    else:
        monkeypatch.setenv("MSGB_ILU_SEG", "0")
        monkeypatch.setenv("MSGB_ILU_LINES", lines)
        if tk:
            monkeypatch.setenv("MSGB_ILU_TK", tk)
    _check_ilu_sweeps(ms, ctx, G.lognormal_box(*shape, seed=37, block=(3, 2, 2), kz_ratio=0.1))


@pytest.mark.parametrize("shape", [(18, 14, 7), (41, 23, 9), (5, 3, 2)])
def test_level_sweeps_match_flag_sweeps(ms, ctx, monkeypatch, shape):
    """Unstructured (faulted) grids: level-synchronous sweeps in one
    cooperative launch and the flag-ordered sweeps sum each row in the same
    slot order, so they agree bit for bit; both match the oracle.  Repeated
    applications reuse the grid barrier's counters."""
    gm = G.faulted(*shape, seed=9, n_fault_x=1, n_fault_y=1, block=(4, 3, 2))
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, _ = O.pin(ref.A, None, 0)
    lu = O.ilu0(Ap)
    xs = [np.random.default_rng(k).standard_normal(Ap.n) for k in range(3)]
    out = {}
    for kernel in ("level", "generic"):
        monkeypatch.setenv("MSGB_ILU_KERNEL", kernel)
        s = _system(ms, ctx, gm)
        ms.ms_profile_reset()
        zs = []
        for x in xs:
            z = np.empty(Ap.n)
            ms.ms_ilu_apply(ctx, s, x, z)
            zr = O.ilu0_apply(Ap, lu, x)
            np.testing.assert_allclose(z, zr, rtol=1e-10, atol=1e-12 * np.abs(zr).max())
            z32 = np.empty(Ap.n)
            ms.ms_ilu_apply(ctx, s, x, z32, ms.MS_PREC_MIXED)
            assert np.abs(z32 - zr).max() <= 1e-4 * np.abs(zr).max()
            zs += [z, z32]
        launched = ms.ms_profile_read()
        assert ("ilu_level_bwd32" in launched) == (kernel == "level")
        out[kernel] = zs
        ms.ms_system_release(s)
    for a, b in zip(out["level"], out["generic"]):
        assert np.array_equal(a, b)


def _long_line_model():
    """700 x 3 x 2 box with one inactive cell: x-lines longer than a segment."""
    gm = G.lognormal_box(700, 3, 2, seed=4, block=(50, 3, 2))
    act = np.ones(gm.grid.N, np.uint8)
    act[5] = 0
    gm.grid.active = act
    return gm


SEG_CASES = {
    "faulted_18x14x7": lambda: G.faulted(18, 14, 7, seed=9, n_fault_x=1, n_fault_y=1, block=(4, 3, 2)),
    "faulted_41x23x9": lambda: G.faulted(41, 23, 9, seed=9, n_fault_x=1, n_fault_y=1, block=(4, 3, 2)),
    "faulted_5x3x2": lambda: G.faulted(5, 3, 2, seed=9, n_fault_x=1, n_fault_y=1, block=(4, 3, 2)),
    "long_lines_700x3x2": _long_line_model,
}


@pytest.mark.parametrize("case", list(SEG_CASES))
def test_segment_sweeps_match_oracle(ms, ctx, monkeypatch, case):
    """Unstructured grids take the segment dataflow sweeps by default: chained
    runs of rows solved by a warp scan, segments handed out by wavefront level.
    They match the oracle's ILU(0) apply and the level-synchronous sweeps
    (same factors; the scan rounds in another order), in FP64 and mixed
    precision, over repeated applications that reuse the flags and tickets."""
    gm = SEG_CASES[case]()
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, _ = O.pin(ref.A, None, 0)
    lu = O.ilu0(Ap)
    xs = [np.random.default_rng(k).standard_normal(Ap.n) for k in range(3)]
    out = {}
    for kernel in ("", "level"):
        if kernel:
            monkeypatch.setenv("MSGB_ILU_KERNEL", kernel)
        else:
            monkeypatch.delenv("MSGB_ILU_KERNEL", raising=False)
        s = _system(ms, ctx, gm)
        ms.ms_profile_reset()
        zs = []
        for x in xs:
            z = np.empty(Ap.n)
            ms.ms_ilu_apply(ctx, s, x, z)
            zr = O.ilu0_apply(Ap, lu, x)
            np.testing.assert_allclose(z, zr, rtol=1e-10, atol=1e-12 * np.abs(zr).max())
            z32 = np.empty(Ap.n)
            ms.ms_ilu_apply(ctx, s, x, z32, ms.MS_PREC_MIXED)
            assert np.abs(z32 - zr).max() <= 1e-4 * np.abs(zr).max()
            zs.append(z)
        launched = ms.ms_profile_read()
        assert ("ilu_seg_fwd" in launched and "ilu_seg_bwd32" in launched) == (kernel == "")
        out[kernel or "seg"] = zs
        ms.ms_system_release(s)
    for a, b in zip(out["seg"], out["level"]):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_ilu_apply_full_size_config2(ms, ctx):
    gm = G.config2(0)
    s = _system(ms, ctx, gm)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(ref.A, gm.q_active(), 0)
    zr = O.ilu0_apply(Ap, O.ilu0(Ap), qp)
    z = np.empty(Ap.n)
    ms.ms_ilu_apply(ctx, s, qp, z)
    np.testing.assert_allclose(z, zr, rtol=1e-9, atol=1e-11 * np.abs(zr).max())
    ms.ms_system_release(s)


# ---------------------------------------------------------------- two-phase
@pytest.mark.parametrize("case", ["3d_10x10x4", "faulted_18x14x7"])
@pytest.mark.parametrize("coop", ["1", "0"])
def test_mobility_and_transport_match_oracle(ms, ctx, monkeypatch, case, coop):
    """Total mobility, and one explicit upstream transport step over many CFL
    substeps: the upstream weights formed once per step, then every substep in
    one cooperative launch with a grid barrier between substeps (coop 1) or one
    launch per substep (coop 0); the substep count and saturations match the
    oracle's face-by-face substeps."""
    monkeypatch.setenv("MSGB_TRANSPORT_COOP", coop)
    gm = CASES[case]()
    n = gm.grid.n_active()
    rng = np.random.default_rng(11)
    S = rng.uniform(0, 1, n)
    fl = ms.fluid(mu_w=1.0, mu_o=3.0, porosity=0.2, cfl=0.9)
    s = ms.ms_system_create(ctx, gm.grid, 0)
    lam = ms.ms_total_mobility(ctx, s, fl, S)
    np.testing.assert_allclose(lam, O.total_mobility(S), rtol=1e-14)
    p_prev = rng.standard_normal(n)
    ms.ms_assemble_tpfa(ctx, s, gm.perm.ravel(), mobility=lam, p_prev=p_prev)
    ref = O.assemble_tpfa(gm.grid, gm.perm, lam=lam, p_prev=p_prev)
    p = rng.standard_normal(n) * 1e6
    q = gm.q_active() * 1e-3
    vol = gm.grid.dx * gm.grid.dy * gm.grid.dz
    dt = 30.0 * vol / np.abs(q).sum()
    S_gpu = S.copy()
    k = ms.ms_transport_step(ctx, s, fl, p, q, dt, S_gpu)
    S_ref, k_ref = O.transport_step(ref.A, p, q, S, dt, porosity=0.2, volume=vol, cfl=0.9)
    assert k == k_ref and k > 1
    np.testing.assert_allclose(S_gpu, S_ref, rtol=1e-11, atol=1e-12)
    # a second step from there (the barrier counters carry over between launches)
    S2 = S_gpu.copy()
    k2 = ms.ms_transport_step(ctx, s, fl, p, q, dt, S2)
    S2_ref, k2_ref = O.transport_step(ref.A, p, q, S_ref, dt, porosity=0.2, volume=vol, cfl=0.9)
    assert k2 == k2_ref
    np.testing.assert_allclose(S2, S2_ref, rtol=1e-10, atol=1e-12)
    ms.ms_system_release(s)


# ------------------------------------------------- finite-volume restriction, well bases
def _fv_setup(ms, ctx, gm, prec):
    s = _system(ms, ctx, gm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
    c = ms.ms_coarse_create(ctx, s, b, prec, ms.MS_RESTRICT_FV)
    return s, b, c


@pytest.mark.parametrize("case", ["3d_10x10x4", "faulted_18x14x7", "ragged_13x11x5", "2d_12x8"])
def test_fv_coarse_operator_matches_oracle(ms, ctx, case):
    """A_c = R A P, R the block indicator (Sec. 5): same entries as the
    oracle's; not symmetric."""
    gm = CASES[case]()
    s, b, c = _fv_setup(ms, ctx, gm, ms.MS_PREC_FP64)
    Ac = ms.ms_coarse_get(ctx, c)
    sysr, Ap, qp, B, _, _ = _oracle_general(gm)
    Acr = O.galerkin_fv(Ap, B)
    np.testing.assert_allclose(Ac, Acr, rtol=0, atol=1e-12 * np.abs(Acr).max())
    ms.ms_coarse_refresh(ctx, s, c)
    assert np.array_equal(ms.ms_coarse_get(ctx, c), Ac)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["3d_10x10x4", "faulted_18x14x7"])
def test_fv_cycle_matches_oracle_and_conserves(ms, ctx, precision, case):
    """Cycles with a finite-volume stage (Gauss-Jordan inverse of the
    non-symmetric A_c): the iterate after one and three cycles matches the
    oracle's (LU solves), and the residual sums to zero over every block."""
    gm = CASES[case]()
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    s, b, c = _fv_setup(ms, ctx, gm, prec)
    sysr, Ap, qp, B, _, _ = _oracle_general(gm)
    F = O.coarse_fv(Ap, B)
    q = gm.q_active()
    for cycles in (1, 3):
        p = np.zeros_like(q)
        info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-30, max_iter=cycles, precision=prec)
        assert info["iters"] == cycles
        r = O.ms_solve(Ap, [(B, F)], qp, tol=1e-30, max_iter=cycles)
        tol = 1e-10 if precision == "fp64" else 1e-5
        assert np.linalg.norm(p - r.x) <= tol * np.linalg.norm(r.x)
        res = qp - Ap.to_scipy() @ p
        sums = np.bincount(B.part, weights=res, minlength=B.M)
        assert np.abs(sums).max() <= (1e-9 if precision == "fp64" else 1e-4) * np.abs(res).sum()
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fv_gmres_matches_oracle(ms, ctx, precision):
    gm = CASES["faulted_18x14x7"]()
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    s, b, c = _fv_setup(ms, ctx, gm, prec)
    q = gm.q_active()
    p = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-8, max_iter=500, precision=prec, outer=ms.MS_OUTER_GMRES)
    sysr, Ap, qp, B, _, _ = _oracle_general(gm)
    r = O.ms_gmres(Ap, [(B, O.coarse_fv(Ap, B))], qp, tol=1e-8, max_iter=500, restart=30)
    assert info["converged"] and r.converged
    assert abs(info["iters"] - r.iters) <= 1, (info["iters"], r.iters)
    tol = 1e-6 if precision == "fp64" else 1e-5
    assert np.linalg.norm(p - r.x) <= tol * np.linalg.norm(r.x)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


def test_fv_gauss_jordan_larger_coarse_system(ms, ctx):
    """Several hundred coarse blocks (many rows per block of the cooperative
    grid): FP64 cycle equals the oracle's LU-based cycle."""
    gm = G.lognormal_box(60, 44, 10, seed=23, block=(4, 4, 2), kz_ratio=0.1)
    s, b, c = _fv_setup(ms, ctx, gm, ms.MS_PREC_FP64)
    sysr, Ap, qp, B, _, _ = _oracle_general(gm)
    assert B.M > 700
    q = gm.q_active()
    p = np.zeros_like(q)
    ms.ms_solve(ctx, s, [c], q, p, tol=1e-30, max_iter=1)
    r = O.ms_solve(Ap, [(B, O.coarse_fv(Ap, B))], qp, tol=1e-30, max_iter=1)
    assert np.linalg.norm(p - r.x) <= 1e-10 * np.linalg.norm(r.x)
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)


def test_well_partition_and_basis_match_oracle(ms, ctx):
    """Well bases (Sec. 6.2): partition {each well's cells, the rest}, MsRSB on
    hop supports, as a second stage beside the general one."""
    gm = CASES["3d_10x10x4"]()
    s = _system(ms, ctx, gm)
    sysr, Ap, qp, B, Ac, L = _oracle_general(gm)
    wells = [np.flatnonzero(qp > 0), np.flatnonzero(qp < 0)]
    wells = [w for w in wells if len(w)]
    part, M = ms.ms_partition_wells(ctx, s, wells)
    rp, rM = O.partition_wells(Ap.n, wells)
    assert M == rM and np.array_equal(part, rp)
    with pytest.raises(ms.MsError):
        ms.ms_partition_wells(ctx, s, [wells[0], wells[0][:1]])
    bw, it = ms.ms_build_basis(ctx, s, part, M, support=ms.MS_SUPPORT_HOP)
    sp, sc = O.support_hop(gm.grid, sysr.cells, sysr.A, part, M)
    Bw = O.msrsb_basis(sysr.A, part, M, sp, sc)
    cptr, cells, val = ms.ms_basis_get(ctx, bw)
    assert np.array_equal(cptr, sp) and np.array_equal(cells, sc) and it == Bw.iters
    np.testing.assert_allclose(val, Bw.pval, rtol=0, atol=1e-12)
    pg, Mg = ms.ms_partition_cartesian(ctx, s, gm.block)
    bg, _ = ms.ms_build_basis(ctx, s, pg, Mg, block=gm.block)
    cg, cw = ms.ms_galerkin(ctx, s, bg), ms.ms_galerkin(ctx, s, bw)
    q = gm.q_active()
    p = np.zeros_like(q)
    info = ms.ms_solve(ctx, s, [cg, cw], q, p, tol=1e-8, max_iter=3000)
    r = O.ms_solve(Ap, [(B, L), (Bw, O.cholesky(O.galerkin(Ap, Bw)))], qp, tol=1e-8, max_iter=3000)
    assert info["converged"] and r.converged and abs(info["iters"] - r.iters) <= 1
    assert np.linalg.norm(p - r.x) <= 1e-6 * np.linalg.norm(r.x)
    for h in (cg, cw):
        ms.ms_coarse_release(h)
    for h in (bg, bw):
        ms.ms_basis_release(h)
    ms.ms_system_release(s)


@pytest.mark.parametrize("M", [1, 2, 5, 37, 152, 153, 700, 1300])
def test_gauss_jordan_inverse_with_pivoting(ms, ctx, M):
    """The Gauss-Jordan kernel on matrices that need row interchanges: a zero
    leading entry and a scaled permutation matrix (an interchange at nearly
    every step), against the oracle's LU solves and X A = I; sizes below,
    at and above one row per block of the cooperative grid, several rows per
    block and a ragged last batch."""
    rng = np.random.default_rng(M)
    A = rng.standard_normal((M, M))
    A[0, 0] = 0.0 if M > 1 else A[0, 0]
    X = ms.ms_dense_inverse(ctx, A)
    LU, piv = O.lu(A)
    E = np.eye(M)
    ks = range(M) if M <= 160 else rng.choice(M, 40, replace=False)
    cond = np.linalg.cond(A)
    for j in ks:
        xr = O.lu_solve(LU, piv, E[:, j])
        assert np.linalg.norm(X[:, j] - xr) <= 1e-13 * cond * np.linalg.norm(xr)
    assert np.abs(X @ A - E).max() <= 1e-13 * cond
    perm = rng.permutation(M)
    d = rng.uniform(1.0, 4.0, M)
    Pm = np.zeros((M, M))
    Pm[np.arange(M), perm] = d
    Xp = ms.ms_dense_inverse(ctx, Pm)
    ref = np.zeros((M, M))
    ref[perm, np.arange(M)] = 1.0 / d
    np.testing.assert_allclose(Xp, ref, rtol=1e-15, atol=0)


def test_gauss_jordan_singular_is_reported(ms, ctx):
    A = np.ones((6, 6))
    with pytest.raises(ms.MsError) as e:
        ms.ms_dense_inverse(ctx, A)
    assert e.value.status == ms.MS_ERR_COARSE_SINGULAR
    X = ms.ms_dense_inverse(ctx, np.eye(6) * 2.0)      # the context and barrier stay usable
    np.testing.assert_array_equal(X, np.eye(6) * 0.5)
