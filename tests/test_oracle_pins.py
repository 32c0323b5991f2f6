"""Pins of the CPU oracle against things other than itself.

Each test checks an oracle routine against a closed form, an invariant the
paper states, a hand-worked example (tests/golden/hand_worked.json), or a
library routine (numpy / scipy) computing the plain definition.  A mistake
anywhere in the oracle (a dropped term, a wrong sign or index, a transposed
operand) should fail at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2001_01624_gb300 import geomodel as G

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")))


def _grid(nx, ny, nz, inactive=None):
    g = G.Grid(nx, ny, nz, 3.0, 2.0, 0.5)
    if inactive:
        a = np.ones(g.N, np.uint8)
        a[list(inactive)] = 0
        g.active = a
    return g


def _perm(N, k=1.0):
    return np.full((N, 3), k)


# ----------------------------------------------------------------------------- TPFA (Sec. 3, Eq. (9))
def test_tpfa_two_cells_harmonic_mean():
    g = _grid(2, 1, 1)
    perm = np.array([[2.0, 7.0, 7.0], [5.0, 7.0, 7.0]])
    s = O.assemble_tpfa(g, perm)
    area, h = g.dy * g.dz, g.dx
    T = 2.0 * area * 2.0 * 5.0 / (h * (2.0 + 5.0))     # harmonic mean by hand
    np.testing.assert_allclose(s.A.dense(), [[T, -T], [-T, T]], rtol=1e-15)


def test_tpfa_axes_multiplier_and_removed_face():
    g = _grid(1, 2, 2)
    perm = np.array([[1.0, 3.0, 4.0]] * 4)
    g.mult_y = np.array([0.5, 0.0])   # y-face at k=0 halved, at k=1 removed
    s = O.assemble_tpfa(g, perm)
    Ty = 3.0 * (g.dx * g.dz) / g.dy                  # equal cells: t/2 = K * area / h
    Tz = 4.0 * (g.dx * g.dy) / g.dz
    expect = np.array([[Ty + Tz, -Ty, -Tz, 0], [-Ty, Ty + Tz, 0, -Tz], [-Tz, 0, Tz, 0], [0, -Tz, 0, Tz]])
    expect[0, 1] = expect[1, 0] = -0.5 * Ty
    expect[0, 0] = 0.5 * Ty + Tz
    expect[1, 1] = 0.5 * Ty + Tz
    np.testing.assert_allclose(s.A.dense(), expect, rtol=1e-14)


def test_tpfa_nnc_and_inactive():
    # 1x1x3 column: face 0-1 removed, NNC 0-2 along z; cell 1 inactive-free
    g = _grid(1, 1, 3)
    g.mult_z = np.array([0.0, 1.0])
    g.nnc = np.array([[0, 2]], np.int32)
    g.nnc_axis = np.array([2], np.int8)
    g.nnc_mult = np.array([0.25])
    perm = np.array([[1, 1, 2.0], [1, 1, 2.0], [1, 1, 6.0]])
    s = O.assemble_tpfa(g, perm)
    a = g.dx * g.dy
    t = lambda k: k * a / (0.5 * g.dz)
    T12 = 1.0 / (1 / t(2.0) + 1 / t(6.0))
    T02 = 0.25 / (1 / t(2.0) + 1 / t(6.0))
    expect = np.array([[T02, 0, -T02], [0, T12, -T12], [-T02, -T12, T02 + T12]])
    np.testing.assert_allclose(s.A.dense(), expect, rtol=1e-14)
    # inactive middle cell: the two others are disconnected
    g2 = _grid(3, 1, 1, inactive=[1])
    s2 = O.assemble_tpfa(g2, _perm(3))
    assert s2.A.n == 2 and list(s2.cells) == [0, 2]
    np.testing.assert_array_equal(s2.A.dense(), np.zeros((2, 2)))


def test_tpfa_row_sums_zero_and_symmetric():
    gm = G.faulted(16, 12, 6, seed=3, n_fault_x=1, n_fault_y=1, block=(4, 4, 2))
    s = O.assemble_tpfa(gm.grid, gm.perm)
    A = s.A.dense()
    assert np.abs(A - A.T).max() == 0.0
    assert np.abs(A.sum(1)).max() <= 1e-12 * np.abs(A).max()
    assert (np.diag(A) > 0).all() and (A - np.diag(np.diag(A)) <= 0).all()


def test_tpfa_rejects_negative_or_nan_perm():
    g = _grid(2, 1, 1)
    for bad in (-1.0, np.nan):
        p = _perm(2)
        p[1, 0] = bad
        with pytest.raises(O.OracleError):
            O.assemble_tpfa(g, p)


def test_tpfa_upstream_mobility():
    g = _grid(3, 1, 1)
    s0 = O.assemble_tpfa(g, _perm(3))
    lam = np.array([2.0, 3.0, 5.0])
    s1 = O.assemble_tpfa(g, _perm(3), lam=lam, p_prev=np.array([3.0, 2.0, 2.0]))
    T = -s0.A.dense()[0, 1]
    A1 = s1.A.dense()
    assert A1[0, 1] == pytest.approx(-2.0 * T)            # p0 > p1: upstream cell 0
    assert A1[1, 2] == pytest.approx(-0.5 * (3.0 + 5.0) * T)   # tie: mean


# ----------------------------------------------------------------------------- solve pins
def _dense_pinned_solve(Ap, qp):
    return np.linalg.solve(Ap.dense(), qp)


def test_1d_closed_form():
    """Homogeneous column, q = +1 / -1 at the ends, p_0 = 0 => p_i = -i / T."""
    n = 23
    gm = G.homogeneous(n, 1, 1, block=(5, 1, 1))
    gm.q[:] = 0
    gm.q[0], gm.q[-1] = 1.0, -1.0
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm, tol=1e-8, max_iter=20000)
    T = -sysm.A.dense()[0, 1]
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-12, max_iter=500)
    assert r.converged
    np.testing.assert_allclose(r.x, -np.arange(n) / T, rtol=1e-9, atol=1e-9 * n / T)


def test_pin_equals_neumann_shift():
    gm = G.lognormal_box(9, 7, 1, seed=4, block=(3, 3, 1))
    s = O.assemble_tpfa(gm.grid, gm.perm)
    q = gm.q_active()
    Ap, qp = O.pin(s.A, q, 0)
    x = _dense_pinned_solve(Ap, qp)
    xn = np.linalg.lstsq(s.A.dense(), q, rcond=None)[0]
    np.testing.assert_allclose(x, xn - xn[0], rtol=1e-9, atol=1e-9 * np.abs(x).max())


@pytest.mark.parametrize("case", ["2d", "3d", "faulted"])
def test_ms_solve_matches_direct_solve(case):
    if case == "2d":
        gm = G.lognormal_box(12, 8, 1, seed=1, block=(4, 4, 1))
    elif case == "3d":
        gm = G.lognormal_box(10, 10, 4, seed=2, block=(5, 5, 2), kz_ratio=0.1)
    else:
        gm = G.faulted(14, 12, 6, seed=5, n_fault_x=1, n_fault_y=1, block=(5, 4, 3))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-11, max_iter=3000)
    assert r.converged
    x = _dense_pinned_solve(Ap, qp)
    assert np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)


def test_jacobi_smoother_converges_to_direct():
    gm = G.lognormal_box(10, 8, 1, seed=6, sigma=1.0, block=(5, 4, 1))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-11, max_iter=20000, smoother="jacobi")
    assert r.converged
    x = _dense_pinned_solve(Ap, qp)
    assert np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)


def test_identity_partition_converges_in_one_cycle():
    gm = G.lognormal_box(6, 5, 2, seed=7, block=(1, 1, 1))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    assert B.M == Ap.n
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-12, max_iter=10)
    assert r.iters == 1 and r.converged


@pytest.mark.parametrize("case", ["3d", "faulted"])
@pytest.mark.parametrize("restart", [30, 4])
def test_gmres_matches_direct_solve(case, restart):
    """Restarted GMRES with the multistage cycle as right preconditioner
    reaches the pinned system's unique solution (also with restarts every 4
    steps)."""
    if case == "3d":
        gm = G.lognormal_box(10, 10, 4, seed=2, block=(5, 5, 2), kz_ratio=0.1)
    else:
        gm = G.faulted(14, 12, 6, seed=5, n_fault_x=1, n_fault_y=1, block=(5, 4, 3))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    r = O.ms_gmres(Ap, [(B, L)], qp, tol=1e-11, max_iter=3000, restart=restart)
    assert r.converged
    x = _dense_pinned_solve(Ap, qp)
    assert np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)
    assert r.hist[-1] <= 1e-11
    assert abs(np.linalg.norm(qp - Ap.dense() @ r.x) / np.linalg.norm(qp) - r.hist[-1]) <= 1e-12


def test_gmres_residual_monotone_within_restart_and_true_at_restart():
    """Within one restart the GMRES residual (least-squares minimum over a
    growing Krylov space) cannot increase; with no restart it ends at the true
    residual of the iterate."""
    gm = G.lognormal_box(12, 10, 3, seed=8, block=(4, 5, 3), kz_ratio=0.1)
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    r = O.ms_gmres(Ap, [(B, L)], qp, tol=1e-10, max_iter=200, restart=200)
    assert r.converged
    assert np.all(np.diff(r.hist) <= 1e-14)
    rr = np.linalg.norm(qp - Ap.dense() @ r.x) / np.linalg.norm(qp)
    assert abs(rr - r.hist[-1]) <= 1e-12


def test_gmres_exact_preconditioner_converges_in_one_step():
    """With one coarse block per cell the cycle is an exact solve, so the
    preconditioned operator is the identity and one Arnoldi step suffices."""
    gm = G.lognormal_box(6, 5, 2, seed=7, block=(1, 1, 1))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    r = O.ms_gmres(Ap, [(B, L)], qp, tol=1e-12, max_iter=10)
    assert r.iters == 1 and r.converged


def test_gmres_needs_no_more_steps_than_richardson_cycles():
    """Richardson's iterate after k cycles lies in the same preconditioned
    Krylov space GMRES minimises over (without restarts), so GMRES needs at
    most as many steps."""
    gm = G.lognormal_box(14, 12, 4, seed=9, block=(7, 6, 2), kz_ratio=0.1)
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    r1 = O.ms_solve(Ap, [(B, L)], qp, tol=1e-8, max_iter=3000)
    r2 = O.ms_gmres(Ap, [(B, L)], qp, tol=1e-8, max_iter=3000, restart=3000)
    assert r1.converged and r2.converged
    assert r2.iters <= r1.iters


def test_coarse_stage_does_not_increase_energy_error():
    """x + P A_c^-1 P^T (q - A x) is the A-orthogonal projection: ||e||_A
    never grows (Eq. (10), Galerkin restriction)."""
    gm = G.lognormal_box(12, 10, 2, seed=8, block=(4, 5, 1))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    A = Ap.dense()
    xs = np.linalg.solve(A, qp)
    P = B.dense(Ap.n)
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.standard_normal(Ap.n) * np.abs(xs).max()
        e0 = x - xs
        xc = O.cholesky_solve(L, P.T @ (qp - A @ x))
        e1 = x + P @ xc - xs
        assert e1 @ A @ e1 <= e0 @ A @ e0 * (1 + 1e-12)
        assert np.abs(P.T @ (qp - A @ (x + P @ xc))).max() <= 1e-9 * np.abs(P.T @ qp).max() + 1e-30


def test_multistage_and_adaptive_converge_to_direct():
    gm = G.faulted(16, 14, 6, seed=9, n_fault_x=1, n_fault_y=1, block=(4, 4, 3))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    ps, Ms = O.partition_static(sysm.A, B.part, gm.facies[sysm.cells])
    sp, sc = O.support_hop(gm.grid, sysm.cells, sysm.A, ps, Ms)
    B2 = O.msrsb_basis(sysm.A, ps, Ms, sp, sc)
    L2 = O.cholesky(O.galerkin(Ap, B2))
    x = _dense_pinned_solve(Ap, qp)
    r = O.ms_solve(Ap, [(B, L), (B2, L2)], qp, tol=1e-10, max_iter=3000)
    assert r.converged and np.linalg.norm(r.x - x) <= 1e-7 * np.linalg.norm(x)
    ra = O.ms_solve(Ap, [(B, L), (B2, L2)], qp, tol=1e-10, max_iter=3000,
                    adapt=dict(schedule=2, grid=gm.grid, cells=sysm.cells, A_unpinned=sysm.A))
    assert ra.converged and np.linalg.norm(ra.x - x) <= 1e-7 * np.linalg.norm(x)
    assert ra.md_hist[0] == 0 and ra.md_hist[1] > 0
    ra1 = O.ms_solve(Ap, [(B, L)], qp, tol=1e-10, max_iter=3000,
                     adapt=dict(schedule=1, smoothed=1, grid=gm.grid, cells=sysm.cells, A_unpinned=sysm.A))
    assert ra1.converged and np.linalg.norm(ra1.x - x) <= 1e-7 * np.linalg.norm(x)


# ----------------------------------------------------------------------------- MsRSB (Sec. 5, 5.1)
def _setup_basis(gm, tol=1e-3, max_iter=500):
    s = O.assemble_tpfa(gm.grid, gm.perm)
    part, M = O.partition_cartesian(gm.grid, s.cells, gm.block)
    sp, sc = O.support_box(gm.grid, s.cells, s.A, part, M, gm.block)
    return s, O.msrsb_basis(s.A, part, M, sp, sc, tol=tol, max_iter=max_iter)


def test_basis_partition_of_unity_confinement_nonnegative():
    gm = G.lognormal_box(20, 24, 5, seed=11, block=(5, 6, 2), kz_ratio=0.1)
    for it in (1, 3, 40):
        s, B = _setup_basis(gm, tol=0.0, max_iter=it)
        assert B.iters == it
        P = B.dense(s.A.n)
        assert np.abs(P.sum(1) - 1).max() <= 1e-12            # requirement 3
        assert (B.pval >= 0).all()                              # M-matrix + omega < 1
        for j in range(B.M):                                    # requirement 2
            S = set(B.scells[B.sptr[j]:B.sptr[j + 1]].tolist())
            assert set(np.flatnonzero(B.part == j).tolist()) <= S
            outside = np.setdiff1d(np.arange(s.A.n), list(S))
            assert np.all(P[outside, j] == 0.0)


def test_basis_converges_to_closed_form_hat_1d():
    gm = G.homogeneous(20, 1, 1, block=(10, 1, 1))
    s, B = _setup_basis(gm, tol=1e-14, max_iter=100000)
    P = B.dense(s.A.n)
    i = np.arange(20)
    np.testing.assert_allclose(P[:, 0], np.clip((15 - i) / 11, 0, 1), atol=1e-12)
    np.testing.assert_allclose(P[:, 1], 1 - np.clip((15 - i) / 11, 0, 1), atol=1e-12)


def test_basis_converges_to_tensor_hat_3d():
    gm = G.homogeneous(20, 40, 4, block=(10, 20, 2))
    s, B = _setup_basis(gm, tol=1e-13, max_iter=200000)
    P = B.dense(s.A.n)
    hx = np.clip((15 - np.arange(20)) / 11, 0, 1)
    hy = np.clip((30 - np.arange(40)) / 21, 0, 1)
    hz = np.clip((3 - np.arange(4)) / 3, 0, 1)
    for j, (fx, fy, fz) in enumerate([(hx, hy, hz), (1 - hx, hy, hz), (hx, 1 - hy, hz), (1 - hx, 1 - hy, hz),
                                      (hx, hy, 1 - hz)]):
        T = (fz[:, None, None] * fy[None, :, None] * fx[None, None, :]).ravel()
        assert np.abs(P[:, j] - T).max() <= 1e-9


def test_basis_constant_reproduction_and_galerkin():
    gm = G.lognormal_box(16, 12, 3, seed=12, block=(4, 4, 3))
    s, B = _setup_basis(gm)
    P = B.dense(s.A.n)
    A = s.A.dense()
    np.testing.assert_allclose(P @ np.ones(B.M), 1.0, atol=1e-12)
    assert np.abs(A @ np.ones(s.A.n)).max() <= 1e-12 * np.abs(A).max()
    Acu = O.galerkin(s.A, B)
    assert np.abs(Acu @ np.ones(B.M)).max() <= 1e-12 * np.abs(Acu).max()
    np.testing.assert_allclose(Acu, P.T @ A @ P, rtol=1e-12, atol=1e-12 * np.abs(Acu).max())
    Ap, _ = O.pin(s.A, None, 0)
    Ac = O.galerkin(Ap, B)
    assert np.abs(Ac - Ac.T).max() <= 1e-12 * np.abs(Ac).max()
    assert np.linalg.eigvalsh(Ac).min() > 0
    np.testing.assert_allclose(Ac, P.T @ Ap.dense() @ P, rtol=1e-12, atol=1e-12 * np.abs(Ac).max())


def _csr_from_rows(rows):
    A = np.array(rows, dtype=np.float64)
    n = A.shape[0]
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0.0 or i == j:
                ci.append(j)
                v.append(A[i, j])
        rp.append(len(ci))
    return O.CSR(n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(v))


def _frac(pairs):
    return np.array([a / b for a, b in pairs])


def _basis_from_support(part, supports):
    sptr = np.cumsum([0] + [len(s) for s in supports]).astype(np.int32)
    return sptr, np.concatenate([np.asarray(s, np.int32) for s in supports])


def test_msrsb_iterations_hand_worked():
    """One and two MsRSB iterations against the hand derivation
    (tests/golden/hand_worked.json: omega = 2/3, update from the old values,
    then renormalisation of every cell); a wrong omega, a Gauss-Seidel update
    or a missing renormalisation each changes these values."""
    gd = GOLD["msrsb_two_iterations_1d"]
    A = _csr_from_rows(gd["A_rows"])
    sptr, sc = _basis_from_support(gd["part"], gd["supports"])
    omega = gd["omega"][0] / gd["omega"][1]
    for k, key in ((1, "expected_iter1"), (2, "expected_iter2")):
        B = O.msrsb_basis(A, gd["part"], 2, sptr, sc, omega=omega, tol=0.0, max_iter=k)
        assert B.iters == k
        for j in range(2):
            ev = gd[key][j]
            want = _frac(list(zip(ev[0::2], ev[1::2])))
            np.testing.assert_allclose(B.pval[sptr[j]:sptr[j + 1]], want, rtol=0, atol=1e-15)
        np.testing.assert_allclose(B.inc_hist, _frac(gd["expected_increments"][:k]), rtol=0, atol=1e-15)
    # the stopping test: the increment of iteration 2 (4/81 = 0.0494) is below 0.05, not below 0.04
    assert O.msrsb_basis(A, gd["part"], 2, sptr, sc, omega=omega, tol=0.05, max_iter=50).iters == 2
    assert O.msrsb_basis(A, gd["part"], 2, sptr, sc, omega=omega, tol=0.04, max_iter=50).iters > 2


def test_ms_cycle_stage_order_hand_worked():
    """First Richardson cycle of the multistage iteration (Eq. (11)) against
    the hand derivation on a four-cell ring whose ILU(0) drops fill: the
    ILU(0) step comes before each stage's coarse correction.  Post-smoothing
    or the coarse correction first gives other iterates."""
    gd = GOLD["ms_cycle_ring4"]
    A = _csr_from_rows(gd["A_rows"])
    q = np.array(gd["q"], np.float64)
    lu = O.ilu0(A)
    np.testing.assert_allclose(O.ilu0_apply(A, lu, q), _frac(gd["expected_smoothed_x_stage1"]), rtol=0,
                               atol=1e-15)
    stages = []
    for part in gd["stage_parts"]:
        B = O.constant_basis(part, 2)
        Ac = O.galerkin(A, B)
        np.testing.assert_array_equal(Ac, np.array(gd["expected_Ac"], np.float64))
        stages.append((B, O.cholesky(Ac)))
    for ns, xk, rk in ((1, "expected_x_one_stage", "expected_res_one_stage"),
                       (2, "expected_x_two_stages", "expected_res_two_stages")):
        r = O.ms_solve(A, stages[:ns], q, tol=0.0, max_iter=1, lu=lu)
        assert r.iters == 1 and not r.converged
        np.testing.assert_allclose(r.x, _frac(gd[xk]), rtol=0, atol=1e-15)
        assert r.hist[1] == pytest.approx(gd[rk][0] / gd[rk][1], rel=1e-13)
    # the same cycle as the preconditioner of GMRES: its first step from
    # x = 0 is the minimal-residual multiple of the one-stage cycle applied to q
    z = _frac(gd["expected_x_one_stage"])
    Az = A.dense() @ z
    alpha = (Az @ q) / (Az @ Az)
    g = O.ms_gmres(A, stages[:1], q, tol=0.0, max_iter=1, restart=30, lu=lu)
    np.testing.assert_allclose(g.x, alpha * z, rtol=1e-13)


# ----------------------------------------------------------------------------- partitions & supports
def _chain(nx, ny=1, nz=1):
    g = _grid(nx, ny, nz)
    return g, O.assemble_tpfa(g, _perm(g.N))


def test_support_box_golden():
    gd = GOLD["support_box_1d"]
    g, s = _chain(*gd["grid"])
    part, M = O.partition_cartesian(g, s.cells, gd["block"])
    sp, sc = O.support_box(g, s.cells, s.A, part, M, gd["block"])
    assert [sc[sp[j]:sp[j + 1]].tolist() for j in range(M)] == gd["expected"]


def test_support_box_respects_reachability():
    # 4x1x2 grid, block 2x1x2: without the z-face at x=2 and with the x-face
    # between x=1 and x=2 removed, cell (2,0,0) is unreachable from block 0
    g = _grid(4, 1, 2)
    g.mult_x = np.array([1.0, 0.0, 1.0, 1.0, 1.0, 1.0])
    g.mult_z = np.array([1.0, 1.0, 0.0, 1.0])
    s = O.assemble_tpfa(g, _perm(g.N))
    part, M = O.partition_cartesian(g, s.cells, (2, 1, 2))
    sp, sc = O.support_box(g, s.cells, s.A, part, M, (2, 1, 2))
    S0 = sc[sp[0]:sp[1]].tolist()
    assert S0 == [0, 1, 4, 5, 6]       # (2,0,1)=6 reachable via (1,0,1)=5; (2,0,0)=2 is not


@pytest.mark.parametrize("key", ["support_hop_1d", "support_hop_2d"])
def test_support_hop_golden(key):
    gd = GOLD[key]
    g, s = _chain(*gd["grid"])
    part, M = O.partition_cartesian(g, s.cells, gd["block"])
    sp, sc = O.support_hop(g, s.cells, s.A, part, M)
    assert [sc[sp[j]:sp[j + 1]].tolist() for j in range(M)] == gd["expected"]


@pytest.mark.parametrize("key", ["dynamic_1d", "dynamic_2d"])
def test_dynamic_partition_golden(key):
    gd = GOLD[key]
    g, s = _chain(*gd["grid"])
    part, M = O.partition_dynamic(s.A, np.array(gd["dp"]), gd["n_bins"], gd["eps"])
    assert part.tolist() == gd["expected_part"] and M == gd["expected_M"]


def test_dynamic_partition_zero_update_is_connected_components():
    g, s = _chain(6, 2)
    part, M = O.partition_dynamic(s.A, np.zeros(12))
    assert M == 1 and (part == 0).all()


def test_static_partition_golden():
    gd = GOLD["static_2d"]
    g, s = _chain(*gd["grid"])
    part, M = O.partition_cartesian(g, s.cells, gd["block"])
    ps, Ms = O.partition_static(s.A, part, np.array(gd["facies"]))
    assert ps.tolist() == gd["expected_part"] and Ms == gd["expected_M"]


def test_cartesian_partition_ragged_golden():
    gd = GOLD["cartesian_ragged"]
    g = _grid(*gd["grid"], inactive=gd["inactive"])
    s = O.assemble_tpfa(g, _perm(g.N))
    part, M = O.partition_cartesian(g, s.cells, gd["block"])
    assert part.tolist() == gd["expected_part"] and M == gd["expected_M"]


def test_components_match_scipy():
    from scipy.sparse.csgraph import connected_components
    gm = G.lognormal_box(13, 11, 3, seed=13)
    s = O.assemble_tpfa(gm.grid, gm.perm)
    cls = (np.log(gm.perm[:, 0]) > np.median(np.log(gm.perm[:, 0]))).astype(np.int32)
    part, M = O.components(s.A, cls)
    A = s.A.to_scipy().tocoo()
    keep = cls[A.row] == cls[A.col]
    from scipy.sparse import coo_matrix
    G2 = coo_matrix((np.ones(keep.sum()), (A.row[keep], A.col[keep])), shape=A.shape)
    nc, lab = connected_components(G2, directed=False)
    assert M == nc
    # same grouping, and numbering by lowest cell index
    first = {}
    for i, l in enumerate(lab):
        first.setdefault(l, len(first))
    np.testing.assert_array_equal(part, [first[l] for l in lab])


# ----------------------------------------------------------------------------- dense coarse algebra
def test_cholesky_solve_matches_numpy():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((40, 40))
    A = X @ X.T + 40 * np.eye(40)
    L = O.cholesky(A)
    np.testing.assert_allclose(L @ L.T, A, rtol=1e-12, atol=1e-12 * np.abs(A).max())
    b = rng.standard_normal(40)
    np.testing.assert_allclose(O.cholesky_solve(L, b), np.linalg.solve(A, b), rtol=1e-10)
    with pytest.raises(O.OracleError):
        O.cholesky(-np.eye(3))


# ----------------------------------------------------------------------------- ILU(0)
def _lu_dense(A, lu):
    LU = O.CSR(A.n, A.rowptr, A.col, lu).dense()
    return np.tril(LU, -1) + np.eye(A.n), np.triu(LU)


@pytest.mark.parametrize("shape", [(9, 7, 1), (6, 5, 4)])
def test_ilu0_defining_property(shape):
    """ILU(0): (L U)_ij = A_ij for every (i, j) in the pattern of A."""
    gm = G.faulted(*shape, seed=14, n_fault_x=1, n_fault_y=0, throw=1, inactive_pct=10.0) if shape[2] > 1 \
        else G.lognormal_box(*shape, seed=14)
    s = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, _ = O.pin(s.A, None, 0)
    lu = O.ilu0(Ap)
    Lm, Um = _lu_dense(Ap, lu)
    A = Ap.dense()
    mask = O.CSR(Ap.n, Ap.rowptr, Ap.col, np.ones_like(Ap.val)).dense() > 0
    np.testing.assert_allclose((Lm @ Um)[mask], A[mask], rtol=1e-12, atol=1e-12 * np.abs(A).max())
    r = np.random.default_rng(0).standard_normal(Ap.n)
    np.testing.assert_allclose(O.ilu0_apply(Ap, lu, r), np.linalg.solve(Lm @ Um, r), rtol=1e-9)


def test_ilu0_exact_on_tridiagonal():
    gm = G.lognormal_box(30, 1, 1, seed=15, block=(5, 1, 1))
    s = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(s.A, gm.q_active(), 0)
    z = O.ilu0_apply(Ap, O.ilu0(Ap), qp)
    np.testing.assert_allclose(z, np.linalg.solve(Ap.dense(), qp), rtol=1e-11)


# ----------------------------------------------------------------------------- cost model (Eq. (12))
@pytest.mark.parametrize("N,Np,d,b,Nc", [(1e6, 1, 7, 8, 1), (78720, 6, 15, 8, 3), (1000, 3, 5, 4, 2)])
def test_cost_model_is_sum_of_itemised_counts(N, Np, d, b, Nc):
    smooth = 2 * N * d + (N * d + N) + N          # two triangular solves, residual, update
    restrict = (N * d + N) + b * N                 # residual + R
    prolong = b * N + N                            # P x_c + update
    predictor = Np * (smooth + restrict + prolong)
    residual_update = Nc * N * d + Nc * N
    corrector = 2 * d * Nc ** 2 * N + Nc * N
    assert O.cost_model(N, Np, d, b, Nc) == pytest.approx(predictor + residual_update + corrector, rel=1e-14)


# ------------------------------------------------------------- two-phase
def test_total_mobility_closed_forms():
    lam = O.total_mobility([0.0, 1.0, 0.5], dict(mu_w=1.0, mu_o=3.0))
    np.testing.assert_allclose(lam, [1.0 / 3.0, 1.0, 0.25 + 0.25 / 3.0], rtol=1e-15)
    # residual saturations: Se clipped, so S <= s_wc is immobile water
    lam = O.total_mobility([0.1, 0.95], dict(mu_w=2.0, mu_o=4.0, s_wc=0.2, s_or=0.1))
    np.testing.assert_allclose(lam, [0.25, 0.5], rtol=1e-15)


def _pressure(gm, lam, p_prev=None):
    sysm = O.assemble_tpfa(gm.grid, gm.perm, lam=lam, p_prev=p_prev)
    Ap, qp = O.pin(sysm.A, gm.q_active(), 0)
    return sysm, np.linalg.solve(Ap.dense(), qp)


def test_transport_keeps_pure_water_and_bounds():
    """A divergence-free total flux carries S = 1 unchanged (f_w = 1 and the
    pressure solution balances every cell); from any S in [0, 1] the monotone
    upstream scheme under the CFL limit stays in [0, 1]."""
    gm = G.lognormal_box(9, 7, 3, seed=4, block=(3, 7, 3), kz_ratio=0.1)
    n = gm.grid.n_active()
    q = gm.q_active() * 1e-3
    gm.q[:] = 0
    gm.q[gm.grid.active_cells()] = q
    S = np.ones(n)
    sysm, p = _pressure(gm, O.total_mobility(S))
    vol = gm.grid.dx * gm.grid.dy * gm.grid.dz
    S1, k = O.transport_step(sysm.A, p, q, S, dt=50.0 * vol / np.abs(q).sum(), volume=vol)
    assert k > 1
    np.testing.assert_allclose(S1, 1.0, atol=1e-9)
    S = np.random.default_rng(3).uniform(0, 1, n)
    sysm, p = _pressure(gm, O.total_mobility(S), p_prev=np.random.default_rng(4).standard_normal(n))
    S1, k = O.transport_step(sysm.A, p, q, S, dt=20.0 * vol / np.abs(q).sum(), volume=vol)
    assert S1.min() >= -1e-12 and S1.max() <= 1 + 1e-12


def test_transport_buckley_leverett_front():
    """1D water flood (mu_w = 1, mu_o = 3, Corey n = 2, no residuals): the
    saturation front moves at f_w'(S_f) times the injected pore volumes, S_f
    the Welge tangent point f_w(S_f) / S_f = f_w'(S_f) (Buckley-Leverett).
    The upstream scheme's smeared front brackets that position."""
    n = 800
    gm = G.homogeneous(n, 1, 1, block=(10, 1, 1))
    gm.q[:] = 0
    gm.q[0], gm.q[n - 1] = 1e-3, -1e-3
    q = gm.q_active()
    vol = gm.grid.dx * gm.grid.dy * gm.grid.dz
    phi = 0.2
    S = np.zeros(n)
    pvi = 0.3
    dt_total = pvi * phi * vol * n / 1e-3
    for _ in range(6):                       # sequential steps (the 1D total flux is q whatever lambda is)
        sysm, p = _pressure(gm, O.total_mobility(S))
        S, _ = O.transport_step(sysm.A, p, q, S, dt=dt_total / 6, porosity=phi, volume=vol)
    fw = lambda s: s * s / (s * s + (1 - s) ** 2 / 3.0)
    ss = np.linspace(0.3, 0.9, 600001)
    d = (fw(ss + 1e-7) - fw(ss - 1e-7)) / 2e-7
    sf = ss[np.argmin(np.abs(fw(ss) / ss - d))]
    dfs = (fw(sf + 1e-7) - fw(sf - 1e-7)) / 2e-7
    x_front = dfs * pvi                      # fraction of the column
    cross = np.argmax(S < 0.5 * sf) / n
    assert abs(cross - x_front) < 0.03, (cross, x_front, sf)
    # mass balance: water in place = water injected (nothing produced yet)
    assert abs(S.sum() * phi * vol - 1e-3 * dt_total) <= 1e-9 * 1e-3 * dt_total


# ----------------------------------------------------------------------------- finite-volume restriction (Sec. 5)
def test_fv_operator_annihilates_constants():
    """A_c = R A P with R the block indicator: A_c 1 = R A P 1 = R A 1 = 0 and,
    A being symmetric, 1^T A_c = 1^T A P = (A 1)^T P = 0 (unpinned A)."""
    gm = G.lognormal_box(16, 12, 3, seed=12, block=(4, 4, 3))
    s, B = _setup_basis(gm)
    Ac = O.galerkin_fv(s.A, B)
    scale = np.abs(Ac).max()
    assert np.abs(Ac @ np.ones(B.M)).max() <= 1e-12 * scale
    assert np.abs(np.ones(B.M) @ Ac).max() <= 1e-12 * scale
    assert np.abs(Ac - Ac.T).max() > 1e-6 * scale          # not the Galerkin operator: not symmetric


def test_fv_operator_constant_basis_closed_form():
    """With the indicator basis P = R^T, R A P = P^T A P, and off the
    diagonal -A_c(j, l) is the sum of the transmissibilities of the faces
    between blocks j and l, the diagonal the sum over the faces leaving j."""
    gm = G.faulted(12, 10, 4, seed=3, n_fault_x=1, n_fault_y=1, block=(4, 5, 2))
    s = O.assemble_tpfa(gm.grid, gm.perm)
    part, M = O.partition_cartesian(gm.grid, s.cells, gm.block)
    B = O.constant_basis(part, M)
    Ac = O.galerkin_fv(s.A, B)
    fa, fb, ft = s.faces
    ref = np.zeros((M, M))
    for a, b, t in zip(fa, fb, ft):
        ja, jb = part[a], part[b]
        if ja != jb:
            ref[ja, jb] -= t
            ref[jb, ja] -= t
            ref[ja, ja] += t
            ref[jb, jb] += t
    np.testing.assert_allclose(Ac, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(Ac, O.galerkin(s.A, B), rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_lu_factors_and_solve():
    rng = np.random.default_rng(5)
    for M in (1, 2, 7, 40):
        A = rng.standard_normal((M, M))
        if M > 1:
            A[0, 0] = 0.0                          # forces an interchange at the first step
        LU, piv = O.lu(A)
        L = np.tril(LU, -1) + np.eye(M)
        U = np.triu(LU)
        PA = A.copy()
        for k in range(M):
            PA[[k, piv[k]]] = PA[[piv[k], k]]
        np.testing.assert_allclose(L @ U, PA, rtol=1e-12, atol=1e-12 * np.abs(A).max())
        assert np.abs(L).max() <= 1.0 + 1e-15     # partial pivoting bounds the multipliers
        b = rng.standard_normal(M)
        np.testing.assert_allclose(O.lu_solve(LU, piv, b), np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)
    P = np.array([[0.0, 2.0], [3.0, 0.0]])        # needs the interchange; inverse by hand
    LU, piv = O.lu(P)
    assert list(piv) == [1, 1]
    np.testing.assert_allclose(O.lu_solve(LU, piv, np.array([4.0, 9.0])), [3.0, 2.0], rtol=1e-15)
    with pytest.raises(O.OracleError):
        O.lu(np.zeros((3, 3)))


def test_partition_wells_hand_worked():
    part, M = O.partition_wells(10, [[2, 3], [7], [9, 0]])
    assert M == 4
    assert list(part) == [2, 3, 0, 0, 3, 3, 3, 1, 3, 2]
    with pytest.raises(O.OracleError):
        O.partition_wells(10, [[1, 2], [2]])
    with pytest.raises(O.OracleError):
        O.partition_wells(10, [[10]])


@pytest.mark.parametrize("case", ["3d", "faulted"])
def test_fv_cycle_conserves_mass_per_block(case):
    """A cycle that ends with a finite-volume coarse correction leaves a
    residual whose sum over every block is zero: R (q - A x) = R q - A_c x_c
    - R A (x - P x_c) = 0 by construction of x_c (local conservation)."""
    if case == "3d":
        gm = G.lognormal_box(10, 10, 4, seed=2, block=(5, 5, 2), kz_ratio=0.1)
    else:
        gm = G.faulted(14, 12, 6, seed=5, n_fault_x=1, n_fault_y=1, block=(5, 4, 3))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    F = O.coarse_fv(Ap, B)
    for cycles in (1, 3):
        r = O.ms_solve(Ap, [(B, F)], qp, tol=1e-30, max_iter=cycles)
        assert r.iters == cycles
        res = qp - Ap.to_scipy() @ r.x
        sums = np.bincount(B.part, weights=res, minlength=B.M)
        assert np.abs(sums).max() <= 1e-10 * np.abs(res).sum()
        # the Galerkin stage does not conserve: its block sums stay of the residual's size
    rg = O.ms_solve(Ap, [(B, L)], qp, tol=1e-30, max_iter=1)
    resg = qp - Ap.to_scipy() @ rg.x
    assert np.abs(np.bincount(B.part, weights=resg, minlength=B.M)).max() > 1e-6 * np.abs(resg).sum()


@pytest.mark.parametrize("outer", ["richardson", "gmres"])
def test_fv_solve_matches_direct(outer):
    """Richardson with a finite-volume stage is not an energy-norm projection
    and may diverge (it does on the faulted case, spectral radius above one),
    so it is pinned on a lognormal box; GMRES on the faulted grid."""
    if outer == "richardson":
        gm = G.lognormal_box(10, 10, 4, seed=2, block=(5, 5, 2), kz_ratio=0.1)
    else:
        gm = G.faulted(14, 12, 6, seed=5, n_fault_x=1, n_fault_y=1, block=(5, 4, 3))
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    F = O.coarse_fv(Ap, B)
    if outer == "richardson":
        r = O.ms_solve(Ap, [(B, F)], qp, tol=1e-11, max_iter=5000)
    else:
        r = O.ms_gmres(Ap, [(B, F)], qp, tol=1e-11, max_iter=5000, restart=30)
    assert r.converged
    x = _dense_pinned_solve(Ap, qp)
    assert np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)


def test_well_basis_stage_converges_to_direct():
    """Well bases (Sec. 6.2): MsRSB on the partition {cells of each well,
    the rest}, hop supports, as an extra stage beside the general one."""
    gm = G.lognormal_box(14, 12, 3, seed=8, block=(7, 6, 3), kz_ratio=0.1)
    sysm, Ap, qp, B, Ac, L = O.setup_general(gm)
    wells = [np.flatnonzero(qp > 0), np.flatnonzero(qp < 0)]
    part, M = O.partition_wells(Ap.n, [w for w in wells if len(w)])
    sp, sc = O.support_hop(gm.grid, sysm.cells, sysm.A, part, M)
    Bw = O.msrsb_basis(sysm.A, part, M, sp, sc)
    P = Bw.dense(Ap.n)
    assert np.abs(P.sum(1) - 1).max() <= 1e-12
    Lw = O.cholesky(O.galerkin(Ap, Bw))
    r = O.ms_solve(Ap, [(B, L), (Bw, Lw)], qp, tol=1e-11, max_iter=3000)
    assert r.converged
    x = _dense_pinned_solve(Ap, qp)
    assert np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)


# ----------------------------------------------------------------------------- CPR pressure stage (Sec. 4)
def _cpr_case(seed=0, faulted=True):
    gm = (G.faulted(12, 10, 4, seed=seed, n_fault_x=1, n_fault_y=1, block=(4, 5, 2)) if faulted
          else G.lognormal_box(9, 7, 3, seed=seed, block=(3, 7, 3), kz_ratio=0.1))
    sysm = O.assemble_tpfa(gm.grid, gm.perm)
    n = sysm.A.n
    rng = np.random.default_rng(seed + 100)
    p = 2e7 + 1e6 * rng.standard_normal(n)
    s = rng.uniform(0.15, 0.85, n)
    p0 = p - 1e5 * rng.uniform(0.0, 1.0, n)
    s0 = np.clip(s - 0.05 * rng.uniform(0, 1, n), 0.0, 1.0)
    qw = np.zeros(n); qo = np.zeros(n)
    qw[0], qo[n - 1], qw[n - 1] = 0.5, -0.4, -0.1
    g = gm.grid
    return gm, sysm, g.dx * g.dy * g.dz, p, s, p0, s0, qw, qo, 86400.0


def test_cpr_jacobian_matches_finite_differences():
    gm, sysm, vol, p, s, p0, s0, qw, qo, dt = _cpr_case()
    fa, fb, _ = sysm.faces
    gap = np.abs(p[fa] - p[fb]).min()
    hp = 1e-3 * gap
    assert hp > 1e-4                                # no upstream direction changes under the perturbation
    out = O.cpr_pressure(sysm, vol, p, s, p0, s0, qw, qo, dt)
    Jw, Jo = out["Jwp"].dense(), out["Jop"].dense()
    n = sysm.A.n
    fdw, fdo = np.zeros((n, n)), np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n); e[k] = hp
        rwp, rop = O.cpr_residual(sysm, vol, p + e, s, p0, s0, qw, qo, dt)
        rwm, rom = O.cpr_residual(sysm, vol, p - e, s, p0, s0, qw, qo, dt)
        fdw[:, k] = (rwp - rwm) / (2 * hp)
        fdo[:, k] = (rop - rom) / (2 * hp)
    np.testing.assert_allclose(Jw, fdw, rtol=0, atol=1e-6 * np.abs(Jw).max())
    np.testing.assert_allclose(Jo, fdo, rtol=0, atol=1e-6 * np.abs(Jo).max())
    hs = 1e-6
    dsw, dso = np.zeros(n), np.zeros(n)
    for k in range(n):
        e = np.zeros(n); e[k] = hs
        rwp, rop = O.cpr_residual(sysm, vol, p, s + e, p0, s0, qw, qo, dt)
        rwm, rom = O.cpr_residual(sysm, vol, p, s - e, p0, s0, qw, qo, dt)
        dsw[k] = (rwp[k] - rwm[k]) / (2 * hs)
        dso[k] = (rop[k] - rom[k]) / (2 * hs)
    np.testing.assert_allclose(out["Dws"], dsw, rtol=1e-6, atol=1e-9 * np.abs(dsw).max())
    np.testing.assert_allclose(out["Dos"], dso, rtol=1e-6, atol=1e-9 * np.abs(dso).max())


def test_cpr_fluxes_cancel_and_weights_decouple():
    gm, sysm, vol, p, s, p0, s0, qw, qo, dt = _cpr_case(seed=4)
    out = O.cpr_pressure(sysm, vol, p, s, p0, s0, qw, qo, dt)
    # fluxes cancel over the whole grid: sum_i R_a,i = accumulation - sources
    cp = O.CPR_DEFAULT
    e = lambda x: np.exp(x)
    ph, ph0 = cp["phi0"] * e(cp["c_r"] * (p - cp["p_ref"])), cp["phi0"] * e(cp["c_r"] * (p0 - cp["p_ref"]))
    rw, rw0 = cp["rho_w0"] * e(cp["c_w"] * (p - cp["p_ref"])), cp["rho_w0"] * e(cp["c_w"] * (p0 - cp["p_ref"]))
    accw = vol / dt * (ph * rw * s - ph0 * rw0 * s0)
    assert abs(out["Rw"].sum() - (accw.sum() - qw.sum())) <= 1e-9 * np.abs(out["Rw"]).sum()
    # and so do their pressure derivatives: column sums of J_wp are the accumulation derivatives
    Jw = out["Jwp"].dense()
    np.testing.assert_allclose(Jw.sum(0), vol / dt * ph * rw * (cp["c_r"] + cp["c_w"]) * s,
                               rtol=0, atol=1e-9 * np.abs(Jw).max())
    # quasi-IMPES: the weighted saturation diagonal vanishes and the weights sum to one
    np.testing.assert_allclose(out["ww"] + out["wo"], 1.0, rtol=1e-14)
    assert np.abs(out["ww"] * out["Dws"] + out["wo"] * out["Dos"]).max() <= 1e-12 * np.abs(out["Dws"]).max()
    np.testing.assert_allclose(out["rstar"], out["ww"] * out["Rw"] + out["wo"] * out["Ro"], rtol=1e-14)


def test_cpr_incompressible_limit_is_half_total_mobility_tpfa():
    """No compressibility, unit densities, uniform pressure and saturation:
    the saturation diagonals are +-V phi / dt, the weights 1/2, and J* is
    half the TPFA matrix with the total mobility."""
    gm, sysm, vol, p, s, p0, s0, qw, qo, dt = _cpr_case(seed=2)
    n = sysm.A.n
    params = dict(c_w=0.0, c_o=0.0, c_r=0.0, rho_w0=1.0, rho_o0=1.0)
    pu, su = np.full(n, 2e7), np.full(n, 0.4)
    out = O.cpr_pressure(sysm, vol, pu, su, pu, su, np.zeros(n), np.zeros(n), dt, params)
    np.testing.assert_allclose(out["ww"], 0.5, rtol=1e-14)
    lam_t = O.total_mobility(np.array([0.4]), dict(mu_w=1e-3, mu_o=3e-3))[0]
    A = sysm.A.dense()
    np.testing.assert_allclose(out["Jstar"].dense(), 0.5 * lam_t * A, rtol=0, atol=1e-13 * lam_t * np.abs(A).max())
    assert np.abs(out["rstar"]).max() == 0.0


def test_cpr_predictor_solve_matches_direct():
    """The pressure stage of CPR: J* dp = -r* by GMRES with the multistage
    cycle (Galerkin stage of the non-symmetric J*, LU coarse solve)."""
    gm, sysm, vol, p, s, p0, s0, qw, qo, dt = _cpr_case(seed=6)
    out = O.cpr_pressure(sysm, vol, p, s, p0, s0, qw, qo, dt)
    J = out["Jstar"]
    part, M = O.partition_cartesian(gm.grid, sysm.cells, gm.block)
    sp, sc = O.support_box(gm.grid, sysm.cells, sysm.A, part, M, gm.block)
    B = O.msrsb_basis(sysm.A, part, M, sp, sc)
    F = O.coarse_lu(J, B)
    rhs = -out["rstar"]
    r = O.ms_gmres(J, [(B, F)], rhs, tol=1e-11, max_iter=500, restart=30)
    assert r.converged
    x = np.linalg.solve(J.dense(), rhs)
    assert np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)
