"""The OpenMP build of the oracle (used only to time the method on all host
cores) computes what the single-threaded oracle computes: bitwise the same
basis, Galerkin operator, Cholesky factor and Richardson iterate (those loops
only split independent outputs), and the same GMRES result up to the rounding
of its dot products."""
import numpy as np
import pytest

import oracle as O
from paper_2001_01624_gb300 import geomodel as G


@pytest.fixture
def both():
    yield
    O.use_openmp(False)


def _run(gm):
    s = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(s.A, gm.q_active(), 0)
    part, M = O.partition_cartesian(gm.grid, s.cells, gm.block)
    sp, sc = O.support_box(gm.grid, s.cells, s.A, part, M, gm.block)
    B = O.msrsb_basis(s.A, part, M, sp, sc, 2.0 / 3.0, 1e-3, 500)
    Ac = O.galerkin(Ap, B)
    L = O.cholesky(Ac)
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-6, max_iter=500)
    g = O.ms_gmres(Ap, [(B, L)], qp, tol=1e-6, max_iter=500, restart=10)
    return B, Ac, L, r, g


def test_openmp_build_matches_single_thread(both, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    gm = G.lognormal_box(24, 20, 6, seed=7, block=(6, 5, 3), kz_ratio=0.1)
    O.use_openmp(False)
    B1, A1, L1, r1, g1 = _run(gm)
    O.use_openmp(True)
    assert O.openmp_threads() >= 1
    B2, A2, L2, r2, g2 = _run(gm)
    assert B1.iters == B2.iters
    assert np.array_equal(B1.pval, B2.pval)
    assert np.array_equal(A1, A2) and np.array_equal(L1, L2)
    assert r1.iters == r2.iters
    np.testing.assert_allclose(r2.x, r1.x, rtol=1e-12, atol=1e-12 * np.abs(r1.x).max())
    assert abs(g1.iters - g2.iters) <= 1
    np.testing.assert_allclose(g2.x, g1.x, rtol=0, atol=1e-7 * np.abs(g1.x).max())
