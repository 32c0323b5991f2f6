"""Full-size parity in the benchmark's launch configuration.

* 2D 60x220 lognormal geomodel (13,200 cells): GPU and oracle solved in full.
* 3D 60x220x85 geomodel (1,122,000 cells): the GPU pipeline as bench.py runs
  it, against the stored full FP64 oracle run (tests/golden/oracle_c2_seed0.json,
  written by tests/golden/make_oracle_c2.py): basis iterations equal,
  Richardson cycles within +/-1, the first residuals to 1e-6 relative,
  pressure at 4096 seeded sample cells to 1e-6 (FP64) / 1e-5 (mixed), and
  the final residual checked independently with the oracle's matrix.
* 3D faulted 200x200x50 geomodel (1,840,020 active cells), two static stages
  with and without the dynamic stage, against the stored FP64 oracle runs
  (tests/golden/oracle_c3_seed0.json, written by tests/golden/make_oracle_c3.py).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2001_01624_gb300 import geomodel as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_c2_seed0.json")


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2001_01624_gb300 as pkg
    return pkg


GOLD_GMRES = os.path.join(os.path.dirname(__file__), "golden", "oracle_c2_seed0_gmres.json")


def _pipeline(ms, gm, prec, dev, outer=0, restart=30):
    stream = torch.cuda.Stream(dev)
    ctx = ms.ms_create(0, stream)
    s = ms.ms_system_create(ctx, gm.grid, 0)
    perm = torch.from_numpy(gm.perm.ravel().copy()).to(dev)
    ms.ms_assemble_tpfa(ctx, s, perm)
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    b, bit = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
    c = ms.ms_galerkin(ctx, s, b, prec)
    q = torch.from_numpy(gm.q_active()).to(dev)
    p = torch.zeros_like(q)
    info = ms.ms_solve(ctx, s, [c], q, p, tol=1e-6, max_iter=5000, precision=prec, outer=outer, restart=restart)
    torch.cuda.synchronize()
    x = p.cpu().numpy()
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)
    ms.ms_destroy(ctx)
    return x, bit, info


def test_config1_full_size(ms):
    gm = G.config1(0)
    sysr, Ap, qp, B, Ac, L = O.setup_general(gm)
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-6, max_iter=5000)
    x, bit, info = _pipeline(ms, gm, ms.MS_PREC_FP64, torch.device("cuda:0"))
    assert bit == B.iters
    assert info["converged"] and abs(info["iters"] - r.iters) <= 1
    assert np.linalg.norm(x - r.x) <= 1e-6 * np.linalg.norm(r.x)
    xm, _, im = _pipeline(ms, gm, ms.MS_PREC_MIXED, torch.device("cuda:0"))
    assert im["converged"] and abs(im["iters"] - r.iters) <= 1, (im["iters"], r.iters)
    assert np.linalg.norm(xm - r.x) <= 1e-5 * np.linalg.norm(r.x)


@pytest.mark.skipif(not os.path.exists(GOLD), reason="stored oracle run missing")
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config2_full_size_against_stored_oracle(ms, prec):
    g = json.load(open(GOLD))
    gm = G.config2(0)
    P = ms.MS_PREC_FP64 if prec == "fp64" else ms.MS_PREC_MIXED
    x, bit, info = _pipeline(ms, gm, P, torch.device("cuda:0"))
    assert info["converged"]
    idx = np.array(g["sample_cells"])
    ps = np.array(g["p_sample"])
    tol = 1e-6 if prec == "fp64" else 1e-5
    assert np.linalg.norm(x[idx] - ps) <= tol * np.linalg.norm(ps)
    assert abs(info["iters"] - g["cycles"]) <= 1, (info["iters"], g["cycles"])
    if prec == "fp64":
        assert bit == g["basis_iters"]
        k = min(len(g["hist_first"]), len(info["history"]))
        np.testing.assert_allclose(info["history"][:k], g["hist_first"][:k], rtol=1e-6)
    # the final residual, recomputed with the oracle's own matrix
    s = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(s.A, gm.q_active(), 0)
    res = np.linalg.norm(qp - Ap.to_scipy() @ x) / np.linalg.norm(qp)
    assert res <= 1e-6 * (1 + 1e-9)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config2_gmres_full_size_against_stored_oracle(ms, prec):
    """The bench's headline solve: GMRES(30) preconditioned by the multistage
    cycle, against the stored full FP64 oracle GMRES run
    (tests/golden/oracle_c2_seed0_gmres.json): steps within +/-1, the residual
    history of the first restart, sampled pressures, the final residual with
    the oracle's matrix."""
    g = json.load(open(GOLD_GMRES))
    gm = G.config2(0)
    P = ms.MS_PREC_FP64 if prec == "fp64" else ms.MS_PREC_MIXED
    x, bit, info = _pipeline(ms, gm, P, torch.device("cuda:0"), outer=ms.MS_OUTER_GMRES, restart=g["restart"])
    assert info["converged"]
    assert abs(info["iters"] - g["steps"]) <= 1, (info["iters"], g["steps"])
    idx = np.array(g["sample_cells"])
    ps = np.array(g["p_sample"])
    tol = 1e-6 if prec == "fp64" else 1e-5
    assert np.linalg.norm(x[idx] - ps) <= tol * np.linalg.norm(ps)
    if prec == "fp64":
        assert bit == g["basis_iters"]
        k = min(25, len(g["hist"]), len(info["history"]))
        np.testing.assert_allclose(info["history"][:k], g["hist"][:k], rtol=1e-5)
    s = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(s.A, gm.q_active(), 0)
    res = np.linalg.norm(qp - Ap.to_scipy() @ x) / np.linalg.norm(qp)
    assert res <= 1e-6 * (1 + 1e-9)


GOLD_C3 = os.path.join(os.path.dirname(__file__), "golden", "oracle_c3_seed0.json")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config3_faulted_full_size(ms, precision):
    """3D faulted 200x200x50 geomodel (1.84 M active cells, 6 faults with
    2-cell throw as non-neighbour connections): general 10x10x5 stage + the
    facies-split static stage, solved without and with the dynamic stage
    rebuilt after cycles 1 and 2 (Dp(Inf)), against the stored full FP64
    oracle runs (tests/golden/oracle_c3_seed0.json, written by
    tests/golden/make_oracle_c3.py): static block count and basis iterations
    equal, Richardson cycles within +/-1, the first residuals to 1e-5
    relative and the dynamic-stage block counts of the first cycles equal
    (FP64), pressure at 4096 seeded sample cells to 1e-6 (FP64) / 1e-5
    (mixed).  Checked at any size besides: the final residual recomputed with
    the oracle's own assembly of the pinned matrix, the static partition
    against the oracle's, and the partition of unity of both bases on sampled
    cells."""
    import scipy.sparse as sp
    g = json.load(open(GOLD_C3))
    dev = torch.device("cuda:0")
    prec = ms.MS_PREC_FP64 if precision == "fp64" else ms.MS_PREC_MIXED
    gm = G.config3(0)
    cells = gm.grid.active_cells()
    n = len(cells)
    assert n == g["n"]
    stream = torch.cuda.Stream(dev)
    ctx = ms.ms_create(0, stream)
    s = ms.ms_system_create(ctx, gm.grid, 0)
    ms.ms_assemble_tpfa(ctx, s, torch.from_numpy(gm.perm.ravel().copy()).to(dev))
    part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
    assert M == g["M_general"]
    fac = gm.facies[cells].astype(np.int32)
    ps = np.empty(n, np.int32)
    Ms = ms.ms_partition_components(ctx, s, part * 2 + fac, ps)
    assert Ms == g["M_static"]
    b1, it1 = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
    b2, it2 = ms.ms_build_basis(ctx, s, ps, Ms, support=ms.MS_SUPPORT_HOP, precision=prec)
    if precision == "fp64":
        assert (it1, it2) == (g["basis_iters_general"], g["basis_iters_static"])
    c1, c2 = ms.ms_galerkin(ctx, s, b1, prec), ms.ms_galerkin(ctx, s, b2, prec)
    q = torch.from_numpy(gm.q_active()).to(dev)
    ref = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(ref.A, gm.q_active(), 0)
    A = sp.csr_matrix((Ap.val, Ap.col, Ap.rowptr), shape=(n, n))
    idx = np.array(g["sample_cells"])
    tol = 1e-6 if precision == "fp64" else 1e-5
    for key, sched in (("static", 0), ("dp_inf", 2)):
        gs = g["solves"][key]
        p = torch.zeros_like(q)
        info = ms.ms_solve(ctx, s, [c1, c2], q, p, tol=1e-6, max_iter=3000, precision=prec, adapt_schedule=sched)
        torch.cuda.synchronize()
        assert info["converged"]
        assert abs(info["iters"] - gs["cycles"]) <= 1, (key, info["iters"], gs["cycles"])
        x = p.cpu().numpy()
        ps_ = np.array(gs["p_sample"])
        assert np.linalg.norm(x[idx] - ps_) <= tol * np.linalg.norm(ps_), key
        assert np.linalg.norm(qp - A @ x) <= 1.001e-6 * np.linalg.norm(qp)
        if precision == "fp64":
            k = min(25, len(gs["hist_first"]), len(info["history"]))
            np.testing.assert_allclose(info["history"][:k], gs["hist_first"][:k], rtol=1e-5)
            if sched:
                k = min(len(gs["dyn_blocks_first"]), len(info["dyn_blocks"]))
                assert list(info["dyn_blocks"][:k]) == gs["dyn_blocks_first"][:k]
        if sched:
            assert info["dyn_blocks"][0] == 0 and info["dyn_blocks"][2] > 0
    # static partition = the oracle's facies split of the same Cartesian blocks
    rps, rMs = O.partition_static(ref.A, part, gm.facies[cells])
    assert rMs == Ms and np.array_equal(rps, ps)
    rng = np.random.default_rng(0)
    sample = rng.choice(n, 4096, replace=False)
    for b in (b1, b2):
        cptr, cc, cv = ms.ms_basis_get(ctx, b)
        w = np.zeros(n)
        np.add.at(w, cc, cv)
        np.testing.assert_allclose(w[sample], 1.0, atol=1e-12 if precision == "fp64" else 1e-5)
    for h in (c1, c2):
        ms.ms_coarse_release(h)
    for h in (b1, b2):
        ms.ms_basis_release(h)
    ms.ms_system_release(s)
    ms.ms_destroy(ctx)
