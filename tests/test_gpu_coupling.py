"""Coupled two-phase steps with dynamic bases (the coupling-strength study):
the library's sequence of total mobility, upstream assembly, coarse refresh,
adaptive Richardson solve from the previous pressure and upstream transport
against the oracle's, step by step."""
import numpy as np
import pytest

import oracle as O

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


def _oracle_run(gm, ratio, q, dt, steps, schedule, tol, volume):
    from paper_2001_01624_gb300 import coupling as CP
    mu_w, mu_o = CP.viscosities(ratio)
    fl = dict(mu_w=mu_w, mu_o=mu_o, n_w=1.0, n_o=1.0)
    sysr, Ap0, qp0, B, Ac0, L0 = O.setup_general(gm)
    n = sysr.A.n
    p = np.zeros(n)
    S = np.zeros(n)
    cycles = []
    for k in range(steps):
        lam = O.total_mobility(S, fl)
        A = O.assemble_tpfa(gm.grid, gm.perm, lam=lam, p_prev=p if k else None).A
        Ap, qp = O.pin(A, q, 0)
        L = O.cholesky(O.galerkin(Ap, B))
        ad = dict(schedule=schedule, grid=gm.grid, cells=sysr.cells, A_unpinned=A) if schedule else None
        r = O.ms_solve(Ap, [(B, L)], qp, tol=tol, max_iter=5000, x0=p, adapt=ad)
        assert r.converged
        p = r.x
        cycles.append(r.iters)
        S, _ = O.transport_step(A, p, q, S, dt, fluid=fl, porosity=0.2, volume=volume, cfl=0.9)
    return cycles, p, S


@pytest.mark.parametrize("ratio", [10.0, 0.1, 1.0])
@pytest.mark.parametrize("schedule", [0, 1, 2])
def test_coupled_steps_match_oracle(ms, ctx, ratio, schedule):
    from paper_2001_01624_gb300 import coupling as CP
    gm = CP.model(seed=3)
    steps = 6
    run = CP.Run(ctx, gm, CP.fluid_for(ratio), steps=steps, pv=0.3)
    out = run.simulate(schedule)
    cycles, p, S = _oracle_run(gm, ratio, run.q, run.dt, steps, schedule, run.tol, run.volume)
    run.release()
    # Dp(1) rebuilds the dynamic stage after every cycle from binned pressure
    # changes (Sec. 5.1): a rounding-level difference in an iterate can move a
    # cell to another bin and change the next stage, so the library and the
    # oracle take different (both converged) paths and a step's count may
    # differ by two; the pressures and saturations below still agree
    dc = 2 if schedule == 1 else 1
    assert all(abs(a - b) <= dc for a, b in zip(out["cycles"], cycles)), (out["cycles"], cycles)
    assert np.linalg.norm(out["p"] - p) <= 1e-5 * np.linalg.norm(p)
    assert np.abs(out["S"] - S).max() <= 1e-5
    assert S.max() > 0.05                       # water has entered


def test_study_table_shape(ms, ctx):
    from paper_2001_01624_gb300 import coupling as CP
    rows = CP.study(ctx, ratios=(0.5, 2.0), steps=4)
    assert [r["mu_w_over_mu_o"] for r in rows] == [0.5, 2.0]
    for r in rows:
        for nm in CP.SCHEDULES:
            assert r[nm] >= 1.0
        assert r["spread"] >= 0.0
