"""Write tests/golden/oracle_c3_seed0.json from full FP64 oracle runs.

Workload: the 3D faulted 200x200x50 geomodel (seed 0; ~8 % inactive cells,
3 + 3 vertical faults with a 2-cell throw as non-neighbour connections,
lognormal K with Kz = 0.1 Kx), two coarse stages in the order the solver
takes them (Sec. 5.1: general partitions, then static partitions adapted to
geology):
  1. the general 10x10x5 Cartesian partition with box supports;
  2. the static partition (each general block split by facies class into
     face-connected components) with hop supports;
both smoothed by MsRSB (omega 2/3, increment 1e-3).  Two MS + ILU(0)
Richardson solves to relative residual 1e-6 from p = 0 (Eq. (11), Sec. 5.2):
the two stages alone, and with the dynamic stage of Sec. 5.1 (constant basis
from binned |dp|) rebuilt after cycles 1 and 2 (the paper's Dp(Inf)).

Only the oracle computes anything here.  Stored per solve: cycles, the
residual history of the first 40 cycles, the dynamic-stage block counts of
the first cycles, the solution at 4096 seeded sample cells and its norm;
plus sizes, basis iteration counts and the oracle's wall times.
Run: python tests/golden/make_oracle_c3.py   (several minutes, one thread)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2001_01624_gb300 import geomodel as G  # noqa: E402


def main():
    gm = G.config3(0)
    t = {}
    t0 = time.perf_counter()
    s = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(s.A, gm.q_active(), 0)
    part, M = O.partition_cartesian(gm.grid, s.cells, gm.block)
    sp, sc = O.support_box(gm.grid, s.cells, s.A, part, M, gm.block)
    ps, Ms = O.partition_static(s.A, part, gm.facies[s.cells])
    sp2, sc2 = O.support_hop(gm.grid, s.cells, s.A, ps, Ms)
    t["setup_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    B1 = O.msrsb_basis(s.A, part, M, sp, sc, 2.0 / 3.0, 1e-3, 500)
    B2 = O.msrsb_basis(s.A, ps, Ms, sp2, sc2, 2.0 / 3.0, 1e-3, 500)
    t["basis_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    L1 = O.cholesky(O.galerkin(Ap, B1))
    L2 = O.cholesky(O.galerkin(Ap, B2))
    lu = O.ilu0(Ap)
    t["coarse_ilu_s"] = time.perf_counter() - t0
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(Ap.n, 4096, replace=False))
    solves = {}
    for key, sched in (("static", 0), ("dp_inf", 2)):
        ad = None if sched == 0 else dict(schedule=sched, smoothed=0, grid=gm.grid, cells=s.cells,
                                          A_unpinned=s.A)
        t0 = time.perf_counter()
        r = O.ms_solve(Ap, [(B1, L1), (B2, L2)], qp, tol=1e-6, max_iter=3000, lu=lu, adapt=ad)
        t[f"solve_{key}_s"] = time.perf_counter() - t0
        solves[key] = dict(cycles=int(r.iters), converged=bool(r.converged), hist_first=r.hist[:40].tolist(),
                           final_rel_res=float(r.hist[-1]), p_sample=r.x[idx].tolist(),
                           p_norm=float(np.linalg.norm(r.x)),
                           dyn_blocks_first=[] if r.md_hist is None else [int(v) for v in r.md_hist[:6]])
        print(key, solves[key]["cycles"], solves[key]["final_rel_res"], flush=True)
    out = dict(workload="c3 seed 0: faulted 200x200x50, general 10x10x5 box supports + facies static stage "
                        "(hop supports), omega 2/3, basis tol 1e-3, ILU(0) Richardson tol 1e-6, FP64 oracle; "
                        "solves: two stages alone, and with the constant dynamic stage rebuilt after cycles "
                        "1 and 2",
               n=int(Ap.n), M_general=int(M), M_static=int(Ms), nnz_P_general=int(sp[-1]),
               nnz_P_static=int(sp2[-1]), basis_iters_general=int(B1.iters), basis_iters_static=int(B2.iters),
               sample_cells=idx.tolist(), solves=solves, oracle_seconds=t)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_c3_seed0.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(json.dumps({k: v for k, v in out.items() if k not in ("sample_cells", "solves")}))


if __name__ == "__main__":
    main()
