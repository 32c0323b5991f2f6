"""Write tests/golden/oracle_c2_seed0_gmres.json from a full FP64 oracle run.

Workload: the 3D 60x220x85 geomodel (seed 0), 10x20x5 coarse blocks, box
supports, MsRSB omega = 2/3 to increment 1e-3, and restarted GMRES(30) right-
preconditioned with one multistage cycle (MS + ILU(0)) to relative residual
1e-6 from p = 0.  Only the oracle computes anything here.  Stored: basis
iterations, GMRES steps, residual history, the solution at the same 4096
seeded sample cells as oracle_c2_seed0.json.
Run: python tests/golden/make_oracle_c2_gmres.py
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
    gm = G.config2(0)
    t = {}
    t0 = time.perf_counter()
    s = O.assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = O.pin(s.A, gm.q_active(), 0)
    part, M = O.partition_cartesian(gm.grid, s.cells, gm.block)
    sp, sc = O.support_box(gm.grid, s.cells, s.A, part, M, gm.block)
    B = O.msrsb_basis(s.A, part, M, sp, sc, 2.0 / 3.0, 1e-3, 500)
    L = O.cholesky(O.galerkin(Ap, B))
    lu = O.ilu0(Ap)
    t["setup_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = O.ms_gmres(Ap, [(B, L)], qp, tol=1e-6, max_iter=2000, restart=30, lu=lu)
    t["solve_s"] = time.perf_counter() - t0
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(Ap.n, 4096, replace=False))
    out = dict(workload="c2 seed 0: 60x220x85, blocks 10x20x5, box supports, omega 2/3, basis tol 1e-3, "
                        "GMRES(30) with the MS + ILU(0) cycle as right preconditioner, tol 1e-6, FP64 oracle",
               n=int(Ap.n), M=int(M), basis_iters=int(B.iters), steps=int(r.iters), restart=30,
               converged=bool(r.converged), hist=r.hist.tolist(), final_rel_res=float(r.hist[-1]),
               sample_cells=idx.tolist(), p_sample=r.x[idx].tolist(), p_norm=float(np.linalg.norm(r.x)),
               oracle_seconds=t)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_c2_seed0_gmres.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(json.dumps({k: v for k, v in out.items() if k not in ("sample_cells", "p_sample", "hist")}))


if __name__ == "__main__":
    main()
