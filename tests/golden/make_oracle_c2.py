"""Write tests/golden/oracle_c2_seed0.json from a full FP64 oracle run.

Workload: the 3D 60x220x85 geomodel (seed 0; top 35 layers lognormal with
Kz = 0.1 Kx, bottom 50 layers 1000:1 channels), 10x20x5 coarse blocks, box
supports, MsRSB omega = 2/3 to increment 1e-3, MS + ILU(0) Richardson to
relative residual 1e-6 from p = 0.  Only the oracle computes anything here.
Stored: basis iterations, Richardson cycles, residual history, the solution
at 4096 seeded sample cells, and sizes.  Run: python tests/golden/make_oracle_c2.py
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
    t["setup_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    B = O.msrsb_basis(s.A, part, M, sp, sc, 2.0 / 3.0, 1e-3, 500)
    t["basis_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    L = O.cholesky(O.galerkin(Ap, B))
    lu = O.ilu0(Ap)
    t["coarse_ilu_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-6, max_iter=5000, lu=lu)
    t["solve_s"] = time.perf_counter() - t0
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(Ap.n, 4096, replace=False))
    out = dict(workload="c2 seed 0: 60x220x85, blocks 10x20x5, box supports, omega 2/3, basis tol 1e-3, "
                        "ILU(0) Richardson tol 1e-6, FP64 oracle",
               n=int(Ap.n), M=int(M), nnz_P=int(sp[-1]), basis_iters=int(B.iters), cycles=int(r.iters),
               converged=bool(r.converged), hist_first=r.hist[:40].tolist(), final_rel_res=float(r.hist[-1]),
               sample_cells=idx.tolist(), p_sample=r.x[idx].tolist(), p_norm=float(np.linalg.norm(r.x)),
               oracle_seconds=t)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_c2_seed0.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(json.dumps({k: v for k, v in out.items() if k not in ("sample_cells", "p_sample", "hist_first")}))


if __name__ == "__main__":
    main()
