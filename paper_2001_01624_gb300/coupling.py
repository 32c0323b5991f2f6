"""Coupling-strength study: dynamic bases against the viscosity ratio.

An analogue of the paper's first example (Sec. 6.1), on synthetic inputs: a
42 x 22 single-layer lognormal field (correlation 8 cells, ln K standard
deviation 2) stands in for the SPE10 subset.  Incompressible two-phase flow
with linear relative permeabilities, no gravity or capillarity; water is
injected along the left column and the same rate is produced along the right
column, one pore volume over the run.  The general basis is MsRSB on a 6 x 2
rectilinear partition (7 x 11 cell blocks), built once from the permeability
alone; the coarse operator is re-formed every time step from the current
total mobility.  Each step solves the pressure equation with Richardson
cycles from the previous pressure (Sec. 5.2) to a relative residual of 1e-6
and advances the saturation by explicit upstream transport.

Three solvers per viscosity ratio mu_w / mu_o (the less viscous phase at
1 cP): the general stage alone; general + a dynamic stage rebuilt from the
pressure update after every cycle ("Dp(1)"); general + a dynamic stage
rebuilt after the first two cycles only ("Dp(Inf)").  The dynamic partition
and its constant basis follow Sec. 5.1.  The paper rebuilds per nonlinear
iteration of a fully implicit step; a sequential step here has one linear
solve, so the rebuild schedule is taken over the Richardson cycles of that
solve.  Reported: average cycles per pressure solve.
"""
from __future__ import annotations

from typing import Dict, List, Optional

import numpy as np

from . import binding as ms
from . import geomodel as G

SCHEDULES = {"general": 0, "Dp(1)": 1, "Dp(Inf)": 2}
RATIOS = (1 / 50, 1 / 10, 1 / 2, 1.0, 2.0, 10.0, 50.0)


def model(seed: int = 0, nx: int = 42, ny: int = 22):
    """The 42 x 22 field with injector (left column) and producer (right
    column) rates of unit sum; 6 x 2 general blocks."""
    gm = G.lognormal_box(nx, ny, 1, seed=seed, sigma=2.0, corr=8.0, block=(nx // 6, ny // 2, 1),
                         name="coupling_%dx%d" % (nx, ny))
    q = np.zeros(gm.grid.N)
    left = np.arange(ny) * nx
    right = left + nx - 1
    q[left] = 1.0 / ny
    q[right] = -1.0 / ny
    gm.q = q
    return gm


def viscosities(ratio: float):
    """mu_w, mu_o with mu_w / mu_o = ratio and the smaller one 1 cP."""
    return (ratio, 1.0) if ratio >= 1.0 else (1.0, 1.0 / ratio)


def fluid_for(ratio: float, porosity: float = 0.2, cfl: float = 0.9):
    mu_w, mu_o = viscosities(ratio)
    return ms.fluid(mu_w=mu_w, mu_o=mu_o, n_w=1.0, n_o=1.0, porosity=porosity, cfl=cfl)


class Run:
    """One simulation: a system, the general basis and its coarse stage."""

    def __init__(self, ctx, gm, fluid, steps: int = 40, pv: float = 1.0, tol: float = 1e-6,
                 precision: int = ms.MS_PREC_FP64):
        self.ctx, self.gm, self.fluid, self.steps, self.tol, self.prec = ctx, gm, fluid, steps, tol, precision
        self.sys = ms.ms_system_create(ctx, gm.grid, 0)
        self.perm = np.ascontiguousarray(gm.perm.ravel())
        self.n = ms.ms_system_get_info(self.sys)["n"]
        ms.ms_assemble_tpfa(ctx, self.sys, self.perm)
        part, M = ms.ms_partition_cartesian(ctx, self.sys, gm.block)
        self.basis, _ = ms.ms_build_basis(ctx, self.sys, part, M, block=gm.block, precision=precision)
        self.coarse = ms.ms_galerkin(ctx, self.sys, self.basis, precision)
        self.q = gm.q_active()
        g = gm.grid
        self.volume = g.dx * g.dy * g.dz
        pore_volume = fluid.porosity * self.volume * self.n
        # rates of unit sum scaled so that `pv` pore volumes enter in `steps` steps of length 1
        self.q = self.q * (pv * pore_volume / steps)
        self.dt = 1.0

    def simulate(self, schedule: int, max_iter: int = 5000):
        """Returns dict(cycles per step, substeps per step, p, S)."""
        ctx, s = self.ctx, self.sys
        p = np.zeros(self.n)
        S = np.zeros(self.n)
        cycles, subs = [], []
        for k in range(self.steps):
            lam = ms.ms_total_mobility(ctx, s, self.fluid, S)
            ms.ms_assemble_tpfa(ctx, s, self.perm, mobility=lam, p_prev=p if k else None)
            ms.ms_coarse_refresh(ctx, s, self.coarse)
            info = ms.ms_solve(ctx, s, [self.coarse], self.q, p, tol=self.tol, max_iter=max_iter,
                               precision=self.prec, adapt_schedule=schedule, use_x0=k > 0)
            if not info["converged"]:
                raise ms.MsError(ms.MS_ERR_NOT_CONVERGED, "pressure solve did not converge at step %d" % k)
            cycles.append(info["iters"])
            subs.append(ms.ms_transport_step(ctx, s, self.fluid, p, self.q, self.dt, S))
        return dict(cycles=cycles, substeps=subs, p=p, S=S)

    def release(self):
        ms.ms_coarse_release(self.coarse)
        ms.ms_basis_release(self.basis)
        ms.ms_system_release(self.sys)


def study(ctx, ratios=RATIOS, steps: int = 40, seed: int = 0, schedules: Optional[Dict[str, int]] = None):
    """Average cycles per pressure solve for each ratio and solver, with the
    relative spread (worst - best) / best per ratio."""
    schedules = schedules or SCHEDULES
    gm = model(seed)
    out: List[dict] = []
    for ratio in ratios:
        run = Run(ctx, gm, fluid_for(ratio), steps=steps)
        row = {"mu_w_over_mu_o": ratio}
        for name, sch in schedules.items():
            r = run.simulate(sch)
            row[name] = float(np.mean(r["cycles"]))
        run.release()
        vals = [row[nm] for nm in schedules]
        row["spread"] = (max(vals) - min(vals)) / min(vals)
        out.append(row)
    return out
