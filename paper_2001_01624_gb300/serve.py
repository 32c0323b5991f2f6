"""Serving loop: sequential-implicit two-phase time steps on resident geomodels.

Each request advances one geomodel by one time step (Sec. 2 two-phase model,
Sec. 5 multiscale solver):

    lambda_t(S)  ->  TPFA assembly with upstream face mobility (previous p)
    ->  Galerkin operator of the resident basis re-formed  (basis kept)
    ->  dynamic stage from the previous pressure change dp (adaptive refresh)
    ->  GMRES preconditioned by the multiscale cycle, from the previous
        pressure to 1e-6
    ->  explicit upstream saturation transport with CFL substeps.

Continuous batching: a pool of worker slots (one library context and CUDA
stream each) takes requests as they arrive and as slots free up, so the
kernels of different requests overlap on the device; steps of one model stay
in arrival order.  A model's device state (system, basis, coarse operator,
pressure, saturation) is resident once admitted; admission of a model that is
not resident waits for free device memory (the measured footprint of its
last load, or an estimate from its size) and evicts idle models least
recently used first, keeping their pressure and saturation on the host.
A model's footprint is what the library itself allocated for it (its
allocation count on the loading thread, for the handles and the workspaces
of its first step) plus the model's own tensors, so concurrent steps of other
models do not disturb the measurement.
"""
from __future__ import annotations

import dataclasses
import heapq
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import binding as ms

BYTES_PER_CELL_ESTIMATE = 2500   # device bytes per cell of a resident model (mixed solve), before measuring


@dataclasses.dataclass
class Request:
    rid: int
    model: int
    arrival: float          # seconds from the start of the stream
    dt: float
    start: float = 0.0
    done: float = 0.0
    cycles: int = 0
    substeps: int = 0
    rel_residual: float = 0.0


class Model:
    """One geomodel: host inputs, and its device state while resident."""

    def __init__(self, mid: int, gm, torch, device):
        self.mid, self.gm, self.torch, self.device = mid, gm, torch, device
        self.n = gm.grid.n_active()
        self.q = gm.q_active()
        self.footprint = self.n * BYTES_PER_CELL_ESTIMATE
        self.lock = threading.Lock()      # steps of one model run one at a time, in order
        self.next_rid = 0                 # request ids of this model are served in this order
        self.cond = threading.Condition(self.lock)
        self.resident = False
        self.last_used = 0.0
        # state kept across evictions (host) and while resident (device)
        self.h_p = np.zeros(self.n)
        self.h_S = np.zeros(self.n)
        self.h_dp: Optional[np.ndarray] = None
        self.steps = 0

    # ------------------------------------------------------------ residency
    def load(self, ctx, stream, precision):
        with self.torch.cuda.stream(stream):
            self._load(ctx, precision)

    def _load(self, ctx, precision):
        t = self.torch
        lib0 = ms.ms_allocation_stats()["thread_bytes"]
        self.sys = ms.ms_system_create(ctx, self.gm.grid, 0)
        self.perm = t.from_numpy(self.gm.perm.ravel().copy()).to(self.device)
        self.qd = t.from_numpy(self.q).to(self.device)
        self.p = t.from_numpy(self.h_p).to(self.device)
        self.S = t.from_numpy(self.h_S).to(self.device)
        self.lam = t.empty_like(self.p)
        self.p_prev = t.empty_like(self.p)
        self.dp = None if self.h_dp is None else t.from_numpy(self.h_dp).to(self.device)
        ms.ms_assemble_tpfa(ctx, self.sys, self.perm)
        part, M = ms.ms_partition_cartesian(ctx, self.sys, self.gm.block)
        self.basis, _ = ms.ms_build_basis(ctx, self.sys, part, M, block=self.gm.block, precision=precision)
        self.coarse = ms.ms_galerkin(ctx, self.sys, self.basis, precision)
        t.cuda.synchronize(self.device)
        tensors = sum(x.numel() * x.element_size() for x in (self.perm, self.qd, self.p, self.S, self.lam,
                                                              self.p_prev))
        # library bytes of the handles, the tensors, and (once measured) the
        # workspaces a step adds; before the first step: the size estimate
        lib = ms.ms_allocation_stats()["thread_bytes"] - lib0
        self.load_bytes = lib + 2 * tensors
        self.footprint = self.load_bytes + getattr(self, "step_bytes", self.n * BYTES_PER_CELL_ESTIMATE // 2)
        self.resident = True

    def evict(self):
        self.torch.cuda.synchronize(self.device)
        self.h_p = self.p.cpu().numpy().copy()
        self.h_S = self.S.cpu().numpy().copy()
        self.h_dp = None if self.dp is None else self.dp.cpu().numpy().copy()
        ms.ms_coarse_release(self.coarse)
        ms.ms_basis_release(self.basis)
        ms.ms_system_release(self.sys)
        del self.perm, self.qd, self.p, self.S, self.lam, self.dp, self.p_prev
        self.resident = False
        self.torch.cuda.empty_cache()      # let the freed tensors show as free device memory

    # ------------------------------------------------------------------ step
    def step(self, ctx, stream, fluid, dt, precision, tol, adapt, max_iter=5000):
        """One sequential-implicit step on `stream` (the stream of ctx);
        returns (cycles, substeps, rel_residual)."""
        with self.torch.cuda.stream(stream):
            return self._step(ctx, fluid, dt, precision, tol, adapt, max_iter)

    def _step(self, ctx, fluid, dt, precision, tol, adapt, max_iter):
        lib0 = ms.ms_allocation_stats()["thread_bytes"]
        ms.ms_total_mobility(ctx, self.sys, fluid, self.S, self.lam)
        ms.ms_assemble_tpfa(ctx, self.sys, self.perm, mobility=self.lam, p_prev=self.p if self.steps else None)
        ms.ms_coarse_refresh(ctx, self.sys, self.coarse)
        stages = [self.coarse]
        dyn_b = dyn_c = None
        if adapt and self.dp is not None:
            dyn_b = ms.ms_add_adaptive_basis(ctx, self.sys, self.dp, precision=precision)
            dyn_c = ms.ms_galerkin(ctx, self.sys, dyn_b, precision)
            stages.append(dyn_c)
        self.p_prev.copy_(self.p)
        info = ms.ms_solve(ctx, self.sys, stages, self.qd, self.p, tol=tol, max_iter=max_iter, precision=precision,
                           use_x0=self.steps > 0, outer=ms.MS_OUTER_GMRES, restart=30)
        if dyn_c is not None:
            ms.ms_coarse_release(dyn_c)
            ms.ms_basis_release(dyn_b)
        if self.dp is None:
            self.dp = self.torch.empty_like(self.p)
        ms.ms_pressure_update(ctx, self.sys, self.p, self.p_prev, self.dp)
        k = ms.ms_transport_step(ctx, self.sys, fluid, self.p, self.qd, dt, self.S)
        if self.steps == 0:
            # workspaces the first step adds (solver vectors, the dynamic stage)
            self.step_bytes = ms.ms_allocation_stats()["thread_bytes"] - lib0 + self.dp.numel() * 8
            self.footprint = self.load_bytes + self.step_bytes
        self.steps += 1
        return info["iters"], k, info["rel_residual"]

    def state(self):
        if self.resident:
            self.torch.cuda.synchronize(self.device)
            return self.p.cpu().numpy().copy(), self.S.cpu().numpy().copy()
        return self.h_p.copy(), self.h_S.copy()


class Server:
    """Worker slots over one GPU; requests for resident geomodels."""

    def __init__(self, torch, device, models: List[Model], workers=8, fluid=None, precision=ms.MS_PREC_MIXED,
                 tol=1e-6, adapt=True, hbm_budget: Optional[int] = None, reserve=2 << 30):
        self.torch, self.device, self.models = torch, device, models
        self.fluid = fluid or ms.fluid()
        self.precision, self.tol, self.adapt = precision, tol, adapt
        self.reserve = reserve
        self.budget = hbm_budget           # bytes of device memory the resident models may use (None: free HBM)
        self.used = 0
        self.mem_lock = threading.Condition()
        self.streams = [torch.cuda.Stream(device) for _ in range(workers)]
        self.ctxs = [ms.ms_create(device if isinstance(device, int) else device.index or 0, st)
                     for st in self.streams]

    def close(self):
        for m in self.models:
            if m.resident:
                m.evict()
        for c in self.ctxs:
            ms.ms_destroy(c)

    def _stream(self, ctx):
        return self.streams[[c.value for c in self.ctxs].index(ctx.value)]

    # ------------------------------------------------------------- admission
    def _free(self):
        if self.budget is not None:
            return self.budget - self.used
        return self.torch.cuda.mem_get_info(self.device)[0] - self.reserve

    def admit(self, m: Model, ctx):
        """Make m resident, evicting idle models (least recently used first)
        while the free device memory is short of its footprint."""
        with self.mem_lock:
            while not m.resident:
                if self._free() >= m.footprint or self.used == 0:
                    m.load(ctx, self._stream(ctx), self.precision)
                    self.used += m.footprint
                    break
                idle = [x for x in self.models if x.resident and x is not m and not x.lock.locked()]
                if idle:
                    v = min(idle, key=lambda x: x.last_used)
                    self.used -= v.footprint
                    v.evict()
                else:
                    self.mem_lock.wait(0.01)

    def warm(self, dt):
        """Admit every model and run one step on it (setup outside the stream)."""
        for m in self.models:
            self.admit(m, self.ctxs[0])
            with m.lock:
                m.step(self.ctxs[0], self.streams[0], self.fluid, dt, self.precision, self.tol, self.adapt)
                m.last_used = time.perf_counter()
        self.torch.cuda.synchronize(self.device)

    # ------------------------------------------------------------------ loop
    def run(self, requests: List[Request]) -> List[Request]:
        """Serve requests (arrival times relative to the call); returns them
        with start / done times and per-step results."""
        pending = [(r.arrival, r.rid, r) for r in requests]
        heapq.heapify(pending)
        per_model: Dict[int, List[int]] = {}
        for r in sorted(requests, key=lambda r: (r.arrival, r.rid)):
            per_model.setdefault(r.model, []).append(r.rid)
        order = {mid: iter(rids) for mid, rids in per_model.items()}
        for m in self.models:
            nxt = next(order.get(m.mid, iter(())), None)
            m.next_rid = -1 if nxt is None else nxt
        qlock = threading.Lock()
        t0 = time.perf_counter()

        def worker(ctx):
            while True:
                with qlock:
                    if not pending:
                        return
                    arrival, rid, r = heapq.heappop(pending)
                wait = t0 + arrival - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                m = self.models[r.model]
                with m.cond:
                    while m.next_rid != r.rid:      # earlier steps of this model first
                        m.cond.wait()
                    self.admit(m, ctx)
                    r.start = time.perf_counter() - t0
                    st = self._stream(ctx)
                    r.cycles, r.substeps, r.rel_residual = m.step(ctx, st, self.fluid, r.dt, self.precision,
                                                                  self.tol, self.adapt)
                    st.synchronize()
                    r.done = time.perf_counter() - t0
                    m.last_used = time.perf_counter()
                    m.next_rid = next(order[m.mid], -1)
                    m.cond.notify_all()
                with self.mem_lock:
                    self.mem_lock.notify_all()

        threads = [threading.Thread(target=worker, args=(c,)) for c in self.ctxs]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        return requests


def poisson_stream(n_requests: int, rate: float, n_models: int, dt_of, seed: int = 7) -> List[Request]:
    """Poisson arrivals (exponential gaps of mean 1/rate), each for a model
    drawn uniformly; dt_of(model) gives that model's time step."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    mids = rng.integers(0, n_models, n_requests)
    return [Request(k, int(mids[k]), float(t[k]), dt_of(int(mids[k]))) for k in range(n_requests)]


def latency_stats(reqs: List[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs])
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "throughput_req_s": len(reqs) / span if span > 0 else 0.0,
            "requests": len(reqs)}
