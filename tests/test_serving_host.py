"""Host pieces of the request server and of the coupling study (CPU): the
Poisson request stream, the latency summary, and the coupling study's
fluids and well rates."""
import numpy as np

from paper_2001_01624_gb300 import coupling as CP
from paper_2001_01624_gb300 import serve as S


def test_poisson_stream():
    reqs = S.poisson_stream(20000, rate=200.0, n_models=32, dt_of=lambda m: 1.0 + m, seed=7)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0) and [r.rid for r in reqs] == list(range(20000))
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.03                 # mean gap 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05             # exponential: coefficient of variation 1
    mids = np.array([r.model for r in reqs])
    assert mids.min() == 0 and mids.max() == 31 and np.bincount(mids).min() > 500
    assert all(r.dt == 1.0 + r.model for r in reqs)
    again = S.poisson_stream(20000, rate=200.0, n_models=32, dt_of=lambda m: 1.0, seed=7)
    assert [r.arrival for r in again] == list(t)


def test_latency_stats():
    reqs = [S.Request(k, 0, arrival=0.01 * k, dt=1.0) for k in range(100)]
    for k, r in enumerate(reqs):
        r.done = r.arrival + 0.001 * (k + 1)                    # latencies 1 .. 100 ms
    st = S.latency_stats(reqs)
    assert abs(st["p50_ms"] - np.percentile(np.arange(1, 101), 50)) < 1e-9
    assert abs(st["p99_ms"] - np.percentile(np.arange(1, 101), 99)) < 1e-9
    assert abs(st["mean_ms"] - 50.5) < 1e-9 and st["requests"] == 100
    assert abs(st["throughput_req_s"] - 100 / (0.99 + 0.1)) < 1e-9


def test_coupling_fluids_and_rates():
    for ratio in CP.RATIOS:
        mw, mo = CP.viscosities(ratio)
        assert abs(mw / mo - ratio) < 1e-12 and min(mw, mo) == 1.0
    gm = CP.model(seed=0)
    q = gm.q.reshape(22, 42)
    assert abs(q.sum()) < 1e-15 and np.allclose(q[:, 0], 1 / 22) and np.allclose(q[:, -1], -1 / 22)
    assert np.all(q[:, 1:-1] == 0) and gm.block == (7, 11, 1)
