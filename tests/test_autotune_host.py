"""Host logic of the batched-smoothing autotuner (CPU, library calls faked):
the fastest shape wins, is cached per device and workload, is set on the
context, and is reused without timing again."""
import json

from paper_2001_01624_gb300 import autotune as A


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    calls = []
    cur = {}
    cost = {(256, 4): 5.0, (1024, 4): 1.0, (4096, 2): 3.0}

    def set_tuning(ctx, t, c):
        cur["shape"] = (t, c)
        calls.append(("set", t, c))

    def rebuild(ctx, s, b):
        calls.append(("run",) + cur["shape"])
        clock["t"] += cost[cur["shape"]]

    clock = {"t": 0.0}
    monkeypatch.setattr(A.B, "ms_set_batch_tuning", set_tuning)
    monkeypatch.setattr(A.B, "ms_basis_rebuild_batch", rebuild)
    monkeypatch.setattr(A.time, "perf_counter", lambda: clock["t"])
    monkeypatch.setattr(A, "_device_key", lambda d: "fakegpu|sm4")
    path = str(tmp_path / "tune.json")
    ent = A.tune(None, [], [], shapes=list(cost), path=path, workload="w")
    assert (ent["tile_cells"], ent["ctas_per_sm"]) == (1024, 4)
    assert calls[-1] == ("set", 1024, 4)
    saved = json.load(open(path))
    assert saved["fakegpu|sm4"]["w"]["tile_cells"] == 1024
    assert len(saved["fakegpu|sm4"]["w"]["candidates"]) == 3
    n = len(calls)
    again = A.tuned(None, [], [], path=path, workload="w")     # cached: set, no timing runs
    assert again["tile_cells"] == 1024 and calls[n:] == [("set", 1024, 4)]
    assert A.apply(None, path=path, workload="other") is None
