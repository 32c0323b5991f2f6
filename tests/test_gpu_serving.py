"""Serving loop: sequential-implicit two-phase steps on resident geomodels
with continuous batching; every result is the same alone and in the mix."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _models(G, serve):
    shapes = [(14, 12, 6), (20, 9, 5), (11, 16, 7), (18, 18, 4)]
    gms = [G.lognormal_box(*sh, seed=50 + k, sigma=1.5, block=(5, 4, 3), kz_ratio=0.1) for k, sh in enumerate(shapes)]
    for gm in gms:
        gm.q[:] *= 1e-4
    return [serve.Model(k, gm, torch, torch.device("cuda:0")) for k, gm in enumerate(gms)]


def _dt(m):
    vol = m.gm.grid.dx * m.gm.grid.dy * m.gm.grid.dz
    return 0.02 * 0.2 * vol * m.n / 1e-4          # 2 % of the pore volume injected per step


def _stream(models, steps, rate):
    from paper_2001_01624_gb300 import serve
    reqs = []
    rid = 0
    t = 0.0
    rng = np.random.default_rng(3)
    order = [m.mid for m in models for _ in range(steps)]
    rng.shuffle(order)
    for mid in order:
        t += rng.exponential(1.0 / rate)
        reqs.append(serve.Request(rid, mid, t, _dt(models[mid])))
        rid += 1
    return reqs


def _run(workers, budget=None, steps=4):
    from paper_2001_01624_gb300 import geomodel as G, serve
    models = _models(G, serve)
    srv = serve.Server(torch, torch.device("cuda:0"), models, workers=workers, hbm_budget=budget)
    reqs = srv.run(_stream(models, steps, rate=400.0))
    out = [m.state() for m in models]
    srv.close()
    return reqs, out, models


def test_results_same_alone_and_in_the_mix():
    reqs1, alone, models = _run(workers=1)
    reqsN, mix, _ = _run(workers=4)
    for (pa, sa), (pm, sm) in zip(alone, mix):
        np.testing.assert_array_equal(pa, pm)
        np.testing.assert_array_equal(sa, sm)
    for r in reqsN:
        assert r.rel_residual <= 1e-6 and r.cycles >= 1 and r.substeps >= 1
        assert r.done >= r.start >= r.arrival - 1e-3
    # water entered the models and saturations stay physical
    for (p, S), m in zip(mix, models):
        assert S.max() > 0.0 and S.min() >= -1e-12 and S.max() <= 1 + 1e-12


def test_admission_by_memory_evicts_and_restores_state():
    _, alone, models = _run(workers=1)
    # room for about two of the four models: loads evict idle ones (state kept on the host)
    budget = int(2.5 * max(m.n for m in models) * 2500)
    _, tight, _ = _run(workers=3, budget=budget)
    for (pa, sa), (pt, st) in zip(alone, tight):
        np.testing.assert_array_equal(pa, pt)
        np.testing.assert_array_equal(sa, st)
