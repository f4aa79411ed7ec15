"""The serving loop on the GPU: every request's result is the same whether it
is evaluated alone or served in a mix (continuous batching, overlapping
classes, HBM-limited admission), within 1e-5 of the bin's pre-subtraction
monopole (batches only reorder FP32 partial sums); mode counts bit-exact."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SAME = 1e-5


@pytest.fixture(scope="module")
def mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    import synth
    from paper_1712_05834_gb300.batch import Catalog
    pk.build()
    pk.load()
    L = 1000.0
    specs = synth.mock_set_specs(10, synth.seed_for(5, 1), n_lo=2e3, n_hi=3e4, meshes=(32, 48))
    pool = [Catalog(synth.lognormal_catalog(s["n"], L, s["nmesh"], s["seed"], device="cuda"),
                    s["nmesh"], s["window"]) for s in specs]
    big = Catalog(synth.lognormal_catalog(400000, L, 96, synth.seed_for(5, 99), device="cuda"), 96, "tsc", True)
    rng = np.random.default_rng(5)
    cats = [big if k % 9 == 4 else pool[int(rng.integers(len(pool)))] for k in range(36)]
    dk = 4 * 2 * math.pi / L
    alone = {}
    for c in set(map(id, cats)):
        cat = next(x for x in cats if id(x) == c)
        cfg = pk.make_config(L, cat.nmesh, cat.window, interlaced=cat.interlaced, dk=dk)
        plan = pk.pk_plan(cfg)
        try:
            pk.pk_paint(plan, cat.pos)
            pk.pk_compute(plan)
            alone[c] = pk.pk_result(plan)
        finally:
            pk.pk_destroy(plan)
    return L, dk, cats, alone


def same(a, b):
    assert np.array_equal(a["modes"], b["modes"])
    ok = a["modes"] > 0
    raw = a["power"] + a["shot_noise"]
    for ell in range(3):
        d = np.abs(a["poles"][ell] - b["poles"][ell])[ok]
        assert np.all(d <= SAME * raw[ok]), (ell, np.max(d / raw[ok]))
    assert a["wsum"] == b["wsum"]


def _requests(cats, arrivals):
    from paper_1712_05834_gb300.serve import Request
    return [Request(i, c, float(t)) for i, (c, t) in enumerate(zip(cats, arrivals))]


@pytest.mark.parametrize("realtime", [True, False])
def test_served_results_equal_alone(mix, realtime):
    from paper_1712_05834_gb300 import serve
    L, dk, cats, alone = mix
    arr = serve.poisson_arrivals(len(cats), 3000.0, 7)
    with serve.PowerServer(L, dk=dk, max_batch=4, max_objects=200000, large_nmesh=96) as srv:
        done = srv.run(_requests(cats, arr), realtime=realtime)
        made = srv.slots_made
    assert all(r.result is not None for r in done)
    for r in done:
        same(alone[id(r.catalog)], r.result)
        assert r.latency >= 0
    if not realtime:
        assert max(r.batch_size for r in done) > 1          # batches actually formed
    assert made >= 2
    s = serve.latency_summary(done)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_hbm_budget_forces_eviction_and_still_serves_everything(mix):
    from paper_1712_05834_gb300 import serve
    L, dk, cats, alone = mix
    big = serve.slot_bytes(96, True, "f32", 1, 400000)
    small = serve.slot_bytes(48, False, "f32", 4, 200000)
    budget = max(big, small) + small // 2            # too small to hold every class at once
    with serve.PowerServer(L, dk=dk, max_batch=4, max_objects=200000, large_nmesh=96,
                           budget_bytes=budget) as srv:
        done = srv.run(_requests(cats, np.zeros(len(cats))), realtime=False)
        assert srv.evictions > 0
        assert srv.peak_bytes <= budget
    for r in done:
        same(alone[id(r.catalog)], r.result)


def test_plain_path_matches_alone(mix):
    from paper_1712_05834_gb300 import serve
    L, dk, cats, alone = mix
    done = serve.plain_serve(_requests(cats[:8], np.zeros(8)), L, realtime=False, dk=dk)
    for r in done:
        same(alone[id(r.catalog)], r.result)
