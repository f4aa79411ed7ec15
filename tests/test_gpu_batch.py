"""Batched mocks on the GPU: capture-safe plans, CUDA-graph replay, size-class
batches with the autotuner, against one-at-a-time evaluation and the oracle.

Tolerances: mode counts bit-exact; a replay or a batch against the same
catalog evaluated alone, 1e-5 of the bin's pre-subtraction monopole (the two
differ only in the order of FP32 partial sums inside the bin kernel); against
the FP64 oracle, the FP32-form 1e-4.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SAME = 1e-5
TOL32 = 1e-4


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    pk.build()
    pk.load()
    return pk


def same(a, b, tol=SAME):
    assert np.array_equal(a["modes"], b["modes"])
    ok = a["modes"] > 0
    raw = a["power"] + a["shot_noise"]
    for ell in range(3):
        d = np.abs(a["poles"][ell] - b["poles"][ell])[ok]
        assert np.all(d <= tol * raw[ok]), (ell, np.max(d / raw[ok]))
    if a["nmu"]:
        assert np.array_equal(a["modes2d"], b["modes2d"])
        ok2 = a["modes2d"] > 0
        raw2 = np.broadcast_to(raw[:, None], ok2.shape)
        d = np.abs(a["power2d"] - b["power2d"])[ok2]
        assert np.all(d <= tol * raw2[ok2])
    assert a["wsum"] == b["wsum"] and a["shot_noise"] == b["shot_noise"]


def _mocks(torch, specs, L):
    import synth
    from paper_1712_05834_gb300.batch import Catalog
    return [Catalog(synth.lognormal_catalog(s["n"], L, s["nmesh"], s["seed"], device="cuda"),
                    s["nmesh"], s["window"]) for s in specs]


def _alone(pk, cat, L, dk, nmu=0):
    cfg = pk.make_config(L, cat.nmesh, cat.window, interlaced=cat.interlaced, dk=dk, nmu=nmu)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint(plan, cat.pos)
        pk.pk_compute(plan)
        return pk.pk_result(plan)
    finally:
        pk.pk_destroy(plan)


@pytest.mark.parametrize("variant", ["sort", "atomic"])
def test_graph_replay_matches_eager_and_sees_refilled_positions(pk, variant):
    import torch
    import synth
    L, N, dk = 500.0, 48, 2 * math.pi / 500.0
    sizes = [20000, 3000, 45000]
    a = [synth.lognormal_catalog(n, L, N, synth.seed_for(4, 100 + k), device="cuda") for k, n in enumerate(sizes)]
    b = [synth.lognormal_catalog(n, L, N, synth.seed_for(4, 200 + k), device="cuda") for k, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    buf = torch.cat(a).contiguous()
    s = torch.cuda.Stream()
    cfg = pk.make_config(L, N, "tsc", interlaced=True, dk=dk, nmu=4, batch=3, capacity=int(off[-1]),
                         paint_variant=variant)
    plan = pk.pk_plan(cfg, s)
    try:
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            pk.pk_paint_many(plan, buf, off)
            pk.pk_compute(plan)
        for cats in (a, b):
            buf.copy_(torch.cat(cats))
            torch.cuda.synchronize()
            with torch.cuda.stream(s):
                g.replay()
            s.synchronize()
            got = [pk.pk_result(plan, k) for k in range(3)]
            for k in range(3):
                cfg1 = pk.make_config(L, N, "tsc", interlaced=True, dk=dk, nmu=4, paint_variant=variant)
                p1 = pk.pk_plan(cfg1)
                try:
                    pk.pk_paint(p1, cats[k])
                    pk.pk_compute(p1)
                    same(pk.pk_result(p1), got[k])
                finally:
                    pk.pk_destroy(p1)
    finally:
        pk.pk_destroy(plan)


def test_capture_refuses_growth_and_host_inputs(pk):
    import torch
    L, N = 200.0, 16
    pos = torch.rand((1000, 3), device="cuda") * L
    s = torch.cuda.Stream()
    plan = pk.pk_plan(pk.make_config(L, N, "cic", dk=0.1, capacity=100), s)
    try:
        torch.cuda.synchronize()
        for arg in (pos, pos[:50].cpu().numpy().astype(np.float32)):
            g = torch.cuda.CUDAGraph()
            with pytest.raises(pk.PkError) as e:
                with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                    pk.pk_paint(plan, arg)
            assert e.value.status == pk.PK_EINVAL
            assert "capture" in str(e.value)
        pk.pk_paint(plan, pos)            # outside capture the plan grows
        pk.pk_compute(plan)
        assert pk.pk_result(plan)["wsum"] == 1000.0
    finally:
        pk.pk_destroy(plan)


@pytest.mark.parametrize("graph,streams", [(True, 1), (False, 1), (True, 3), (False, 2)])
def test_size_class_batches_match_one_at_a_time(pk, graph, streams):
    import torch
    import synth
    from paper_1712_05834_gb300 import batch
    L = 1000.0
    dk = 0.01 * 4
    specs = synth.mock_set_specs(14, synth.seed_for(4, 500), n_lo=2e3, n_hi=6e4, meshes=(32, 48, 64))
    cats = _mocks(torch, specs, L)
    tuner = batch.Autotuner(sample=4, repeats=1)
    with batch.BatchPower(cats, L, dk=dk, tuner=tuner, graph=graph, streams=streams) as bp:
        assert len(bp.classes) == len(batch.group_classes(cats))
        assert len({c.stream_index for c in bp.classes}) == min(streams, len(bp.classes))
        res = bp.run()
        res2 = bp.run()
        assert bp.launches_per_run >= 5 * len(bp.classes)
    for tk, (variant, tile) in tuner.cache.items():       # the fastest timed candidate
        times = tuner.timings[tk]
        assert "atomic/0" in times and len(times) >= 2
        assert min(times, key=times.get) == "%s/%d" % (variant, tile)
    for i, cat in enumerate(cats):
        alone = _alone(pk, cat, L, dk)
        same(alone, res[i])
        same(alone, res2[i])


def test_size_class_batch_against_the_oracle(pk, oracle):
    import torch
    import synth
    from paper_1712_05834_gb300 import batch
    L = 1000.0
    dk = 0.01 * 4
    specs = synth.mock_set_specs(6, synth.seed_for(4, 600), n_lo=2e3, n_hi=2e4, meshes=(32, 48))
    cats = _mocks(torch, specs, L)
    with batch.BatchPower(cats, L, dk=dk, tuner=batch.Autotuner(sample=2, repeats=1)) as bp:
        res = bp.run()
    for cat, got in zip(cats, res):
        ref = oracle.fft_power(cat.pos.double().cpu().numpy(), None, L, cat.nmesh, cat.window, False,
                               True, dk=dk)
        assert np.array_equal(got["modes"], ref["modes"])
        ok = ref["modes"] > 0
        for ell in range(3):
            d = np.abs(got["poles"][ell] - ref["poles"][ell])[ok]
            assert np.all(d <= TOL32 * ref["power_raw"][ok]), ell
