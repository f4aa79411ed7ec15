"""pipeline.PowerStream on the GPU: catalogs from pinned host memory, pageable
host memory and the device, streamed through 1, 2 and 3 plans, give the
results of one plan taking them one at a time.

Mode counts bit-exact; P(k), P(k, mu) and the multipoles within 1e-6 of the
bin's unsubtracted monopole (the meshes are bit-identical; only the order
of the per-CTA FP32 bin additions differs between runs)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    pk.build()
    pk.load()
    return pk


def _close(got, ref):
    assert np.array_equal(got["modes"], ref["modes"])
    assert np.array_equal(got["modes2d"], ref["modes2d"])
    ok = ref["modes"] > 0
    raw0 = (ref["power"] + ref["shot_noise"])[ok]
    assert np.all(np.abs(got["power"] - ref["power"])[ok] <= TOL * raw0)
    assert np.all(np.abs(got["poles"] - ref["poles"])[:, ok] <= TOL * raw0[None, :])
    ok2 = ref["modes2d"] > 0
    lim = TOL * np.broadcast_to((ref["power"] + ref["shot_noise"])[:, None], ok2.shape)
    assert np.all(np.abs(got["power2d"] - ref["power2d"])[ok2] <= lim[ok2])


@pytest.mark.parametrize("own", [True, False])
def test_stream_matches_one_plan(pk, own):
    import torch

    import synth
    from paper_1712_05834_gb300.pipeline import PowerStream, power_stream
    L, N = 500.0, 128
    cats = [synth.lognormal_catalog(150_000 + 20_000 * k, L, 64, synth.seed_for(15, k)) for k in range(5)]
    inputs = [cats[0].pin_memory(), cats[1].numpy(), cats[2].cuda(), cats[3].pin_memory(), cats[4].numpy()]
    cfg = pk.make_config(L, N, "tsc", interlaced=True, dk=0.05, nmu=5)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_use_own_fft(plan, own)
        ref = []
        for c in cats:
            pk.pk_paint(plan, c.numpy())
            pk.pk_compute(plan)
            ref.append(pk.pk_result(plan, 0))
    finally:
        pk.pk_destroy(plan)
    for depth in (1, 2, 3):
        got = list(power_stream(cfg, inputs, depth=depth, own_fft=own))
        assert len(got) == len(ref)
        for g, r in zip(got, ref):
            _close(g, r)
    # plans kept across two maps; weights alongside
    w = [np.random.default_rng(k).uniform(0.5, 1.5, len(c)).astype(np.float32) for k, c in enumerate(cats[:2])]
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_use_own_fft(plan, own)
        refw = []
        for c, wk in zip(cats[:2], w):
            pk.pk_paint(plan, c.numpy(), wk)
            pk.pk_compute(plan)
            refw.append(pk.pk_result(plan, 0))
    finally:
        pk.pk_destroy(plan)
    with PowerStream(cfg, depth=2, own_fft=own) as ps:
        for g, r in zip(ps.map(inputs[:3]), ref[:3]):
            _close(g, r)
        for g, r in zip(ps.map([cats[0].pin_memory(), cats[1].pin_memory()], weights=w), refw):
            _close(g, r)
    torch.cuda.synchronize()
