"""Cross power (pk_cross) and painted values (pk_paint_values) through the C
ABI against the FP64 oracle.

Tolerances per bin, relative to a scale that cannot cross zero: cross powers
against sqrt(P_aa,raw P_bb,raw) of the bin (the geometric mean of the two
unsubtracted auto powers), painted-value powers against their unsubtracted
power; FP32 form 1e-4, FP64 form 1e-6; mode counts bit-exact."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f64": 1e-6}


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    pk.build()
    pk.load()
    return pk


def _cats(L):
    import synth
    a = synth.lognormal_catalog(60000, L, 48, synth.seed_for(7, 1)).double().numpy()
    extra = synth.lognormal_catalog(30000, L, 48, synth.seed_for(7, 2)).double().numpy()
    b = np.concatenate([a[:36000], extra])                   # correlated with a
    rng = np.random.default_rng(7)
    return a, rng.uniform(0.5, 1.5, len(a)).astype(np.float32), b, rng.uniform(0.5, 1.5, len(b)).astype(np.float32)


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("window,interlaced", [("cic", False), ("tsc", True), ("pcs", True)])
def test_cross_power_matches_oracle(pk, oracle, precision, window, interlaced):
    L, N = 600.0, 48
    dk = 1.5 * 2 * math.pi / L
    a, wa, b, wb = _cats(L)
    pos = np.concatenate([a, b])
    w = np.concatenate([wa, wb])
    cfg = pk.make_config(L, N, window, interlaced=interlaced, dk=dk, nmu=5, precision=precision, batch=2)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint_many(plan, pos, [0, len(a), len(a) + len(b)], weights=w)
        pk.pk_compute(plan)
        ra, rb = pk.pk_result(plan, 0), pk.pk_result(plan, 1)
        got = pk.pk_cross(plan, 0, 1)
        self_a = pk.pk_cross(plan, 0, 0)
    finally:
        pk.pk_destroy(plan)
    ref = oracle.cross_power(a, wa.astype(np.float64), b, wb.astype(np.float64), L, N, window, interlaced,
                             dk=dk, nmu=5)
    assert np.array_equal(got["modes"], ref["modes"])
    ok = ref["modes"] > 0
    scale = np.sqrt((ra["power"] + ra["shot_noise"]) * (rb["power"] + rb["shot_noise"]))
    for ell in range(3):
        d = np.abs(got["poles"][ell] - ref["poles"][ell])[ok]
        assert np.all(d <= TOL[precision] * scale[ok]), (ell, np.max(d / scale[ok]))
    ok2 = ref["modes2d"] > 0
    s2 = np.broadcast_to(scale[:, None], ok2.shape)
    assert np.all(np.abs(got["power2d"] - ref["power2d"])[ok2] <= TOL[precision] * s2[ok2])
    assert got["shot_noise"] == 0.0
    assert abs(got["wsum"] - wa.astype(np.float64).sum()) <= 1e-9 * got["wsum"]
    assert abs(got["w2sum"] - wb.astype(np.float64).sum()) <= 1e-9 * got["w2sum"]
    raw_a = ra["power"] + ra["shot_noise"]
    assert np.all(np.abs(self_a["power"] - raw_a)[ok] <= 1e-6 * raw_a[ok])


@pytest.mark.parametrize("variant", ["sort", "atomic"])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_momentum_field_matches_oracle(pk, oracle, variant, precision):
    L, N = 600.0, 48
    dk = 1.5 * 2 * math.pi / L
    a, wa, _, _ = _cats(L)
    v = np.random.default_rng(9).normal(0.0, 300.0, len(a)).astype(np.float32)
    cfg = pk.make_config(L, N, "tsc", interlaced=True, dk=dk, nmu=4, precision=precision, paint_variant=variant)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint_values(plan, a, v, weights=wa)
        pk.pk_compute(plan)
        got = pk.pk_result(plan)
    finally:
        pk.pk_destroy(plan)
    ref = oracle.fft_power(a, wa.astype(np.float64), L, N, "tsc", True, dk=dk, nmu=4,
                           values=v.astype(np.float64))
    assert np.array_equal(got["modes"], ref["modes"])
    ok = ref["modes"] > 0
    raw = ref["power_raw"][ok]
    for ell in range(3):
        d = np.abs(got["poles"][ell] - ref["poles"][ell])[ok]
        assert np.all(d <= TOL[precision] * raw), (ell, np.max(d / raw))
    assert abs(got["shot_noise"] - ref["shot_noise"]) <= 1e-9 * ref["shot_noise"]
    assert abs(got["wsum"] - ref["wsum"]) <= 1e-9 * ref["wsum"]


def test_density_momentum_cross_matches_oracle(pk, oracle):
    L, N = 600.0, 48
    dk = 1.5 * 2 * math.pi / L
    a, wa, _, _ = _cats(L)
    v = np.random.default_rng(11).normal(0.0, 300.0, len(a)).astype(np.float32)
    pos = np.concatenate([a, a])
    w = np.concatenate([wa, wa])
    vals = np.concatenate([np.ones(len(a), np.float32), v])
    cfg = pk.make_config(L, N, "pcs", interlaced=True, dk=dk, nmu=3, batch=2)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint_values(plan, pos, vals, offsets=[0, len(a), 2 * len(a)], weights=w)
        pk.pk_compute(plan)
        rd, rm = pk.pk_result(plan, 0), pk.pk_result(plan, 1)
        got = pk.pk_cross(plan, 0, 1)
    finally:
        pk.pk_destroy(plan)
    ref = oracle.cross_power(a, wa.astype(np.float64), a, wa.astype(np.float64), L, N, "pcs", True, dk=dk,
                             nmu=3, values_b=v.astype(np.float64))
    ok = ref["modes"] > 0
    scale = np.sqrt((rd["power"] + rd["shot_noise"]) * (rm["power"] + rm["shot_noise"]))
    d = np.abs(got["power"] - ref["power"])[ok]
    assert np.all(d <= TOL["f32"] * scale[ok]), np.max(d / scale[ok])


def test_cross_call_order_errors(pk):
    cfg = pk.make_config(100.0, 16, "cic", dk=0.2, batch=2)
    plan = pk.pk_plan(cfg)
    try:
        with pytest.raises(pk.PkError) as e:
            pk.pk_cross(plan, 0, 1)
        assert e.value.status == pk.PK_ESTATE
        pos = np.random.default_rng(1).uniform(0, 100, (200, 3))
        pk.pk_paint_many(plan, pos, [0, 100, 200])
        with pytest.raises(pk.PkError) as e:
            pk.pk_cross(plan, 0, 1)                          # painted, not computed
        assert e.value.status == pk.PK_ESTATE
        pk.pk_compute(plan)
        with pytest.raises(pk.PkError) as e:
            pk.pk_cross(plan, 0, 2)
        assert e.value.status == pk.PK_EINVAL
        assert pk.pk_cross(plan, 1, 0)["nk"] > 0
    finally:
        pk.pk_destroy(plan)
