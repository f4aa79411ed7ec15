"""Projected power spectra (pk_projected) through the C ABI against the FP64
oracle, which projects the painted mesh itself (sums over the dropped axes)
and transforms the projection: the CUDA path reads the plane of the 3D
transform instead, so this also checks the projection-slice route.
Mode counts bit-exact, mean k 1e-12, power within 1e-4 (FP32 form) / 1e-6
(FP64 form) of the bin's unsubtracted power plus the shot-noise level: a
projected line has one or two modes per bin, whose power can fall far below
its mean by chance, so the noise floor joins the scale."""
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


@pytest.mark.parametrize("axes", [(0, 1), (0, 2), (1, 2), (2,), (0,)])
@pytest.mark.parametrize("window,interlaced,precision", [("tsc", True, "f32"), ("cic", False, "f64"),
                                                         ("pcs", True, "f64")])
def test_projected_power_matches_oracle(pk, oracle, axes, window, interlaced, precision):
    import synth
    L, N = 400.0, 40
    pos = synth.lognormal_catalog(80000, L, N, synth.seed_for(8, len(axes))).double().numpy()
    w = np.random.default_rng(3).uniform(0.5, 1.5, len(pos)).astype(np.float32)
    dk = (2.0 if len(axes) == 2 else 1.0) * 2 * math.pi / L
    cfg = pk.make_config(L, N, window, interlaced=interlaced, dk=dk, precision=precision)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint(plan, pos, w)
        pk.pk_compute(plan)
        got = pk.pk_projected(plan, 0, axes)
    finally:
        pk.pk_destroy(plan)
    ref = oracle.projected_power(pos, w.astype(np.float64), L, N, window, interlaced, dk=dk, axes=axes)
    assert got["ndim"] == len(axes)
    assert np.array_equal(got["modes"], ref["modes"])
    ok = ref["modes"] > 0
    np.testing.assert_allclose(got["k"][ok], ref["k"][ok], rtol=1e-12)
    d = np.abs(got["power"] - ref["power"])[ok]
    scale = ref["power_raw"][ok] + ref["shot_noise"]
    assert np.all(d <= TOL[precision] * scale), np.max(d / scale)
    assert abs(got["shot_noise"] - ref["shot_noise"]) <= 1e-12 * ref["shot_noise"]


def test_projected_argument_errors(pk):
    plan = pk.pk_plan(pk.make_config(100.0, 16, "cic", dk=0.2))
    try:
        with pytest.raises(pk.PkError) as e:
            pk.pk_projected(plan, 0, (0, 1))
        assert e.value.status == pk.PK_ESTATE
        pk.pk_paint(plan, np.random.default_rng(1).uniform(0, 100, (100, 3)))
        pk.pk_compute(plan)
        for bad in [(0, 1, 2), ()]:
            with pytest.raises(pk.PkError) as e:
                pk.pk_projected(plan, 0, bad)
            assert e.value.status == pk.PK_EINVAL
        assert pk.pk_projected(plan, 0, ("x", "y"))["nk"] > 0
    finally:
        pk.pk_destroy(plan)
