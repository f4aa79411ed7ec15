"""The library's own r2c transform (y and x passes, then the z transform fused
into the bin pass) through the C ABI, against the FP64 oracle and against the
cuFFT path on the same painted meshes (N = 128, 192, 256, 512, 1024).

Tolerances per bin against the unsubtracted monopole of the bin (as in the
parity tests): 1e-4 against the oracle (FP32 form); the two GPU transforms of
the same FP32 meshes agree within 1e-5 of it (both are FP32 FFTs with errors
near 1e-7 of the bin's power).  Mode counts bit-exact.  Cross and projected
power after a compute on the own transform read the r2c transform that the
finishing pass writes into the meshes."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_ORACLE = 1e-4
TOL_PATHS = 1e-5


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    pk.build()
    pk.load()
    return pk


def _run(pk, cfg, pos, own, w=None):
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_use_own_fft(plan, own)
        pk.pk_paint(plan, pos, w)
        pk.pk_compute(plan)
        return pk.pk_result(plan, 0)
    finally:
        pk.pk_destroy(plan)


def _check_bins(got, ref, raw0, tol):
    assert np.array_equal(got["modes"], ref["modes"])
    ok = ref["modes"] > 0
    d = np.abs(got["power"] - ref["power"])[ok]
    assert np.all(d <= tol * raw0[ok]), np.max(d / raw0[ok])
    dp = np.abs(got["poles"] - ref["poles"])[:, ok]
    assert np.all(dp <= tol * raw0[ok][None, :]), np.max(dp / raw0[ok][None, :])
    if "power2d" in ref:
        assert np.array_equal(got["modes2d"], ref["modes2d"])
        ok2 = ref["modes2d"] > 0
        d2 = np.abs(got["power2d"] - ref["power2d"])
        lim = tol * np.broadcast_to(raw0[:, None], d2.shape)
        assert np.all(d2[ok2] <= lim[ok2]), np.max(d2[ok2] / lim[ok2] * tol)


@pytest.mark.parametrize("window,interlaced,nmu", [("cic", False, 0), ("tsc", True, 5), ("pcs", True, 10)])
def test_own_transform_matches_oracle_at_256(pk, oracle, window, interlaced, nmu):
    import synth
    L, N = 500.0, 256
    pos = synth.lognormal_catalog(200000, L, 128, synth.seed_for(11, nmu)).double().numpy()
    dk = 2.5 * 2 * math.pi / L
    cfg = pk.make_config(L, N, window, interlaced=interlaced, dk=dk, nmu=nmu)
    got = _run(pk, cfg, pos, True)
    ref = oracle.fft_power(pos, None, L, N, window, interlaced, dk=dk, nmu=nmu)
    _check_bins(got, ref, ref["power_raw"], TOL_ORACLE)


@pytest.mark.parametrize("N,window,interlaced,nmu,weighted", [(512, "tsc", True, 10, False),
                                                              (512, "cic", False, 0, True),
                                                              (256, "pcs", True, 4, True),
                                                              (128, "cic", False, 0, False),
                                                              (128, "tsc", True, 5, True),
                                                              (192, "cic", False, 0, False),
                                                              (192, "tsc", True, 4, True),
                                                              (1024, "pcs", True, 10, False),
                                                              (1024, "tsc", False, 0, True)])
def test_own_and_cufft_transforms_agree(pk, N, window, interlaced, nmu, weighted):
    import synth
    L = 1000.0
    pos = synth.lognormal_catalog(2_000_000, L, 256, synth.seed_for(12, N + nmu)).numpy()
    w = np.random.default_rng(N).uniform(0.5, 1.5, len(pos)).astype(np.float32) if weighted else None
    cfg = pk.make_config(L, N, window, interlaced=interlaced, dk=0.005, nmu=nmu)
    own = _run(pk, cfg, pos, True, w)
    lib = _run(pk, cfg, pos, False, w)
    _check_bins(own, lib, lib["power"] + lib["shot_noise"], TOL_PATHS)


def test_cross_and_projected_after_own_compute(pk, oracle):
    import synth
    L, N = 500.0, 256
    a = synth.lognormal_catalog(150000, L, 128, synth.seed_for(13, 1)).double().numpy()
    b = np.concatenate([a[:90000], synth.lognormal_catalog(60000, L, 128, synth.seed_for(13, 2)).double().numpy()])
    dk = 2.5 * 2 * math.pi / L
    cfg = pk.make_config(L, N, "tsc", interlaced=True, dk=dk, nmu=4, batch=2)
    out = {}
    for own in (True, False):
        plan = pk.pk_plan(cfg)
        try:
            pk.pk_use_own_fft(plan, own)
            pk.pk_paint_many(plan, np.concatenate([a, b]), [0, len(a), len(a) + len(b)])
            pk.pk_compute(plan)
            ra, rb = pk.pk_result(plan, 0), pk.pk_result(plan, 1)
            out[own] = (ra, rb, pk.pk_cross(plan, 0, 1), pk.pk_projected(plan, 0, (0, 1)),
                        pk.pk_projected(plan, 1, (2,)))
        finally:
            pk.pk_destroy(plan)
    ra, rb, cross, pxy, pz = out[True]
    ref = oracle.cross_power(a, None, b, None, L, N, "tsc", True, dk=dk, nmu=4)
    assert np.array_equal(cross["modes"], ref["modes"])
    ok = ref["modes"] > 0
    scale = np.sqrt((ra["power"] + ra["shot_noise"]) * (rb["power"] + rb["shot_noise"]))
    d = np.abs(cross["power"] - ref["power"])[ok]
    assert np.all(d <= TOL_ORACLE * scale[ok]), np.max(d / scale[ok])
    for got, pos, axes in ((pxy, a, (0, 1)), (pz, b, (2,))):
        refp = oracle.projected_power(pos, None, L, N, "tsc", True, dk=dk, axes=axes)
        assert np.array_equal(got["modes"], refp["modes"])
        okp = refp["modes"] > 0
        dp = np.abs(got["power"] - refp["power"])[okp]
        sp = refp["power_raw"][okp] + refp["shot_noise"]
        assert np.all(dp <= TOL_ORACLE * sp), np.max(dp / sp)
    # the cuFFT path on the same meshes
    _, _, cross_l, pxy_l, pz_l = out[False]
    assert np.all(np.abs(cross["power"] - cross_l["power"])[ok] <= TOL_PATHS * scale[ok])
    for got, lib in ((pxy, pxy_l), (pz, pz_l)):
        okp = lib["modes"] > 0
        sp = np.abs(lib["power"][okp]) + lib["shot_noise"]
        assert np.all(np.abs(got["power"] - lib["power"])[okp] <= TOL_PATHS * sp)


def test_cross_and_projected_after_own_compute_at_1024(pk):
    # the CTA-per-pair z pass and its in-place finish (N = 1024): cross and
    # projected power against the cuFFT path on the same meshes
    import synth
    L, N = 1000.0, 1024
    a = synth.lognormal_catalog(1_000_000, L, 256, synth.seed_for(14, 1)).numpy()
    b = np.concatenate([a[:600000], synth.lognormal_catalog(400000, L, 256, synth.seed_for(14, 2)).numpy()])
    cfg = pk.make_config(L, N, "tsc", interlaced=True, dk=0.01, nmu=4, batch=2)
    out = {}
    for own in (True, False):
        plan = pk.pk_plan(cfg)
        try:
            pk.pk_use_own_fft(plan, own)
            pk.pk_paint_many(plan, np.concatenate([a, b]), [0, len(a), len(a) + len(b)])
            pk.pk_compute(plan)
            ra, rb = pk.pk_result(plan, 0), pk.pk_result(plan, 1)
            out[own] = (ra, rb, pk.pk_cross(plan, 0, 1), pk.pk_projected(plan, 1, (0, 2)))
        finally:
            pk.pk_destroy(plan)
    for k in (0, 1):
        _check_bins(out[True][k], out[False][k], out[False][k]["power"] + out[False][k]["shot_noise"], TOL_PATHS)
    ra, rb, cross, proj = out[False]
    ok = cross["modes"] > 0
    scale = np.sqrt((ra["power"] + ra["shot_noise"]) * (rb["power"] + rb["shot_noise"]))
    assert np.array_equal(out[True][2]["modes"], cross["modes"])
    assert np.all(np.abs(out[True][2]["power"] - cross["power"])[ok] <= TOL_PATHS * scale[ok])
    okp = proj["modes"] > 0
    sp = np.abs(proj["power"][okp]) + proj["shot_noise"]
    assert np.array_equal(out[True][3]["modes"], proj["modes"])
    assert np.all(np.abs(out[True][3]["power"] - proj["power"])[okp] <= TOL_PATHS * sp)


def test_own_transform_switch(pk):
    for cfg in (pk.make_config(100.0, 48, "cic", dk=0.2), pk.make_config(100.0, 256, "cic", dk=0.2, precision="f64")):
        plan = pk.pk_plan(cfg)
        try:
            with pytest.raises(pk.PkError) as e:
                pk.pk_use_own_fft(plan, True)
            assert e.value.status == pk.PK_EINVAL
            pk.pk_use_own_fft(plan, False)
        finally:
            pk.pk_destroy(plan)
    plan = pk.pk_plan(pk.make_config(100.0, 256, "cic", dk=0.2))
    try:
        pk.pk_use_own_fft(plan, True)
        pk.pk_use_own_fft(plan, False)
    finally:
        pk.pk_destroy(plan)
