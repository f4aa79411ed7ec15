"""Survey multipoles (pk_survey_*, the ConvolvedFFTPower of Sec. 3.4.1)
through the C ABI against the FP64 oracle (oracle/survey.py, which builds A_l
from Cartesian moments while the CUDA path uses spherical harmonics).

Mode counts bit-exact, mean k 1e-12, alpha / I / S 1e-12 (FP64 sums of the
same inputs), P_0, P_2, P_4 within 1e-4 (FP32 form) / 1e-6 (FP64 form) of the
bin's P_0 before shot-noise subtraction."""
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


@pytest.fixture(scope="module")
def sv(oracle):
    import oracle.survey as survey
    return survey


@pytest.fixture(scope="module")
def cats():
    import synth
    return synth.survey_catalogs(30000, 150000, 400.0, synth.seed_for(9, 0), ngrid=64)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _gpu_cat(pk, torch, pos, wcomp=None, nbar=None, wfkp=None, coord="cartesian", device=True):
    p = np.ascontiguousarray(pos, dtype=np.float64)
    cols = [_f32(wcomp), _f32(wfkp), _f32(nbar)]
    if device:
        p = torch.from_numpy(p).cuda()
        cols = [None if c is None else torch.from_numpy(c).cuda() for c in cols]
    keep = (p, cols)
    return pk.survey_catalog(p, coord, wcomp=cols[0], wfkp=cols[1], nbar=cols[2]), keep


def _oracle_cat(pos, wcomp=None, nbar=None, wfkp=None):
    d = {"pos": np.asarray(pos, dtype=np.float64)}
    for k, v in (("wcomp", wcomp), ("nbar", nbar), ("wfkp", wfkp)):
        if v is not None:
            d[k] = np.asarray(v, dtype=np.float32).astype(np.float64)
    return d


def _run_gpu(pk, cfg, data, rand):
    plan = pk.pk_survey_plan(cfg)
    try:
        pk.pk_survey_paint(plan, data, rand)
        pk.pk_survey_compute(plan)
        return pk.pk_survey_result(plan), pk.pk_survey_launch_count(plan)
    finally:
        pk.pk_survey_destroy(plan)


def _compare(got, ref, precision, poles=(0, 2, 4)):
    assert np.array_equal(got["modes"], ref["modes"])
    ok = ref["modes"] > 0
    np.testing.assert_allclose(got["k"][ok], ref["k"][ok], rtol=1e-12)
    for key in ("alpha", "norm", "shot_noise"):
        assert abs(got[key] - ref[key]) <= 1e-12 * abs(ref[key]), key
    scale = np.abs(ref["power_raw"][ok])
    for row, ell in enumerate((0, 2, 4)):
        if ell not in poles:
            assert np.all(np.isnan(got["poles"][row]))
            continue
        d = np.abs(got["poles"][row][ok] - ref["poles"][ell][ok])
        assert np.all(d <= TOL[precision] * scale), (ell, float(np.max(d / scale)))


CASES = [
    # N, window, interlaced, precision, max_batch, poles
    (64, "cic", False, "f32", 0, (0, 2, 4)),
    (48, "tsc", True, "f32", 0, (0, 2, 4)),
    (40, "pcs", True, "f64", 0, (0, 2, 4)),
    (64, "tsc", False, "f64", 4, (0, 2, 4)),
    (48, "pcs", True, "f32", 3, (0, 4)),
    (32, "cic", True, "f32", 0, (0, 2)),
    (36, "tsc", False, "f32", 0, (0,)),
]


@pytest.mark.parametrize("N,window,interlaced,precision,max_batch,poles", CASES)
def test_survey_multipoles_match_oracle(pk, sv, cats, N, window, interlaced, precision, max_batch, poles):
    import torch
    ext = cats["extent"]
    L, origin = 1.04 * ext, (-0.02 * ext,) * 3
    dk = 2 * (2 * math.pi / L)
    d_w, d_nb = cats["data_wcomp"], cats["data_nbar"]
    r_nb = cats["rand_nbar"]
    cfg = pk.make_survey_config(L, origin, N, window, interlaced, dk=dk, poles=poles, precision=precision,
                                max_batch=max_batch)
    gd, kd = _gpu_cat(pk, torch, cats["data"], d_w, d_nb)
    gr, kr = _gpu_cat(pk, torch, cats["randoms"], None, r_nb)
    got, launches = _run_gpu(pk, cfg, gd, gr)
    ref = sv.convolved_power(_oracle_cat(cats["data"], d_w, d_nb), _oracle_cat(cats["randoms"], None, r_nb),
                             L, origin, N, window, interlaced, True, dk, poles=poles)
    _compare(got, ref, precision, poles)
    assert got["n_data"] == len(cats["data"]) and got["n_randoms"] == len(cats["randoms"])
    assert got["n_outside"] == 0 and got["n_rejected"] == 0
    assert launches > 0


def test_survey_fkp_weights_and_observer_on_a_node(pk, sv, cats):
    """FKP weights from nbar and P0, the observer exactly on mesh node
    (N/2, N/2, N/2) (a node without a line of sight), uncompensated."""
    import torch
    ext = cats["extent"]
    N, L = 50, 2.0 * ext                    # H = 16 exactly
    origin = (-ext, -ext, -ext)             # node (25, 25, 25) at the observer
    dk = 2 * (2 * math.pi / L)
    p0 = 2e4
    cfg = pk.make_survey_config(L, origin, N, "tsc", False, compensated=False, dk=dk, p0_fkp=p0)
    gd, kd = _gpu_cat(pk, torch, cats["data"], cats["data_wcomp"], cats["data_nbar"])
    gr, kr = _gpu_cat(pk, torch, cats["randoms"], None, cats["rand_nbar"])
    got, _ = _run_gpu(pk, cfg, gd, gr)
    ref = sv.convolved_power(_oracle_cat(cats["data"], cats["data_wcomp"], cats["data_nbar"]),
                             _oracle_cat(cats["randoms"], None, cats["rand_nbar"]), L, origin, N, "tsc", False,
                             False, dk, p0_fkp=p0)
    _compare(got, ref, "f32")


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_survey_sky_coordinates(pk, sv, precision):
    """(RA, Dec, z) input: the device's tabulated chi(z) against the oracle's
    quadrature; objects with z outside [0, zmax] are rejected (weight 0)."""
    import torch
    import synth
    om = 0.31
    d = synth.survey_sky(20000, 41)
    r = synth.survey_sky(100000, 42)
    d["z"][:5] = [-0.1, 6.0, np.nan, 0.3, 0.4]           # three rejected
    keep = np.isfinite(d["z"]) & (d["z"] >= 0) & (d["z"] <= 5.0)
    xd = sv.sky_to_cartesian(d["ra"][keep], d["dec"][keep], d["z"][keep], om)
    xr = sv.sky_to_cartesian(r["ra"], r["dec"], r["z"], om)
    lo = np.minimum(xd.min(0), xr.min(0))
    hi = np.maximum(xd.max(0), xr.max(0))
    L = float(np.max(hi - lo)) * 1.05
    origin = tuple(lo - 0.025 * L)
    N = 48
    dk = 2 * (2 * math.pi / L)
    cfg = pk.make_survey_config(L, origin, N, "cic", True, dk=dk, precision=precision, omega_m=om)
    sky_d = np.stack([d["ra"], d["dec"], d["z"]], axis=1)
    sky_r = np.stack([r["ra"], r["dec"], r["z"]], axis=1)
    gd, kd = _gpu_cat(pk, torch, sky_d, d["wcomp"], d["nbar"], coord="sky")
    gr, kr = _gpu_cat(pk, torch, sky_r, r["wcomp"], r["nbar"], coord="sky")
    got, _ = _run_gpu(pk, cfg, gd, gr)
    ref = sv.convolved_power(
        {"pos": xd, "wcomp": d["wcomp"][keep].astype(np.float32).astype(np.float64),
         "nbar": d["nbar"][keep].astype(np.float32).astype(np.float64)},
        {"pos": xr, "wcomp": r["wcomp"].astype(np.float32).astype(np.float64),
         "nbar": r["nbar"].astype(np.float32).astype(np.float64)},
        L, origin, N, "cic", True, True, dk)
    assert got["n_rejected"] == 3 and got["n_outside"] == 0
    _compare(got, ref, precision)


def test_survey_reuses_randoms_and_host_inputs(pk, cats):
    """randoms=None keeps the randoms of the previous paint; host (numpy)
    inputs give the same result as device inputs (up to the summation order
    of the FP32 bin histograms)."""
    import torch
    import synth
    ext = cats["extent"]
    L, origin, N = 1.04 * ext, (-0.02 * ext,) * 3, 48
    cfg = pk.make_survey_config(L, origin, N, "tsc", True)
    other = synth.survey_catalogs(25000, 1000, ext, synth.seed_for(9, 1), ngrid=64)
    gd, kd = _gpu_cat(pk, torch, cats["data"], cats["data_wcomp"], cats["data_nbar"])
    gr, kr = _gpu_cat(pk, torch, cats["randoms"], None, cats["rand_nbar"])
    g2, k2 = _gpu_cat(pk, torch, other["data"], other["data_wcomp"], other["data_nbar"])
    h2, kh = _gpu_cat(pk, torch, other["data"], other["data_wcomp"], other["data_nbar"], device=False)
    hr, khr = _gpu_cat(pk, torch, cats["randoms"], None, cats["rand_nbar"], device=False)
    plan = pk.pk_survey_plan(cfg)
    try:
        pk.pk_survey_paint(plan, gd, gr)
        pk.pk_survey_compute(plan)
        pk.pk_survey_result(plan)
        pk.pk_survey_paint(plan, g2, None)
        pk.pk_survey_compute(plan)
        reused = pk.pk_survey_result(plan)
    finally:
        pk.pk_survey_destroy(plan)
    fresh, _ = _run_gpu(pk, cfg, g2, gr)
    host, _ = _run_gpu(pk, cfg, h2, hr)
    # the meshes and the FP64 catalog sums are bit-identical; the per-CTA FP32
    # histograms add in the order the shared-memory atomics land
    ok = fresh["modes"] > 0
    scale = np.abs(fresh["poles"][0][ok])
    for res in (reused, host):
        assert np.array_equal(res["modes"], fresh["modes"])
        assert np.all(np.abs(res["poles"][:, ok] - fresh["poles"][:, ok]) <= 1e-6 * scale)
        assert res["alpha"] == fresh["alpha"] and res["norm"] == fresh["norm"]


def test_survey_argument_errors(pk, cats):
    import torch
    ext = cats["extent"]
    cfg = pk.make_survey_config(1.04 * ext, (-0.02 * ext,) * 3, 32, omega_m=0.0)
    gd, kd = _gpu_cat(pk, torch, cats["data"][:100], None, cats["data_nbar"][:100])
    no_nbar, k1 = _gpu_cat(pk, torch, cats["randoms"][:100])
    sky, k2 = _gpu_cat(pk, torch, cats["randoms"][:100], None, cats["rand_nbar"][:100], coord="sky")
    plan = pk.pk_survey_plan(cfg)
    try:
        with pytest.raises(pk.PkError) as e:
            pk.pk_survey_paint(plan, gd, None)
        assert e.value.status == pk.PK_ESTATE
        with pytest.raises(pk.PkError) as e:
            pk.pk_survey_paint(plan, gd, no_nbar)
        assert e.value.status == pk.PK_EINVAL and "nbar" in str(e.value)
        with pytest.raises(pk.PkError) as e:
            pk.pk_survey_paint(plan, gd, sky)
        assert e.value.status == pk.PK_EINVAL and "omega_m" in str(e.value)
        with pytest.raises(pk.PkError) as e:
            pk.pk_survey_compute(plan)
        assert e.value.status == pk.PK_ESTATE
    finally:
        pk.pk_survey_destroy(plan)


def test_survey_empty_data_and_single_random(pk, cats):
    """No data objects: alpha = 0 and I = 0, so every P_l is NaN (no crash);
    a one-object random catalog is accepted."""
    import torch
    ext = cats["extent"]
    cfg = pk.make_survey_config(1.04 * ext, (-0.02 * ext,) * 3, 32)
    empty = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    gd = pk.survey_catalog(empty)
    gr, kr = _gpu_cat(pk, torch, cats["randoms"][:1], None, cats["rand_nbar"][:1])
    got, _ = _run_gpu(pk, cfg, gd, gr)
    assert got["n_data"] == 0 and got["alpha"] == 0.0 and got["norm"] == 0.0
    assert np.all(np.isnan(got["poles"][:, got["modes"] > 0]))


@pytest.mark.parametrize("device", [True, False])
def test_survey_bounds_match_the_oracle(pk, sv, device):
    """Device bounds of sky (RA, Dec, z) and Cartesian catalogs against the
    oracle's conversion; rejected redshifts are skipped."""
    import torch
    import synth
    om = 0.31
    d = synth.survey_sky(50000, 43)
    d["z"][:3] = [-0.5, 7.0, np.nan]
    keep = np.isfinite(d["z"]) & (d["z"] >= 0) & (d["z"] <= 5.0)
    x = sv.sky_to_cartesian(d["ra"][keep], d["dec"][keep], d["z"][keep], om)
    sky = np.stack([d["ra"], d["dec"], d["z"]], axis=1)
    cat, k = _gpu_cat(pk, torch, sky, coord="sky", device=device)
    lo, hi = pk.pk_survey_bounds(cat, omega_m=om)
    scale = float(np.max(np.abs(x)))
    assert np.all(np.abs(lo - x.min(0)) <= 1e-9 * scale) and np.all(np.abs(hi - x.max(0)) <= 1e-9 * scale)
    cat2, k2 = _gpu_cat(pk, torch, x, device=device)
    lo2, hi2 = pk.pk_survey_bounds(cat2)
    assert np.array_equal(lo2, x.min(0)) and np.array_equal(hi2, x.max(0))
    L, origin = pk.survey_box(lo, hi, pad=0.02)
    cfg = pk.make_survey_config(L, origin, 32, omega_m=om)
    rcat, kr = _gpu_cat(pk, torch, sky[keep][:2000], None, d["nbar"][keep][:2000], coord="sky", device=device)
    dcat, kd = _gpu_cat(pk, torch, sky, None, None, coord="sky", device=device)
    got, _ = _run_gpu(pk, cfg, dcat, rcat)
    assert got["n_outside"] == 0 and got["n_rejected"] == 3
