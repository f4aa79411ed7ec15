"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated per bin b, relative to the bin's pre-subtraction monopole
P_raw,0(b) because shot-subtracted powers and P_2, P_4 cross zero):
  FP32 mesh form (int64 fixed paint -> FP32 mesh -> cuFFT R2C -> FP64 bin sums):
      |dP| <= 1e-4 P_raw,0(b)
  FP64 mesh form (int64 fixed paint -> FP64 mesh -> cuFFT D2Z -> FP64 sums):
      |dP| <= 1e-6 P_raw,0(b)
  mode counts (1D and 2D): bit-exact.
  mean k, mean mu (geometry only, FP64): relative 1e-12.
Painted meshes are compared cell by cell with the oracle's paint.
"""
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
def torch_mod(pk):
    import torch
    return torch


def run_gpu(pk, pos, weights, L, N, window, interlaced, dk, nmu=0, precision="f32",
            compensated=True, stream=None, kmin=0.0, kmax=None, subtract_shot=True, variant="sort"):
    cfg = pk.make_config(L, N, window, interlaced=interlaced, compensated=compensated, dk=dk,
                         nmu=nmu, precision=precision, kmin=kmin, kmax=kmax,
                         subtract_shot=subtract_shot, paint_variant=variant)
    plan = pk.pk_plan(cfg, stream)
    try:
        pk.pk_paint(plan, pos, weights)
        pk.pk_compute(plan)
        return pk.pk_result(plan, 0)
    finally:
        pk.pk_destroy(plan)


def as_np64(a):
    if a is None:
        return None
    if hasattr(a, "cpu"):
        return a.double().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def run_oracle(oracle, pos, weights, L, N, window, interlaced, dk, nmu=0, compensated=True,
               kmin=0.0, kmax=None, subtract_shot=True):
    return oracle.fft_power(as_np64(pos), as_np64(weights), L, N, window, interlaced, compensated,
                            dk=dk, kmin=kmin, kmax=kmax, nmu=nmu, subtract_shot=subtract_shot)


def compare(got, ref, tol, nmu=0, ktol=1e-12):
    """ktol: the mean k of a bin is an FP64 sum over its modes in another
    order on each side (relative error up to ~ modes x 1e-16)."""
    assert got["nk"] == ref["nk"]
    assert np.array_equal(got["modes"], ref["modes"]), "1D mode counts differ"
    ok = ref["modes"] > 0
    assert np.all(np.isnan(got["power"][~ok]))
    scale = ref["power_raw"][ok]
    np.testing.assert_allclose(got["k"][ok], ref["k"][ok], rtol=ktol)
    errs = {"P": np.max(np.abs(got["power"][ok] - ref["power"][ok]) / scale)}
    for ell in range(3):
        errs["P%d" % (2 * ell)] = np.max(np.abs(got["poles"][ell][ok] - ref["poles"][ell][ok]) / scale)
    if nmu:
        assert np.array_equal(got["modes2d"], ref["modes2d"]), "2D mode counts differ"
        ok2 = ref["modes2d"] > 0
        np.testing.assert_allclose(got["k2d"][ok2], ref["k2d"][ok2], rtol=ktol)
        np.testing.assert_allclose(got["mu2d"][ok2], ref["mu2d"][ok2], rtol=ktol, atol=1e-15)
        sc2 = np.broadcast_to(ref["power_raw"][:, None], ok2.shape)[ok2]
        errs["Pkmu"] = np.max(np.abs(got["power2d"][ok2] - ref["power2d"][ok2]) / sc2)
    assert abs(got["shot_noise"] - ref["shot_noise"]) <= 1e-12 * ref["shot_noise"]
    assert abs(got["wsum"] - ref["wsum"]) <= 1e-12 * abs(ref["wsum"])
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)
    return errs


# ------------------------------------------------------------ paint step --

@pytest.mark.parametrize("variant", ["sort", "atomic"])
@pytest.mark.parametrize("window,interlaced", [("cic", False), ("tsc", True), ("pcs", True), ("cic", True)])
@pytest.mark.parametrize("N", [32, 40])
@pytest.mark.parametrize("form", ["f64 weighted", "f32 unit"])
def test_painted_mesh_matches_oracle_cell_by_cell(pk, oracle, window, interlaced, N, variant, form):
    """Weighted FP64-mesh paint and unit-weight FP32 paint (the one-sweep
    path of 16^3 tiles at N = 32; N = 40 uses 10^3 tiles) against the
    oracle's per-cell sums, including objects on the box faces and outside it."""
    rng = np.random.default_rng(1000 + N)
    L = 250.0
    pos = rng.uniform(-0.5 * L, 1.5 * L, size=(20000, 3))
    pos[:8] = [[0, 0, 0], [L, L, L], [L - 1e-9, 0, 0], [-1e-9, 3.0, 7.0],
               [L / N * 5, L / N * 7, L / N * 9], [L / N * 5.5, 0.5 * L / N, L],
               [3 * L, -2 * L, 0.25 * L], [1e-300, 1e-300, 1e-300]]
    weighted = form == "f64 weighted"
    w = rng.uniform(0.2, 2.0, 20000).astype(np.float32) if weighted else None
    cfg = pk.make_config(L, N, window, interlaced=interlaced, dk=2 * math.pi / L * 2,
                         precision="f64" if weighted else "f32", paint_variant=variant)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint(plan, pos, w)
        for m in range(2 if interlaced else 1):
            got = pk.pk_mesh(plan, 0, m, N, f64=weighted).astype(np.float64)
            ref = oracle.paint(pos, None if w is None else w.astype(np.float64), L, N, window, 0.5 * m)
            err = np.abs(got - ref)
            assert np.max(err) <= 1e-5 * (1.0 + np.max(np.abs(ref))), (m, np.max(err))
            assert abs(got.sum() - ref.sum()) <= 1e-6 * ref.sum()
    finally:
        pk.pk_destroy(plan)


@pytest.mark.parametrize("variant", ["sort", "atomic"])
def test_mesh_is_bit_identical_and_order_free(pk, torch_mod, variant):
    """int64 fixed-point paint: the same catalog, painted twice and painted in
    a shuffled order, gives byte-identical meshes (both paint variants)."""
    torch = torch_mod
    import synth
    L, N = 1000.0, 64
    pos = synth.lognormal_catalog(300000, L, N, synth.seed_for(2, 7), device="cuda")
    perm = torch.randperm(pos.shape[0], device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    cfg = pk.make_config(L, N, "tsc", interlaced=True, dk=0.02, paint_variant=variant)
    plan = pk.pk_plan(cfg)
    try:
        meshes = []
        for p in (pos, pos, pos[perm].contiguous()):
            pk.pk_paint(plan, p)
            meshes.append([pk.pk_mesh(plan, 0, m, N) for m in range(2)])
        for m in range(2):
            assert meshes[0][m].tobytes() == meshes[1][m].tobytes()
            assert meshes[0][m].tobytes() == meshes[2][m].tobytes()
    finally:
        pk.pk_destroy(plan)


# ------------------------------------------------------- full-path parity --

def test_tiny_uniform_cic_both_precisions_host_and_device(pk, oracle, torch_mod):
    """The tiny plain workload: 100,000 uniform objects, FP64 positions,
    L = 1000, CIC on N = 64, no interlacing, dk = 0.01 to k_N, shot noise
    subtracted."""
    import synth
    L, N, dk = 1000.0, 64, 0.01
    pos = synth.uniform_catalog(100000, L, synth.seed_for(1))
    ref = run_oracle(oracle, pos, None, L, N, "cic", False, dk)
    assert ref["nk"] == 20
    for prec in ("f32", "f64"):
        compare(run_gpu(pk, pos, None, L, N, "cic", False, dk, precision=prec), ref, TOL[prec])
        dpos = torch_mod.from_numpy(pos).cuda()
        compare(run_gpu(pk, dpos, None, L, N, "cic", False, dk, precision=prec), ref, TOL[prec])


@pytest.mark.parametrize("window", ["cic", "tsc", "pcs"])
@pytest.mark.parametrize("interlaced", [False, True])
@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("variant", ["sort", "atomic"])
def test_window_interlace_precision_matrix(pk, oracle, torch_mod, window, interlaced, precision, variant):
    import synth
    L, N = 800.0, 48
    pos = synth.lognormal_catalog(60000, L, N, synth.seed_for(2, 11), device="cuda",
                                  dtype=torch_mod.float32 if precision == "f32" else torch_mod.float64)
    w = (torch_mod.rand(pos.shape[0], device="cuda", generator=torch_mod.Generator("cuda").manual_seed(4))
         + 0.5).float()
    dk = 1.5 * 2 * math.pi / L
    ref = run_oracle(oracle, pos, w, L, N, window, interlaced, dk, nmu=10)
    got = run_gpu(pk, pos, w, L, N, window, interlaced, dk, nmu=10, precision=precision, variant=variant)
    compare(got, ref, TOL[precision], nmu=10)


@pytest.mark.parametrize("N,tile", [(36, 0), (40, 0), (6, 0), (4, 0), (64, 8), (72, 18)])
def test_ragged_and_small_tiles(pk, oracle, N, tile):
    rng = np.random.default_rng(N)
    L = 100.0
    pos = rng.uniform(0, L, size=(5000, 3))
    dk = 2 * math.pi / L
    ref = run_oracle(oracle, pos, None, L, N, "pcs", True, dk, nmu=4)
    cfg = pk.make_config(L, N, "pcs", interlaced=True, dk=dk, nmu=4, precision="f64", tile=tile)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint(plan, pos)
        pk.pk_compute(plan)
        compare(pk.pk_result(plan), ref, TOL["f64"], nmu=4)
    finally:
        pk.pk_destroy(plan)


@pytest.mark.parametrize("N", [4, 6, 36])
def test_atomic_variant_small_and_ragged_meshes(pk, oracle, N):
    """The atomic variant wraps each deposit itself: windows wider than half
    the mesh (PCS interlaced reaches 5 cells on N = 4) and N not a multiple
    of 4."""
    rng = np.random.default_rng(300 + N)
    L = 100.0
    pos = rng.uniform(-L, 2 * L, size=(5000, 3))
    dk = 2 * math.pi / L
    ref = run_oracle(oracle, pos, None, L, N, "pcs", True, dk, nmu=4)
    got = run_gpu(pk, pos, None, L, N, "pcs", True, dk, nmu=4, precision="f64", variant="atomic")
    compare(got, ref, TOL["f64"], nmu=4)


def test_kmin_kmax_and_unsubtracted(pk, oracle):
    rng = np.random.default_rng(77)
    L, N = 300.0, 32
    pos = rng.uniform(0, L, size=(30000, 3))
    kF = 2 * math.pi / L
    kw = dict(kmin=3.3 * kF, kmax=14.2 * kF, subtract_shot=False)
    ref = run_oracle(oracle, pos, None, L, N, "tsc", False, 0.7 * kF, nmu=3, **kw)
    got = run_gpu(pk, pos, None, L, N, "tsc", False, 0.7 * kF, nmu=3, precision="f64", **kw)
    compare(got, ref, TOL["f64"], nmu=3)


def test_mesh_above_512_uses_single_mesh_transforms(pk, oracle):
    """N = 528 (> 512): each mesh gets its own cuFFT call instead of one plan
    batched over the interlaced pair; full pipeline against the oracle, with
    (k, mu) bins and multipoles, in both precision forms."""
    import synth
    L, N = 1056.0, 528
    pos = synth.lognormal_catalog(200000, L, 64, synth.seed_for(2, 7)).double().numpy()
    dk = 4 * (2 * math.pi / L)
    ref = run_oracle(oracle, pos, None, L, N, "tsc", True, dk, nmu=4)
    for precision in ("f32", "f64"):
        got = run_gpu(pk, pos, None, L, N, "tsc", True, dk, nmu=4, precision=precision)
        compare(got, ref, TOL[precision], nmu=4, ktol=1e-10)


def test_uncompensated(pk, oracle):
    rng = np.random.default_rng(78)
    L, N = 300.0, 32
    pos = rng.uniform(0, L, size=(30000, 3))
    dk = 2 * math.pi / L
    ref = run_oracle(oracle, pos, None, L, N, "cic", True, dk, compensated=False)
    got = run_gpu(pk, pos, None, L, N, "cic", True, dk, compensated=False)
    compare(got, ref, TOL["f32"])


# ------------------------------------------------------------ edge cases --

def test_empty_catalog_gives_nan_not_a_crash(pk):
    cfg = pk.make_config(100.0, 16, "cic", dk=0.2)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint(plan, np.zeros((0, 3)))
        pk.pk_compute(plan)
        r = pk.pk_result(plan)
        assert r["wsum"] == 0.0 and np.all(np.isnan(r["power"]))
        assert np.all(r["modes"][1:] > 0)
    finally:
        pk.pk_destroy(plan)


@pytest.mark.parametrize("variant", ["sort", "atomic"])
def test_single_object_and_one_dense_cell(pk, oracle, variant):
    L, N = 64.0, 16
    dk = 2 * math.pi / L
    one = np.array([[12.3, 45.6, 63.999]])
    compare(run_gpu(pk, one, None, L, N, "pcs", True, dk, precision="f64", variant=variant),
            run_oracle(oracle, one, None, L, N, "pcs", True, dk), TOL["f64"])
    dense = np.tile(np.array([[20.01, 20.02, 20.03]]), (200000, 1))
    compare(run_gpu(pk, dense, None, L, N, "tsc", True, dk, precision="f64", variant=variant),
            run_oracle(oracle, dense, None, L, N, "tsc", True, dk), TOL["f64"])


@pytest.mark.parametrize("variant", ["sort", "atomic"])
def test_batch_equals_single(pk, torch_mod, variant):
    import synth
    L, N = 500.0, 32
    sizes = [1000, 25000, 0, 7000]
    cats = [synth.lognormal_catalog(max(n, 1), L, N, synth.seed_for(4, k), device="cuda")[:n]
            for k, n in enumerate(sizes)]
    allpos = torch_mod.cat(cats).contiguous()
    off = np.concatenate([[0], np.cumsum(sizes)])
    cfg = pk.make_config(L, N, "tsc", dk=2 * math.pi / L, nmu=4, batch=len(sizes), paint_variant=variant)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint_many(plan, allpos, off)
        pk.pk_compute(plan)
        batched = [pk.pk_result(plan, k) for k in range(len(sizes))]
    finally:
        pk.pk_destroy(plan)
    for k, n in enumerate(sizes):
        if n == 0:
            assert np.all(np.isnan(batched[k]["power"]))
            continue
        single = run_gpu(pk, cats[k].contiguous(), None, L, N, "tsc", False, 2 * math.pi / L, nmu=4,
                         variant=variant)
        ok = single["modes"] > 0
        raw = single["power"] + single["shot_noise"]          # pre-subtraction power
        assert np.all(np.abs(batched[k]["power"] - single["power"])[ok] <= 1e-6 * raw[ok])
        ok2 = single["modes2d"] > 0
        raw2 = np.broadcast_to(raw[:, None], ok2.shape)
        assert np.all(np.abs(batched[k]["power2d"] - single["power2d"])[ok2] <= 1e-6 * raw2[ok2])
        assert np.all(np.isnan(batched[k]["power2d"][~ok2]))


def test_partial_batches_transform_only_what_was_painted(pk, torch_mod):
    """A batch-8 plan computing 1, 3, 5, 8 and 7 catalogs in turn (the FFT runs
    over the painted catalogs only, as a sum of power-of-two plans) gives
    each catalog's single-plan result."""
    import synth
    L, N = 400.0, 32
    dk = 2 * math.pi / L
    cats = [synth.lognormal_catalog(4000 + 1500 * k, L, N, synth.seed_for(4, 300 + k), device="cuda")
            for k in range(8)]
    single = [run_gpu(pk, c, None, L, N, "cic", True, dk) for c in cats]
    plan = pk.pk_plan(pk.make_config(L, N, "cic", interlaced=True, dk=dk, batch=8))
    try:
        for n in (1, 3, 5, 8, 7):
            sel = cats[8 - n:]
            off = np.concatenate([[0], np.cumsum([c.shape[0] for c in sel])])
            pk.pk_paint_many(plan, torch_mod.cat(sel).contiguous(), off)
            pk.pk_compute(plan)
            for k in range(n):
                got, ref = pk.pk_result(plan, k), single[8 - n + k]
                ok = ref["modes"] > 0
                raw = ref["power"] + ref["shot_noise"]
                assert np.all(np.abs(got["power"] - ref["power"])[ok] <= 1e-5 * raw[ok]), (n, k)
    finally:
        pk.pk_destroy(plan)


@pytest.mark.parametrize("variant", ["sort", "atomic"])
def test_accumulate_matches_single_paint(pk, variant):
    rng = np.random.default_rng(5)
    L, N = 200.0, 32
    pos = rng.uniform(0, L, size=(40000, 3)).astype(np.float32)
    cfg = pk.make_config(L, N, "tsc", interlaced=True, dk=2 * math.pi / L, paint_variant=variant)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint(plan, pos)
        pk.pk_compute(plan)
        whole = pk.pk_result(plan)
        pk.pk_paint(plan, pos[:15000].copy())
        pk.pk_paint(plan, pos[15000:].copy(), accumulate=True)
        pk.pk_compute(plan)
        parts = pk.pk_result(plan)
    finally:
        pk.pk_destroy(plan)
    assert whole["wsum"] == parts["wsum"] == 40000.0
    ok = whole["modes"] > 0
    raw = whole["power"] + whole["shot_noise"]                 # pre-subtraction power
    assert np.all(np.abs(parts["power"] - whole["power"])[ok] <= 1e-5 * raw[ok])


def test_call_order_errors(pk):
    cfg = pk.make_config(100.0, 16, "cic", dk=0.2)
    plan = pk.pk_plan(cfg)
    try:
        with pytest.raises(pk.PkError) as e:
            pk.pk_compute(plan)
        assert e.value.status == pk.PK_ESTATE
        with pytest.raises(pk.PkError) as e:
            pk.pk_result(plan)
        assert e.value.status == pk.PK_ESTATE
        pos = np.random.default_rng(1).uniform(0, 100, (100, 3))
        pk.pk_paint(plan, pos)
        pk.pk_compute(plan)
        with pytest.raises(pk.PkError) as e:
            pk.pk_paint(plan, pos, accumulate=True)
        assert e.value.status == pk.PK_ESTATE
        with pytest.raises(pk.PkError) as e:
            pk.pk_result(plan, 1)
        assert e.value.status == pk.PK_EINVAL
        x4 = np.zeros((10, 4), np.float32)
        with pytest.raises(pk.PkError) as e:
            pk.pk_paint(plan, x4, weights=np.ones(10, np.float32))
        assert e.value.status == pk.PK_EINVAL
    finally:
        pk.pk_destroy(plan)


@pytest.mark.parametrize("variant", ["sort", "atomic"])
def test_overflow_headroom_reported(pk, variant):
    cfg = pk.make_config(100.0, 16, "cic", dk=0.2, fixed_scale_log2=40, paint_variant=variant)
    plan = pk.pk_plan(cfg)
    try:
        pos = np.random.default_rng(2).uniform(0, 100, (10, 3))
        pk.pk_paint(plan, pos, weights=np.full(10, 1e6, np.float32))
        pk.pk_compute(plan)
        with pytest.raises(pk.PkError) as e:
            pk.pk_result(plan)
        assert e.value.status == pk.PK_EOVERFLOW
    finally:
        pk.pk_destroy(plan)


def test_xyzw_layout_and_stream(pk, oracle, torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(9)
    L, N = 400.0, 32
    xyz = rng.uniform(0, L, size=(50000, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 50000).astype(np.float32)
    x4 = torch.from_numpy(np.concatenate([xyz, w[:, None]], axis=1)).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = run_gpu(pk, x4, None, L, N, "tsc", True, 2 * math.pi / L, nmu=5, stream=s)
    ref = run_oracle(oracle, xyz, w, L, N, "tsc", True, 2 * math.pi / L, nmu=5)
    compare(got, ref, TOL["f32"], nmu=5)


# ---------------------------------------------- the 512^3 lognormal workload --

@pytest.fixture(scope="module")
def lognormal_512(torch_mod):
    import synth
    pos = synth.lognormal_catalog(10_000_000, 1000.0, 512, synth.seed_for(2), device="cuda")
    return pos


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_lognormal_1e7_tsc_interlaced_512(pk, oracle, lognormal_512, precision):
    """1e7 objects Poisson-sampled from a log-normal field (P ~ k^-1.5, sigma^2
    ~ 1 at the cell scale) with RSD f = 0.75, L = 1000, TSC + interlacing on
    N = 512, (k, mu) bins dk = 0.005 and 10 mu bins, multipoles 0, 2, 4 --
    in the same launch configuration the benchmark times."""
    L, N, dk = 1000.0, 512, 0.005
    pos = lognormal_512 if precision == "f32" else lognormal_512.double()
    got = run_gpu(pk, pos, None, L, N, "tsc", True, dk, nmu=10, precision=precision)
    ref = _oracle_512(oracle, lognormal_512)
    errs = compare(got, ref, TOL[precision], nmu=10)
    print("lognormal 512 %s max errors:" % precision, errs)


_ORACLE_CACHE = {}


def _oracle_512(oracle, pos):
    if "r" not in _ORACLE_CACHE:
        _ORACLE_CACHE["r"] = run_oracle(oracle, pos, None, 1000.0, 512, "tsc", True, 0.005, nmu=10)
    return _ORACLE_CACHE["r"]


# -------------------------------------- the 2048^3 Zel'dovich workload --

@pytest.fixture(scope="module")
def zeldovich_1024cubed(torch_mod):
    """1024^3 objects on a Zel'dovich-displaced lattice (P ~ k^-2, rms 0.25
    spacings), L = 2000, FP32 positions on the device (12.9 GB)."""
    import synth
    pos = synth.zeldovich_lattice(1024, 2000.0, synth.seed_for(3), device="cuda")
    torch_mod.cuda.synchronize()
    torch_mod.cuda.empty_cache()
    yield pos
    del pos
    torch_mod.cuda.empty_cache()


def with_raw(r):
    """A GPU result used as the reference: add its pre-subtraction monopole."""
    r = dict(r)
    r["power_raw"] = r["power"] + r["shot_noise"]
    return r


def per_bin_errors(got, ref):
    """Largest |got - ref| per quantity over the bins, relative to the
    reference's pre-subtraction monopole of the bin (mode counts must agree)."""
    assert np.array_equal(got["modes"], ref["modes"]) and np.array_equal(got["modes2d"], ref["modes2d"])
    ok = ref["modes"] > 0
    scale = ref["power_raw"][ok]
    errs = {"P": float(np.max(np.abs(got["power"][ok] - ref["power"][ok]) / scale))}
    for ell in range(3):
        errs["P%d" % (2 * ell)] = float(np.max(np.abs(got["poles"][ell][ok] - ref["poles"][ell][ok]) / scale))
    ok2 = ref["modes2d"] > 0
    sc2 = np.broadcast_to(ref["power_raw"][:, None], ok2.shape)[ok2]
    errs["Pkmu"] = float(np.max(np.abs(got["power2d"][ok2] - ref["power2d"][ok2]) / sc2))
    return errs


def test_zeldovich_1024cubed_objects_pcs_interlaced_2048(pk, oracle, torch_mod, zeldovich_1024cubed):
    """1024^3 objects on a Zel'dovich-displaced lattice, PCS + interlacing on
    N = 2048, FP32 mesh with int64 fixed-point paint, (k, mu) bins dk = 0.005
    x 10, multipoles.  The painted field at full size: mass on both meshes,
    sampled cell blocks against the oracle's block paint, and every mode count
    (bit-exact)."""
    torch = torch_mod
    import ctypes
    pos = zeldovich_1024cubed
    L, N, dk, nmu = 2000.0, 2048, 0.005, 10
    n = pos.shape[0]
    cfg = pk.make_config(L, N, "pcs", interlaced=True, dk=dk, nmu=nmu)
    plan = pk.pk_plan(cfg)
    blocks = [((0, 0, 0), 8), ((1019, 517, 2044), 8)]
    try:
        pk.pk_paint(plan, pos)
        host = pos.cpu().double().numpy()
        for m in range(2):
            dev = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
            assert pk.load().pk_mesh(plan, 0, m, ctypes.c_void_p(dev.data_ptr())) == pk.PK_OK
            total = float(dev.sum(dtype=torch.float64))
            assert abs(total - n) <= 1e-6 * n, (m, total, n)
            for c0, B in blocks:
                idx = [torch.arange(c, c + B, device="cuda") % N for c in c0]
                got = dev[idx[0]][:, idx[1]][:, :, idx[2]].double().cpu().numpy()
                ref = oracle.paint_block(host, None, L, N, "pcs", c0, B, 0.5 * m)
                assert np.max(np.abs(got - ref)) <= 1e-5 * (1.0 + np.max(np.abs(ref))), (m, c0)
            del dev
            torch.cuda.empty_cache()
        del host
        pk.pk_compute(plan)
        r = pk.pk_result(plan)
    finally:
        pk.pk_destroy(plan)
    c1, c2 = oracle.mode_counts(N, L, dk, nmu=nmu)
    assert np.array_equal(r["modes"], c1)
    assert np.array_equal(r["modes2d"], c2)
    ok = c1 > 0
    assert r["wsum"] == float(n) and abs(r["shot_noise"] - L ** 3 / n) <= 1e-12 * L ** 3 / n
    assert np.all(np.isfinite(r["power"][ok])) and np.all(r["power"][ok] + r["shot_noise"] > 0)
    assert np.all(np.isfinite(r["poles"][:, ok]))


def test_zeldovich_2048_fp32_form_per_bin_error_against_fp64_form(pk, torch_mod, zeldovich_1024cubed):
    """The per-bin error of the precision form at scale.  The same 1024^3
    objects, PCS + interlacing on N = 2048, in the FP32 form (int64 fixed-point
    paint -> FP32 mesh -> R2C -> FP32 per-CTA bin partials -> FP64 sums) and in
    the FP64 mesh form (FP64 mesh, D2Z, FP64 sums; itself held to 1e-6 of the
    oracle in the tests above and at N = 1024 below).  The FP32 plan is
    destroyed before the FP64 one (two FP64 2048^3 meshes take 137 GB).  Every
    P(k), P(k, mu) and P_l bin must agree within 1e-4 of the bin's
    pre-subtraction monopole."""
    L, N, dk, nmu = 2000.0, 2048, 0.005, 10
    pos = zeldovich_1024cubed
    r32 = run_gpu(pk, pos, None, L, N, "pcs", True, dk, nmu=nmu, precision="f32")
    torch_mod.cuda.empty_cache()
    r64 = run_gpu(pk, pos, None, L, N, "pcs", True, dk, nmu=nmu, precision="f64")
    torch_mod.cuda.empty_cache()
    errs = per_bin_errors(r32, with_raw(r64))
    print("2048^3 FP32 form vs FP64 form, max per-bin error / P_raw,0:", errs)
    bad = {k: v for k, v in errs.items() if not v <= TOL["f32"]}
    assert not bad, (bad, errs)


# The FP64 mesh form sums, transforms and bins in FP64, but its objects enter
# the paint as FP32 coordinates local to their tile (resolution ~1e-6 cell)
# with FP32 window weights.  On a displaced lattice, whose power at high k is
# far below a Poisson sample's, that rounding noise reaches ~2e-6 of a bin's
# power (measured 1.9e-6 at N = 1024), so the lattice is held to 1e-5 in this
# form; the log-normal catalogs above hold it to 1e-6.
TOL_LATTICE_F64 = 1e-5


def test_zeldovich_catalog_at_1024_against_the_oracle(pk, oracle, torch_mod, zeldovich_1024cubed):
    """The oracle cannot hold a 2048^3 FP64 mesh pair plus its transforms on
    the host, so it runs on the same 1.07e9-object catalog at N = 1024 (PCS +
    interlacing, dk = 0.005 x 10 mu bins, multipoles): the FP32 form within
    1e-4 and the FP64 mesh form within TOL_LATTICE_F64 of each bin's
    pre-subtraction monopole, mode counts bit-exact."""
    L, N, dk, nmu = 2000.0, 1024, 0.005, 10
    pos = zeldovich_1024cubed
    got = {prec: run_gpu(pk, pos, None, L, N, "pcs", True, dk, nmu=nmu, precision=prec)
           for prec in ("f32", "f64")}
    torch_mod.cuda.empty_cache()
    host = pos.cpu().double().numpy()
    ref = oracle.fft_power(host, None, L, N, "pcs", True, True, dk=dk, nmu=nmu)
    del host
    for prec, tol in (("f32", TOL["f32"]), ("f64", TOL_LATTICE_F64)):
        errs = compare(got[prec], ref, tol, nmu=nmu, ktol=1e-10)
        print("1.07e9 objects at 1024^3, %s form vs oracle:" % prec, errs)
