"""The allocation-free binning entry point, pk_bin_static, through the C ABI.

Some callers cannot call cudaMalloc: a framework that is capturing a stream
into a CUDA graph and owns all device memory, a program whose device memory is
handed out by a pool it does not control, or a host that forbids allocation
after start-up.  pk_bin_static lets them bin transforms they already hold,
using a fixed scratch array inside the library instead of allocating.

Each case paints a catalog through the plan path (pk_plan / pk_paint), copies
out the painted meshes, transforms them with torch's FFT, and calls
pk_bin_static twice in a row on those transforms, with and without
interlacing, (k, mu) bins and multipoles.  Each call's raw sums must

* equal the FP64 oracle's mode loop on the very same transforms (the sums of
  h |d|^2, h |d|^2 L_2(mu), h |d|^2 L_4(mu) per bin) within 1e-5 of the bin's
  monopole sum: the inputs are identical, so only the kernel's FP32 per-mode
  arithmetic and per-CTA partials differ;
* normalized with the plan path's mode counts and weights, reproduce the plan
  path's P(k), P(k, mu), P_2 and P_4 within the FP32-form tolerance used
  throughout the tests: 1e-4 of each bin's pre-subtraction monopole;

and the second call must leave the device's free memory unchanged.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-4
TOL_SAME_INPUT = 1e-5


@pytest.mark.parametrize("poles", [(0,), (0, 2, 4)])
@pytest.mark.parametrize("nmu", [0, 5])
@pytest.mark.parametrize("interlaced", [False, True])
def test_static_bin_matches_oracle_and_plan_path_on_two_calls(oracle, interlaced, nmu, poles):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    import synth

    pk.build()
    lib = pk.load()
    L, N = 600.0, 64
    dk = 2 * (2 * math.pi / L)
    pos = synth.lognormal_catalog(200000, L, N, synth.seed_for(5, 1), device="cuda")
    cfg = pk.make_config(L, N, "tsc", interlaced=interlaced, dk=dk, nmu=nmu, poles=poles)
    plan = pk.pk_plan(cfg)
    nm = 2 if interlaced else 1
    try:
        pk.pk_paint(plan, pos)
        meshes = [pk.pk_mesh(plan, 0, m, N) for m in range(nm)]
        pk.pk_compute(plan)
        ref = pk.pk_result(plan, 0)
    finally:
        pk.pk_destroy(plan)

    transforms = [torch.fft.rfftn(torch.from_numpy(m).cuda()).contiguous() for m in meshes]
    assert transforms[0].shape == (N, N, N // 2 + 1) and transforms[0].dtype == torch.complex64
    host = [t.cpu().numpy().astype(np.complex128) for t in transforms]
    osum = oracle.bin_modes(host[0], host[1] if interlaced else None, L, "tsc", True, 1.0, dk, nmu=nmu)
    L3 = L ** 3                                       # the oracle's sums carry P = L^3 |d|^2
    nk = ref["nk"]
    with_poles = 2 in poles or 4 in poles
    hb = nk * max(nmu, 1)
    nh = hb + (2 * nk if with_poles else 0)
    norm = L ** 3 / ref["wsum"] ** 2
    shot = ref["shot_noise"]
    modes = ref["modes"].astype(np.float64)
    ok = modes > 0
    raw0 = ref["power"] + shot                       # pre-subtraction monopole
    S0_oracle = osum["psum1d"] / L3
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    m2_ptr = transforms[1].data_ptr() if interlaced else None
    for call in range(2):
        sums = torch.full((nh,), float("nan"), dtype=torch.float64, device="cuda")
        err = ctypes.create_string_buffer(256)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        status = lib.pk_bin_static(ctypes.byref(cfg), transforms[0].data_ptr(), m2_ptr,
                                   sums.data_ptr(), stream.cuda_stream, err, len(err))
        assert status == pk.PK_OK, (call, status, err.value)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before, "the second call changed free device memory"
        s = sums.cpu().numpy()
        assert np.all(np.isfinite(s)), call
        S0 = s[:hb].reshape(nk, -1).sum(axis=1)
        # the oracle's mode loop on the same transforms
        scale = S0_oracle[ok]
        assert np.all(np.abs(S0 - S0_oracle)[ok] <= TOL_SAME_INPUT * scale), (call, "S0")
        if nmu > 0:
            s2 = s[:hb].reshape(nk, nmu)
            o2 = osum["psum2d"].reshape(nk, nmu) / L3
            sc2 = np.broadcast_to(S0_oracle[:, None], o2.shape)
            assert np.all(np.abs(s2 - o2)[ok] <= TOL_SAME_INPUT * sc2[ok]), (call, "(k, mu) sums")
        if with_poles:
            for row, key in ((0, "p2sum1d"), (1, "p4sum1d")):
                got = s[hb + row * nk: hb + (row + 1) * nk]
                assert np.all(np.abs(got - osum[key] / L3)[ok] <= TOL_SAME_INPUT * scale), (call, key)
        # the plan path's results, normalized the same way
        with np.errstate(invalid="ignore", divide="ignore"):
            p0 = norm * S0 / modes - shot
            assert np.all(np.abs(p0 - ref["power"])[ok] <= TOL * raw0[ok]), (call, "P0")
            if with_poles:
                p2 = 5.0 * norm * s[hb: hb + nk] / modes
                p4 = 9.0 * norm * s[hb + nk: hb + 2 * nk] / modes
                assert np.all(np.abs(p2 - ref["poles"][1])[ok] <= TOL * raw0[ok]), (call, "P2")
                assert np.all(np.abs(p4 - ref["poles"][2])[ok] <= TOL * raw0[ok]), (call, "P4")
            if nmu > 0:
                modes2d = ref["modes2d"].astype(np.float64)
                ok2 = modes2d > 0
                raw2d = np.broadcast_to(raw0[:, None], ok2.shape)
                pkmu = norm * s[:hb].reshape(nk, nmu) / modes2d - shot
                assert np.all(np.abs(pkmu - ref["power2d"])[ok2] <= TOL * raw2d[ok2]), (call, "P(k,mu)")


def test_static_bin_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk

    pk.build()
    lib = pk.load()
    cfg = pk.make_config(1000.0, 512, "cic", dk=0.0001, nmu=10)   # 16084 k bins: beyond 8192
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    status = lib.pk_bin_static(ctypes.byref(cfg), buf.data_ptr(), None, buf.data_ptr(), None, err, len(err))
    assert status == pk.PK_EINVAL and b"8192" in err.value
