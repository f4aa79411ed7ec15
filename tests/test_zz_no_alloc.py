"""The allocation-free binning entry point, pk_bin_static, through the C ABI.

Some callers cannot call cudaMalloc: a framework that is capturing a stream
into a CUDA graph and owns all device memory, a program whose device memory is
handed out by a pool it does not control, or a host that forbids allocation
after start-up.  pk_bin_static lets them bin transforms they already hold,
using a fixed scratch array inside the library instead of allocating.

This test paints a catalog through the plan path (pk_plan / pk_paint),
copies out the two painted meshes, transforms them with torch's FFT, and calls
pk_bin_static twice in a row on those transforms.  Each call's raw sums,
normalized with the plan path's mode counts and weights, must reproduce the
plan path's P(k), P(k, mu), P_2 and P_4 within the FP32-form tolerance used
throughout the tests: 1e-4 of each bin's pre-subtraction monopole.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-4


def test_static_bin_matches_plan_path_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    import synth

    pk.build()
    lib = pk.load()
    L, N, nmu = 600.0, 64, 5
    dk = 2 * (2 * math.pi / L)
    pos = synth.lognormal_catalog(200000, L, N, synth.seed_for(5, 1), device="cuda")
    cfg = pk.make_config(L, N, "tsc", interlaced=True, dk=dk, nmu=nmu)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_paint(plan, pos)
        meshes = [pk.pk_mesh(plan, 0, m, N) for m in range(2)]
        pk.pk_compute(plan)
        ref = pk.pk_result(plan, 0)
    finally:
        pk.pk_destroy(plan)

    transforms = [torch.fft.rfftn(torch.from_numpy(m).cuda()).contiguous() for m in meshes]
    assert transforms[0].shape == (N, N, N // 2 + 1) and transforms[0].dtype == torch.complex64
    nk = ref["nk"]
    nh = nk * nmu + 2 * nk
    norm = L ** 3 / ref["wsum"] ** 2
    shot = ref["shot_noise"]
    modes = ref["modes"].astype(np.float64)
    modes2d = ref["modes2d"].astype(np.float64)
    ok, ok2 = modes > 0, modes2d > 0
    raw0 = ref["power"] + shot                       # pre-subtraction monopole
    raw2d = np.broadcast_to(raw0[:, None], ok2.shape)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    for call in range(2):
        sums = torch.full((nh,), float("nan"), dtype=torch.float64, device="cuda")
        err = ctypes.create_string_buffer(256)
        status = lib.pk_bin_static(ctypes.byref(cfg), transforms[0].data_ptr(), transforms[1].data_ptr(),
                                   sums.data_ptr(), stream.cuda_stream, err, len(err))
        assert status == pk.PK_OK, (call, status, err.value)
        torch.cuda.synchronize()
        s = sums.cpu().numpy()
        assert np.all(np.isfinite(s)), call
        s2d = s[: nk * nmu].reshape(nk, nmu)
        m2 = s[nk * nmu: nk * nmu + nk]
        m4 = s[nk * nmu + nk:]
        S0 = s2d.sum(axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            p0 = norm * S0 / modes - shot
            p2 = 5.0 * norm * (1.5 * m2 - 0.5 * S0) / modes
            p4 = 9.0 * norm * (35.0 * m4 - 30.0 * m2 + 3.0 * S0) / (8.0 * modes)
            pkmu = norm * s2d / modes2d - shot
        assert np.all(np.abs(p0 - ref["power"])[ok] <= TOL * raw0[ok]), (call, "P0")
        assert np.all(np.abs(p2 - ref["poles"][1])[ok] <= TOL * raw0[ok]), (call, "P2")
        assert np.all(np.abs(p4 - ref["poles"][2])[ok] <= TOL * raw0[ok]), (call, "P4")
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
