"""Bit-exact check of the bin kernels' own mode-to-bin assignment (k_bin and the
own transform's fused z + bin pass).

The mode counts that pk_result reports come from the plan-time geometry pass;
the bin kernel itself places every mode in a k bin from an FP32 estimate plus
one exact integer step against the edges in m = |n|^2, and in a mu bin the
same way (Sec. 3.4.1 FFTPower binning; the exact rules are floor((kF sqrt(m) -
kmin) / dk) and the largest q with q^2 m <= nmu^2 l^2).  A mode placed one bin
off would only move power between bins, which a power tolerance can absorb.

Here the production bin kernel (through pk_bin_static, which launches the same
kernel as pk_compute) bins a transform whose every mode is exactly 1 + 0i,
uncompensated and not interlaced.  Each (k, mu) slot then holds its own
h-weighted mode count (h = 1 on the l = 0 and l = N/2 planes, else 2), summed
from small integers, which are exact in the kernel's FP32 per-CTA sums (every
per-CTA slot stays far below 2^24) and in the FP64 cross-CTA sums.  They must
equal the oracle's integer enumeration bit for bit, at the binnings of the
tiny, the 512^3 and the 2048^3 workloads, near the k-bin resolution limit
(kmax / dk just below 2^20) and with a mu-bin rule that needs 64-bit products.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    pk.build()
    pk.load()
    return pk


_UNIT = {}


def unit_transform(torch, N):
    """N x N x (N/2+1) complex64, every element 1 + 0i (one kept at a time)."""
    if N not in _UNIT:
        _UNIT.clear()
        torch.cuda.empty_cache()
        _UNIT[N] = torch.ones((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
    return _UNIT[N]


def kernel_counts(pk, torch, L, N, dk, nmu, kmin=0.0, kmax=None):
    cfg = pk.make_config(L, N, "cic", interlaced=False, compensated=False, dk=dk, nmu=nmu, kmin=kmin,
                         kmax=kmax, poles=(0,))
    nk = int(math.floor(((kmax if kmax else math.pi * N / L) - kmin) / dk))
    nh = nk * max(nmu, 1)
    t = unit_transform(torch, N)
    sums = torch.full((nh,), float("nan"), dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream()
    status = pk.load().pk_bin_static(ctypes.byref(cfg), t.data_ptr(), None, sums.data_ptr(),
                                     stream.cuda_stream, err, len(err))
    assert status == pk.PK_OK, err.value
    torch.cuda.synchronize()
    s = sums.cpu().numpy()
    assert np.all(s == np.floor(s)), "a slot sum is not an integer"
    return s.astype(np.int64), nk


@pytest.mark.parametrize("L,N,dk,nmu,kmin,kmax", [
    (1000.0, 64, 0.01, 0, 0.0, None),            # the tiny workload's binning (20 k bins)
    (1000.0, 64, 0.01, 5, 0.0, None),
    (777.0, 96, 0.0131, 7, 0.0051, 0.35),        # ragged edges, kmin > 0, kmax < k_N
    (1000.0, 512, 0.005, 10, 0.0, None),         # the 512^3 workload: 321 x 10 bins
    (2000.0, 2048, 0.005, 10, 0.0, None),        # the 2048^3 workload: 643 x 10 bins
    (2000.0, 2048, 0.005, 64, 3.0, None),        # nmu^2 m beyond 32 bits: 64-bit mu rule
])
def test_bin_kernel_places_every_mode_in_its_exact_bin(pk, oracle, L, N, dk, nmu, kmin, kmax):
    import torch
    got, nk = kernel_counts(pk, torch, L, N, dk, nmu, kmin, kmax)
    c1, c2 = oracle.mode_counts(N, L, dk, kmin=kmin, kmax=kmax, nmu=nmu)
    assert got.shape[0] == nk * max(nmu, 1)
    if nmu > 0:
        assert np.array_equal(got.reshape(nk, nmu), c2)
        assert np.array_equal(got.reshape(nk, nmu).sum(axis=1), c1)
    else:
        assert np.array_equal(got, c1)
    assert c1.sum() > 0


@pytest.mark.parametrize("N,L", [(64, 1000.0), (128, 333.0)])
def test_bin_kernel_near_the_k_resolution_limit(pk, oracle, N, L):
    """kmax / dk just below 2^20 (the plan's limit for the FP32 estimate plus
    one exact step): 8000 bins of width ~kmax / 2^20 ending at k_N, where most
    bins are empty and every occupied one must still be exact."""
    import torch
    kN = math.pi * N / L
    dk = kN / (2.0 ** 20 - 3.0)
    kmin = kN - 8000 * dk
    got, nk = kernel_counts(pk, torch, L, N, dk, 0, kmin, kN)
    c1, _ = oracle.mode_counts(N, L, dk, kmin=kmin, kmax=kN, nmu=0)
    assert nk == c1.shape[0] and 7990 <= nk <= 8000
    assert np.array_equal(got, c1)
    assert np.count_nonzero(c1) > 10


# The own transform's fused z + bin pass has no transform to inject, so its
# placement is checked through the plan path with a painted delta: one object
# of weight 1 exactly on node (0, 0, 0), CIC, not interlaced, uncompensated,
# no shot-noise subtraction.  Its mesh is 1 at cell 0 and 0 elsewhere, every
# step of the own transform is then exact in FP32 (sums of one 1 and zeros,
# twiddles W^0 = 1), the split gives 2 D = 2 exactly and every mode's power is
# L^3 * 1.  Each bin's sum is its own h-weighted mode count (exact in the FP32
# partials), so P(k) and P(k, mu) equal L^3 exactly iff the kernel placed
# every mode where the plan's exact geometry counted it.  L = 512 makes L^3 a
# power of two, so the FP64 normalization is exact too.
@pytest.mark.parametrize("N,dk_kf,nmu,kmin_kf,kmax_kn,own", [
    (128, 1.5, 7, 0.0, None, True),
    (128, 1.0, 0, 0.37, 0.9, True),
    (192, 1.3, 5, 0.0, None, True),        # radix-3 steps
    (256, 0.9, 10, 2.1, 0.8, True),
    (512, 1.226, 10, 0.0, None, True),
    (1024, 1.7, 3, 0.0, None, True),       # CTA-per-pair z pass (opt-in size)
    (2048, 2.3, 64, 0.0, None, True),      # CTA per pair, 64-bit mu rule
])
def test_own_transform_places_every_mode_in_its_exact_bin(pk, N, dk_kf, nmu, kmin_kf, kmax_kn, own):
    L = 512.0
    kF, kN = 2.0 * math.pi / L, math.pi * N / L
    cfg = pk.make_config(L, N, "cic", interlaced=False, compensated=False, dk=dk_kf * kF, nmu=nmu,
                         kmin=kmin_kf * kF, kmax=None if kmax_kn is None else kmax_kn * kN, subtract_shot=False)
    plan = pk.pk_plan(cfg)
    try:
        pk.pk_use_own_fft(plan, own)
        pk.pk_paint(plan, np.zeros((1, 3), np.float32))
        pk.pk_compute(plan)
        r = pk.pk_result(plan, 0)
    finally:
        pk.pk_destroy(plan)
    ok = r["modes"] > 0
    assert np.count_nonzero(ok) > 3
    assert np.all(r["power"][ok] == L ** 3), np.unique(r["power"][ok] / L ** 3)
    assert np.all(np.isnan(r["power"][~ok]))
    if nmu > 0:
        ok2 = r["modes2d"] > 0
        assert np.all(r["power2d"][ok2] == L ** 3), np.unique(r["power2d"][ok2] / L ** 3)
        assert np.array_equal(r["modes2d"].sum(axis=1), r["modes"])
