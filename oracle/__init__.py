"""FP64 CPU oracle for the FFT power-spectrum path (nbodykit, arXiv:1712.05834).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may import
this package.  It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``pk_oracle.c`` (plain FP64 loops, one function per
step of the method, including its own mixed-radix FFT between painting and
binning: Sec. 3.3.1 relates the real and complex fields by an r2c FFT).  This
module only marshals arrays and finalizes the bin sums:

    P(k, mu) = sum h P / sum h - P_shot                      (Sec. 3.4.1)
    P_l(k)   = (2l + 1) sum h P L_l(mu) / sum h - [l = 0] P_shot
    P_shot   = L^3 sum(w^2) / sum(w)^2        (= 1 / nbar for unit weights)

Every pin that ties this oracle to the paper and to mathematics is in
``tests/test_oracle_*.py`` (run with ``-m "not gpu"``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pk_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "lognormal_oracle.c")]
_LIB = os.path.join(_HERE, "_pk_oracle.so")
_lib = None

WINDOW_ORDER = {"cic": 2, "tsc": 3, "pcs": 4}


def build(force: bool = False) -> str:
    """Compile pk_oracle.c into oracle/_pk_oracle.so with gcc (FP64, no FMA
    contraction so the k-bin expression rounds exactly as written)."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-fopenmp"] + _SRCS + ["-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.oracle_window_weight.argtypes = [i, d]
        lib.oracle_window_weight.restype = d
        lib.oracle_paint.argtypes = [p, p, i64, d, i, i, d, p]
        lib.oracle_paint.restype = i
        lib.oracle_kbin.argtypes = [i64, d, d, d]
        lib.oracle_kbin.restype = i64
        lib.oracle_mubin.argtypes = [i64, i64, i64]
        lib.oracle_mubin.restype = i64
        lib.oracle_bin.argtypes = [p, p, i, d, i, i, d, d, d, i, i] + [p] * 9
        lib.oracle_bin.restype = i
        lib.oracle_bin_pair.argtypes = [p, p, p, p, i, d, i, i, d, d, d, d, i, i] + [p] * 9
        lib.oracle_bin_pair.restype = i
        lib.oracle_paint_block.argtypes = [p, p, i64, d, i, i, d, p, i, p]
        lib.oracle_paint_block.restype = i
        lib.oracle_mode_counts.argtypes = [i, d, d, d, i, i, p, p]
        lib.oracle_mode_counts.restype = i
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = i
        lib.oracle_set_threads.argtypes = [i]
        lib.oracle_set_threads.restype = None
        lib.oracle_r2c.argtypes = [p, i, p]
        lib.oracle_r2c.restype = i
        lib.oracle_twiddles.argtypes = [i, p]
        lib.oracle_twiddles.restype = None
        lib.oracle_dft_line.argtypes = [p, i, p, p]
        lib.oracle_dft_line.restype = None
        lib.oracle_philox4x64.argtypes = [p, p, p]
        lib.oracle_philox4x64.restype = None
        lib.oracle_white_noise.argtypes = [i, ctypes.c_uint64, p]
        lib.oracle_white_noise.restype = i
        lib.oracle_place.argtypes = [p, i, d, p, d, ctypes.c_uint64, i64, p]
        lib.oracle_place.restype = i
        _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _order(window) -> int:
    return WINDOW_ORDER[window] if isinstance(window, str) else int(window)


def threads() -> int:
    """Host threads the oracle's parallel loops use."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    """Use n host threads in the oracle's parallel loops from now on."""
    _load().oracle_set_threads(int(n))


def window_weight(window, d: float) -> float:
    """B-spline window of order p at distance d cells (Sec. 3.3.2)."""
    return _load().oracle_window_weight(_order(window), float(d))


def kbin(m: int, box_size: float, kmin: float, dk: float) -> int:
    return _load().oracle_kbin(int(m), float(box_size), float(kmin), float(dk))


def mubin(m: int, l: int, nmu: int) -> int:
    return _load().oracle_mubin(int(m), int(l), int(nmu))


def paint(pos, weights, box_size: float, nmesh: int, window, shift: float = 0.0):
    """Painted field F on an (N, N, N) FP64 mesh (Sec. 3.3.1), nodes at c*H."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    mesh = np.zeros((nmesh, nmesh, nmesh), dtype=np.float64)
    rc = _load().oracle_paint(_ptr(pos), _ptr(w), pos.shape[0], float(box_size),
                              int(nmesh), _order(window), float(shift), _ptr(mesh))
    if rc != 0:
        raise ValueError("oracle_paint: bad arguments")
    return mesh


def paint_block(pos, weights, box_size, nmesh, window, c0, block, shift=0.0):
    """Painted field on the block of cells c0 + [0, block)^3 (periodic) only:
    oracle_paint restricted to a block, for meshes too large to hold."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    c0 = np.ascontiguousarray(np.asarray(c0, dtype=np.int64).reshape(3))
    out = np.zeros((block, block, block), dtype=np.float64)
    rc = _load().oracle_paint_block(_ptr(pos), _ptr(w), pos.shape[0], float(box_size), int(nmesh),
                                    _order(window), float(shift), _ptr(c0), int(block), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_paint_block: bad arguments")
    return out


def mode_counts(nmesh, box_size, dk, kmin=0.0, kmax=None, nmu=0):
    """Weighted mode counts of the k bins and (k, mu) bins (Sec. 3.4.1)."""
    nk = nbins(box_size, nmesh, dk, kmin, kmax)
    nm = max(int(nmu), 0)
    c1 = np.zeros(nk, np.int64)
    c2 = np.zeros(nk * max(nm, 1), np.int64)
    rc = _load().oracle_mode_counts(int(nmesh), float(box_size), float(kmin), float(dk), nk, nm,
                                    _ptr(c1), _ptr(c2))
    if rc != 0:
        raise ValueError("oracle_mode_counts: bad arguments")
    return c1, (c2.reshape(nk, nm) if nm > 0 else None)


def r2c(mesh):
    """Forward r2c transform, F~(n) = sum_c F[c] exp(-2 pi i c.n / N), last axis
    halved: the oracle's own mixed-radix FFT (pk_oracle.c, oracle_r2c)."""
    mesh = np.ascontiguousarray(mesh, dtype=np.float64)
    N = mesh.shape[0]
    assert mesh.shape == (N, N, N)
    out = np.empty((N, N, N // 2 + 1), dtype=np.complex128)
    rc = _load().oracle_r2c(_ptr(mesh), int(N), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_r2c failed (%d)" % rc)
    return out


def dft(x):
    """One-dimensional transform X[k] = sum_j x[j] exp(-2 pi i j k / n) of a
    complex vector by the same mixed-radix routine (for its pins)."""
    x = np.array(x, dtype=np.complex128).reshape(-1)
    n = x.shape[0]
    tw = np.empty(2 * n)
    work = np.empty(4 * n)
    _load().oracle_twiddles(int(n), _ptr(tw))
    _load().oracle_dft_line(_ptr(x), int(n), _ptr(tw), _ptr(work))
    return x


def nbins(box_size: float, nmesh: int, dk: float, kmin: float = 0.0, kmax=None) -> int:
    """nk = floor((kmax - kmin) / dk); kmax defaults to k_N = (pi N) / L."""
    if kmax is None or kmax <= 0:
        kmax = (math.pi * nmesh) / box_size
    return int(math.floor((kmax - kmin) / dk))


def bin_modes(F1, F2, box_size, window, compensated, wsum, dk, kmin=0.0, kmax=None, nmu=0):
    """Raw FFTPower bin sums from stored half-grid transforms (Sec. 3.4.1)."""
    F1 = np.ascontiguousarray(F1, dtype=np.complex128)
    N = F1.shape[0]
    assert F1.shape == (N, N, N // 2 + 1)
    if F2 is not None:
        F2 = np.ascontiguousarray(F2, dtype=np.complex128)
        assert F2.shape == F1.shape
    nk = nbins(box_size, N, dk, kmin, kmax)
    nm = max(int(nmu), 0)
    out = {
        "modes1d": np.zeros(nk, np.int64), "ksum1d": np.zeros(nk), "psum1d": np.zeros(nk),
        "p2sum1d": np.zeros(nk), "p4sum1d": np.zeros(nk),
        "modes2d": np.zeros(nk * max(nm, 1), np.int64), "ksum2d": np.zeros(nk * max(nm, 1)),
        "musum2d": np.zeros(nk * max(nm, 1)), "psum2d": np.zeros(nk * max(nm, 1)),
    }
    rc = _load().oracle_bin(
        _ptr(F1), _ptr(F2), int(N), float(box_size), _order(window), int(bool(compensated)),
        float(wsum), float(kmin), float(dk), int(nk), int(nm),
        _ptr(out["modes1d"]), _ptr(out["ksum1d"]), _ptr(out["psum1d"]), _ptr(out["p2sum1d"]),
        _ptr(out["p4sum1d"]), _ptr(out["modes2d"]), _ptr(out["ksum2d"]), _ptr(out["musum2d"]),
        _ptr(out["psum2d"]))
    if rc != 0:
        raise ValueError("oracle_bin: bad arguments")
    out["nk"], out["nmu"] = nk, nm
    return out


def bin_cross(Fa1, Fa2, Fb1, Fb2, box_size, window, compensated, wsum_a, wsum_b, dk, kmin=0.0, kmax=None,
              nmu=0):
    """Raw bin sums of the cross power Re(delta_a conj(delta_b)) of two catalogs
    painted on equal meshes (the auto-power loop with a second field)."""
    Fa1 = np.ascontiguousarray(Fa1, dtype=np.complex128)
    Fb1 = np.ascontiguousarray(Fb1, dtype=np.complex128)
    N = Fa1.shape[0]
    assert Fa1.shape == Fb1.shape == (N, N, N // 2 + 1)
    Fa2 = None if Fa2 is None else np.ascontiguousarray(Fa2, dtype=np.complex128)
    Fb2 = None if Fb2 is None else np.ascontiguousarray(Fb2, dtype=np.complex128)
    nk = nbins(box_size, N, dk, kmin, kmax)
    nm = max(int(nmu), 0)
    out = {
        "modes1d": np.zeros(nk, np.int64), "ksum1d": np.zeros(nk), "psum1d": np.zeros(nk),
        "p2sum1d": np.zeros(nk), "p4sum1d": np.zeros(nk),
        "modes2d": np.zeros(nk * max(nm, 1), np.int64), "ksum2d": np.zeros(nk * max(nm, 1)),
        "musum2d": np.zeros(nk * max(nm, 1)), "psum2d": np.zeros(nk * max(nm, 1)),
    }
    rc = _load().oracle_bin_pair(
        _ptr(Fa1), _ptr(Fa2), _ptr(Fb1), _ptr(Fb2), int(N), float(box_size), _order(window),
        int(bool(compensated)), float(wsum_a), float(wsum_b), float(kmin), float(dk), int(nk), int(nm),
        _ptr(out["modes1d"]), _ptr(out["ksum1d"]), _ptr(out["psum1d"]), _ptr(out["p2sum1d"]),
        _ptr(out["p4sum1d"]), _ptr(out["modes2d"]), _ptr(out["ksum2d"]), _ptr(out["musum2d"]),
        _ptr(out["psum2d"]))
    if rc != 0:
        raise ValueError("oracle_bin_pair: bad arguments")
    out["nk"], out["nmu"] = nk, nm
    return out


def cross_power(pos_a, w_a, pos_b, w_b, box_size, nmesh, window="cic", interlaced=False, compensated=True,
                dk=None, kmin=0.0, kmax=None, nmu=0, values_a=None, values_b=None):
    """Cross power spectrum of two catalogs on the CPU in FP64 (no shot noise:
    the catalogs are taken as independent samples).  values_a / values_b
    paint W V with normalization by sum W, as in fft_power."""
    sides = []
    for pos, w, v in ((pos_a, w_a, values_a), (pos_b, w_b, values_b)):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        wv = np.ones(pos.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
        wsum = float(np.sum(wv))
        amp = w if v is None else wv * np.asarray(v, dtype=np.float64)
        F1 = r2c(paint(pos, amp, box_size, nmesh, window, 0.0))
        F2 = r2c(paint(pos, amp, box_size, nmesh, window, 0.5)) if interlaced else None
        sides.append((F1, F2, wsum))
    (Fa1, Fa2, wa), (Fb1, Fb2, wb) = sides
    sums = bin_cross(Fa1, Fa2, Fb1, Fb2, box_size, window, compensated, wa, wb, dk, kmin, kmax, nmu)
    res = finalize(sums, 0.0, False)
    res["nk"], res["nmu"] = sums["nk"], sums["nmu"]
    return res


def finalize(sums, shot_noise: float, subtract_shot: bool = True):
    """Bin averages, multipoles and shot-noise subtraction (Sec. 3.4.1)."""
    nk, nm = sums["nk"], sums["nmu"]
    with np.errstate(invalid="ignore", divide="ignore"):
        m1 = sums["modes1d"].astype(np.float64)
        ps = shot_noise if subtract_shot else 0.0
        res = {
            "k": sums["ksum1d"] / m1,
            "modes": sums["modes1d"].copy(),
            "power_raw": sums["psum1d"] / m1,
            "power": sums["psum1d"] / m1 - ps,
            "poles": np.stack([sums["psum1d"] / m1 - ps,
                               5.0 * sums["p2sum1d"] / m1,
                               9.0 * sums["p4sum1d"] / m1]),
            "shot_noise": shot_noise,
        }
        if nm > 0:
            m2 = sums["modes2d"].astype(np.float64)
            res["modes2d"] = sums["modes2d"].reshape(nk, nm).copy()
            res["k2d"] = (sums["ksum2d"] / m2).reshape(nk, nm)
            res["mu2d"] = (sums["musum2d"] / m2).reshape(nk, nm)
            res["power2d_raw"] = (sums["psum2d"] / m2).reshape(nk, nm)
            res["power2d"] = res["power2d_raw"] - ps
    return res


def fft_power(pos, weights, box_size, nmesh, window="cic", interlaced=False,
              compensated=True, dk=None, kmin=0.0, kmax=None, nmu=0,
              subtract_shot=True, values=None):
    """The whole path on the CPU in FP64: paint (one or two meshes), r2c FFT,
    compensate + interlace, bin, multipoles, shot noise.  ``values`` (V per
    object, Sec. 3.3.1: F = [1 + delta'] V) paints W V but keeps the
    normalization by sum W; the shot noise is L^3 sum (W V)^2 / (sum W)^2."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    w = np.ones(pos.shape[0]) if weights is None else np.asarray(weights, dtype=np.float64)
    a = w if values is None else w * np.asarray(values, dtype=np.float64)
    wsum = float(np.sum(w))
    w2sum = float(np.sum(a * a))
    amp = None if (weights is None and values is None) else a
    F1 = r2c(paint(pos, amp, box_size, nmesh, window, 0.0))
    F2 = r2c(paint(pos, amp, box_size, nmesh, window, 0.5)) if interlaced else None
    sums = bin_modes(F1, F2, box_size, window, compensated, wsum, dk, kmin, kmax, nmu)
    shot = box_size ** 3 * w2sum / wsum ** 2
    res = finalize(sums, shot, subtract_shot)
    res["wsum"], res["w2sum"] = wsum, w2sum
    res["nk"], res["nmu"] = sums["nk"], sums["nmu"]
    return res


# ------------------------------------------------------------------------
# Log-normal mock generator (LogNormalCatalog of the paper's tests and
# benchmarks, Sec. 3.2), FP64.  Random numbers: Philox4x64-10 (see
# lognormal_oracle.c for the stream layout).
# ------------------------------------------------------------------------

def philox4x64(ctr, key):
    """One Philox4x64-10 block: four 64-bit words."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, np.uint64)
    _load().oracle_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return [int(v) for v in out]


def white_noise(ng: int, seed: int):
    """ng^3 unit Gaussians (Box-Muller on Philox words), C order, z fastest."""
    out = np.zeros((ng, ng, ng), np.float64)
    if _load().oracle_white_noise(int(ng), int(seed), _ptr(out)) != 0:
        raise ValueError("oracle_white_noise: bad arguments")
    return out


def _k2_grid(ng: int, box_size: float):
    kf = 2.0 * math.pi / box_size
    f = np.fft.fftfreq(ng, 1.0 / ng) * kf
    fz = np.fft.rfftfreq(ng, 1.0 / ng) * kf
    return f[:, None, None], f[None, :, None], fz[None, None, :]


def lognormal_amplitude(ng: int, box_size: float, slope: float, variance: float = 1.0) -> float:
    """A with (1 / L^3) sum_{k != 0} A k^slope = variance over the full ng^3 grid."""
    kf = 2.0 * math.pi / box_size
    f = np.fft.fftfreq(ng, 1.0 / ng)
    total = 0.0
    for i in f:
        m = i * i + f[:, None] ** 2 + f[None, :] ** 2
        m = m[m > 0]
        total += float(np.sum((kf * kf * m) ** (0.5 * slope)))
    return variance * box_size ** 3 / total


def linear_field(ng: int, box_size: float, slope: float, seed: int, amp=None, variance: float = 1.0):
    """Gaussian field G with P(k) = A k^slope on the grid: G~ = FFT(W) sqrt(P ng^3 / L^3),
    G = IFFT(G~) (numpy's normalized inverse).  Returns (G, G~, A)."""
    if amp is None or amp <= 0:
        amp = lognormal_amplitude(ng, box_size, slope, variance)
    wk = np.fft.rfftn(white_noise(ng, seed))
    kx, ky, kz = _k2_grid(ng, box_size)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    factor = np.sqrt(amp * k2 ** (0.5 * slope) * ng ** 3 / box_size ** 3)
    factor[0, 0, 0] = 0.0
    gk = wk * factor
    return np.fft.irfftn(gk, s=(ng, ng, ng), axes=(0, 1, 2)), gk, amp


def displacement_z(gk, box_size: float):
    """psi_z = IFFT(i k_z / k^2 G~) (linear displacement, z component); the
    z-Nyquist plane of psi~ is set to zero (its sign is ambiguous on the half grid)."""
    ng = gk.shape[0]
    kx, ky, kz = _k2_grid(ng, box_size)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    pk_ = gk * (1j * kz / k2)
    pk_[0, 0, 0] = 0.0
    pk_[:, :, ng // 2] = 0.0
    return np.fft.irfftn(pk_, s=(ng, ng, ng), axes=(0, 1, 2))


def lognormal_weights(G):
    """Integer cell weights round(2^30 exp(G - sigma^2 / 2)), sigma^2 the grid variance of G."""
    sig2 = float(np.mean(G * G) - np.mean(G) ** 2)
    return np.rint(np.exp(G - 0.5 * sig2) * 2.0 ** 30).astype(np.int64)


def place(q, box_size: float, psi_z, f_rsd: float, seed: int, n: int):
    """Exactly n objects from integer cell weights q (ng^3): cell by inverse
    CDF, uniform in the cell, z + f psi_z(cell), wrapped into [0, L)."""
    ng = q.shape[0]
    excl = np.zeros(q.size + 1, np.int64)
    np.cumsum(q.reshape(-1), out=excl[1:])
    pz = None if psi_z is None else np.ascontiguousarray(psi_z, dtype=np.float64)
    pos = np.zeros((int(n), 3), np.float64)
    rc = _load().oracle_place(_ptr(excl), int(ng), float(box_size), _ptr(pz), float(f_rsd), int(seed),
                              int(n), _ptr(pos))
    if rc != 0:
        raise ValueError("oracle_place: bad arguments (%d)" % rc)
    return pos


def lognormal_catalog(n: int, box_size: float, ng: int, seed: int, slope: float = -1.5, amp=None,
                      variance: float = 1.0, f_rsd: float = 0.75):
    """The whole generator in FP64: linear field, log-normal transform,
    integer cell weights, n objects, linear redshift-space displacement."""
    G, gk, _ = linear_field(ng, box_size, slope, seed, amp, variance)
    psi = displacement_z(gk, box_size) if f_rsd else None
    return place(lognormal_weights(G), box_size, psi, f_rsd, seed, n)


def projected_power(pos, weights, box_size, nmesh, window="cic", interlaced=False, compensated=True,
                    dk=None, kmin=0.0, kmax=None, axes=(0, 1), subtract_shot=True):
    """Power spectrum of the painted field projected onto `axes` (summed over
    the other axes; the ProjectedFFTPower of Sec. 3.4.1), FP64: the projected
    field's d-dimensional FFT (d = len(axes)), the interlacing combine and
    the compensation over the kept axes, delta = F~ / sum w, P = L^d |delta|^2
    per mode (every mode of the full d-dimensional grid counted once), binned
    in |k| with the FFTPower k bins; shot noise L^d sum w^2 / (sum w)^2."""
    axes = tuple(sorted(int(a) for a in axes))
    d = len(axes)
    drop = tuple(a for a in range(3) if a not in axes)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    w = np.ones(pos.shape[0]) if weights is None else np.asarray(weights, dtype=np.float64)
    wsum, w2sum = float(np.sum(w)), float(np.sum(w * w))
    T = np.fft.fftn(paint(pos, weights, box_size, nmesh, window, 0.0).sum(axis=drop))
    n1 = np.fft.fftfreq(nmesh, 1.0 / nmesh)
    grids = np.meshgrid(*([n1] * d), indexing="ij")
    if interlaced:
        T2 = np.fft.fftn(paint(pos, weights, box_size, nmesh, window, 0.5).sum(axis=drop))
        T = 0.5 * (T + T2 * np.exp(1j * np.pi * sum(grids) / nmesh))
    if compensated:
        W = np.ones_like(grids[0])
        for g in grids:
            W = W * np.sinc(g / nmesh) ** _order(window)
        T = T / W
    delta = T / wsum
    P = box_size ** d * np.abs(delta) ** 2
    m = sum(g.astype(np.int64) ** 2 for g in grids).astype(np.int64)
    nk = nbins(box_size, nmesh, dk, kmin, kmax)
    b = np.full(m.shape, -1, np.int64)
    for mv in np.unique(m):
        if mv > 0:
            b[m == mv] = kbin(int(mv), box_size, kmin, dk)
    ok = (m > 0) & (b >= 0) & (b < nk)
    kF = 2.0 * math.pi / box_size
    modes = np.bincount(b[ok], minlength=nk).astype(np.int64)
    ksum = np.bincount(b[ok], weights=kF * np.sqrt(m[ok].astype(np.float64)), minlength=nk)
    psum = np.bincount(b[ok], weights=P[ok], minlength=nk)
    shot = box_size ** d * w2sum / wsum ** 2
    with np.errstate(invalid="ignore", divide="ignore"):
        res = {"k": ksum / modes, "modes": modes, "power_raw": psum / modes,
               "power": psum / modes - (shot if subtract_shot else 0.0), "shot_noise": shot, "nk": nk,
               "wsum": wsum, "w2sum": w2sum}
    return res
