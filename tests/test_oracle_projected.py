"""Pins of the oracle's projected power spectrum (ProjectedFFTPower), CPU.

The projection-slice theorem ties the d-dimensional transform of the field
summed over the dropped axes to the plane (or line) of the 3D transform
through k = 0 along them; a uniform catalog's projected power is the aliased
shot noise L^d sum w^2 / (sum w)^2 S_d(k), with S_d the product of the
per-axis alias sums over the kept axes (even total alias index only, when
interlaced)."""
import math

import numpy as np
import pytest

from test_oracle_pins import alias_factor, fftfreq_int


@pytest.mark.parametrize("axes", [(0, 1), (0, 2), (1, 2), (2,), (0,)])
def test_projection_slice(oracle, axes):
    rng = np.random.default_rng(5)
    L, N = 50.0, 12
    pos = rng.uniform(0, L, (500, 3))
    mesh = oracle.paint(pos, None, L, N, "tsc", 0.0)
    full = np.fft.fftn(mesh)
    drop = tuple(a for a in range(3) if a not in axes)
    proj = np.fft.fftn(mesh.sum(axis=drop))
    sl = tuple(slice(None) if a in axes else 0 for a in range(3))
    np.testing.assert_allclose(proj, full[sl], rtol=1e-10, atol=1e-9)


def _expected(N, L, p, interlaced, d, dk, nk, oracle):
    A, B = alias_factor(N, p, interlaced)
    n = fftfreq_int(N)
    idx = np.meshgrid(*([np.arange(N)] * d), indexing="ij")
    SA = np.ones(idx[0].shape)
    SB = np.ones(idx[0].shape)
    for ix in idx:
        SA = SA * A[ix]
        SB = SB * B[ix]
    S = 0.5 * (SA + SB) if interlaced else SA
    m = sum(n[ix].astype(np.int64) ** 2 for ix in idx)
    kF = 2 * math.pi / L
    b = np.floor(kF * np.sqrt(m) / dk).astype(np.int64)
    ok = (m > 0) & (b < nk)
    H = np.bincount(b[ok], minlength=nk).astype(float)
    E = np.bincount(b[ok], weights=S[ok], minlength=nk) / H
    V = np.bincount(b[ok], weights=S[ok] ** 2, minlength=nk) / H ** 2
    return E, V, H


@pytest.mark.parametrize("axes,window,interlaced", [((0, 1), "cic", False), ((0, 2), "tsc", True),
                                                    ((2,), "pcs", False), ((1,), "tsc", True)])
def test_uniform_catalog_gives_projected_shot_noise(oracle, axes, window, interlaced):
    scipy_stats = pytest.importorskip("scipy.stats")
    L, N, n = 400.0, 32, 30000
    d = len(axes)
    dk = 2 * 2 * math.pi / L if d == 2 else 2 * math.pi / L
    nk = oracle.nbins(L, N, dk)
    E, V, H = _expected(N, L, oracle.WINDOW_ORDER[window], interlaced, d, dk, nk, oracle)
    zs, means, mvars = [], [], []
    for s in range(4):
        rng = np.random.default_rng(700 + s)
        pos = rng.uniform(0, L, (n, 3))
        w = rng.uniform(0.5, 1.5, n)
        r = oracle.projected_power(pos, w, L, N, window, interlaced, dk=dk, axes=axes, subtract_shot=False)
        assert np.array_equal(r["modes"], H.astype(np.int64))
        good = H > 0
        ratio = (r["power"] / r["shot_noise"])[good]
        # |delta|^2 of a mode is exponential and the +-k pairs are equal: the
        # bin mean has variance 2 sum S^2 / H^2
        zs.append((ratio - E[good]) / np.sqrt(2.0 * V[good]))
        means.append(ratio / E[good])
        mvars.append(2.0 * V[good] / E[good] ** 2)
    z = np.concatenate(zs)
    mean = np.concatenate(means)
    sigma = math.sqrt(np.sum(np.concatenate(mvars))) / mean.size
    assert abs(mean.mean() - 1.0) < 5 * sigma, (mean.mean(), sigma)
    if d == 2:                       # many modes per bin: Gaussian z-scores
        assert np.max(np.abs(z)) < 5.0 and scipy_stats.chi2.sf(np.sum(z * z), z.size) > 1e-4
