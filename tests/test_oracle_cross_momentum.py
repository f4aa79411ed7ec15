"""Pins of the oracle's cross power and painted-value (momentum) field, CPU.

Cross power P_ab = L^3 Re(delta_a conj(delta_b)): a catalog crossed with
itself is its auto power (before shot-noise subtraction), the cross is
symmetric, two independent uniform catalogs cross to zero within the
Gaussian scatter P_aa P_bb / (mode count), and a catalog crossed with a
subset of itself has the aliased shot noise L^3 / n_a S(k).

Painted values (F = [1 + delta'] V, Sec. 3.3.1): V = 1 is the plain field,
V = c scales the power by c^2, and independent zero-mean values on a uniform
catalog give the aliased shot noise L^3 sum (W V)^2 / (sum W)^2 S(k)."""
import math

import numpy as np
import pytest

from test_oracle_pins import expected_shot

L, N = 500.0, 32


def _cat(seed, n=40000):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, L, size=(n, 3)), rng.uniform(0.5, 1.5, n)


@pytest.mark.parametrize("window,interlaced", [("cic", False), ("tsc", True)])
def test_self_cross_is_the_unsubtracted_auto_power(oracle, window, interlaced):
    pos, w = _cat(1, 5000)
    dk = 2 * 2 * math.pi / L
    auto = oracle.fft_power(pos, w, L, N, window, interlaced, dk=dk, nmu=4, subtract_shot=False)
    cross = oracle.cross_power(pos, w, pos, w, L, N, window, interlaced, dk=dk, nmu=4)
    ok = auto["modes"] > 0
    assert np.array_equal(auto["power"][ok], cross["power"][ok])
    assert np.array_equal(auto["poles"][:, ok], cross["poles"][:, ok])
    assert cross["shot_noise"] == 0.0


def test_cross_is_symmetric(oracle):
    (pa, wa), (pb, wb) = _cat(2, 6000), _cat(3, 9000)
    dk = 2 * 2 * math.pi / L
    ab = oracle.cross_power(pa, wa, pb, wb, L, N, "pcs", True, dk=dk, nmu=3)
    ba = oracle.cross_power(pb, wb, pa, wa, L, N, "pcs", True, dk=dk, nmu=3)
    ok = ab["modes"] > 0
    assert np.array_equal(ab["power"][ok], ba["power"][ok])
    assert np.array_equal(ab["power2d"][ab["modes2d"] > 0], ba["power2d"][ab["modes2d"] > 0])


def test_independent_catalogs_cross_to_zero(oracle):
    scipy_stats = pytest.importorskip("scipy.stats")
    dk = 2 * 2 * math.pi / L
    chi2, dof = 0.0, 0
    for s in range(3):
        (pa, wa), (pb, wb) = _cat(10 + s), _cat(20 + s)
        ab = oracle.cross_power(pa, wa, pb, wb, L, N, "tsc", True, dk=dk)
        aa = oracle.fft_power(pa, wa, L, N, "tsc", True, dk=dk, subtract_shot=False)
        bb = oracle.fft_power(pb, wb, L, N, "tsc", True, dk=dk, subtract_shot=False)
        ok = ab["modes"] > 0
        z = ab["power"][ok] / np.sqrt(aa["power"][ok] * bb["power"][ok] / ab["modes"][ok])
        chi2 += float(np.sum(z * z))
        dof += int(ok.sum())
    assert scipy_stats.chi2.sf(chi2, dof) > 1e-4 and scipy_stats.chi2.cdf(chi2, dof) > 1e-4, (chi2, dof)


def test_subset_cross_has_the_aliased_shot_noise(oracle):
    dk = 2 * 2 * math.pi / L
    nk = oracle.nbins(L, N, dk)
    Eb, _ = expected_shot(N, L, 3, True, dk, nk)
    ratios = []
    for s in range(4):
        pa, _ = _cat(30 + s)
        pb = pa[: pa.shape[0] // 2]
        ab = oracle.cross_power(pa, None, pb, None, L, N, "tsc", True, dk=dk)
        ratios.append(ab["power"] / (L ** 3 / pa.shape[0]) / Eb)
    r = np.nanmean(np.array(ratios), axis=0)
    assert abs(np.nanmean(r) - 1.0) < 0.02, np.nanmean(r)


def test_unit_values_are_the_plain_field(oracle):
    pos, w = _cat(4, 5000)
    dk = 2 * 2 * math.pi / L
    a = oracle.fft_power(pos, w, L, N, "tsc", True, dk=dk, nmu=2)
    b = oracle.fft_power(pos, w, L, N, "tsc", True, dk=dk, nmu=2, values=np.ones(len(w)))
    ok = a["modes"] > 0
    assert np.array_equal(a["power"][ok], b["power"][ok]) and a["shot_noise"] == b["shot_noise"]


def test_constant_values_scale_the_power(oracle):
    pos, w = _cat(5, 5000)
    dk = 2 * 2 * math.pi / L
    a = oracle.fft_power(pos, w, L, N, "cic", False, dk=dk, subtract_shot=False)
    b = oracle.fft_power(pos, w, L, N, "cic", False, dk=dk, subtract_shot=False, values=np.full(len(w), -2.5))
    ok = a["modes"] > 0
    np.testing.assert_allclose(b["power"][ok], 6.25 * a["power"][ok], rtol=1e-12)
    assert abs(b["shot_noise"] - 6.25 * a["shot_noise"]) <= 1e-12 * b["shot_noise"]


def test_random_values_give_the_momentum_shot_noise(oracle):
    scipy_stats = pytest.importorskip("scipy.stats")
    dk = 2 * 2 * math.pi / L
    nk = oracle.nbins(L, N, dk)
    Eb, var = expected_shot(N, L, 3, False, dk, nk)
    chi2, dof, zmax = 0.0, 0, 0.0
    for s in range(3):
        pos, w = _cat(40 + s)
        v = np.random.default_rng(50 + s).normal(0.0, 300.0, len(w))
        r = oracle.fft_power(pos, w, L, N, "tsc", False, dk=dk, subtract_shot=False, values=v)
        z = (r["power"] / r["shot_noise"] - Eb) / np.sqrt(var)
        chi2 += float(np.sum(z * z))
        dof += nk
        zmax = max(zmax, float(np.max(np.abs(z))))
    assert zmax < 5.0 and scipy_stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof, zmax)
