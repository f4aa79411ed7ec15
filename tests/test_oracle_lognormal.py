"""Pins of the oracle's log-normal mock generator (CPU only).

Random numbers: Philox4x64-10 is checked against numpy's independent
implementation (numpy.random.Philox, whose raw draw from counter c is the
block of counter c + 1).  The rest is checked against statistics and closed
forms: Box-Muller output is standard normal; the Gaussian field has the
requested power spectrum and grid variance; the linear displacement of a
single plane wave is the closed-form sine; the log-normal weights average to
one; inverse-CDF placement follows the multinomial law, never picks a
zero-weight cell and keeps objects inside their cell (up to the z shift)."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("key,counter", [
    ((0, 0), (0, 0, 0, 0)), ((0x1234, 0x5678), (7, 0, 0, 0)), ((2**64 - 1, 3), (2**64 - 2, 5, 0, 9)),
    ((20171215, 1), (123456789, 0, 0, 0)),
])
def test_philox_matches_numpy(key, counter):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(counter, dtype=np.uint64))
    raw = [int(v) for v in bg.random_raw(8)]
    c = list(counter)

    def inc(c):
        c = c[:]
        for k in range(4):
            c[k] = (c[k] + 1) % 2 ** 64
            if c[k] != 0:
                break
        return c
    c1 = inc(c)
    c2 = inc(c1)
    assert oracle.philox4x64(c1, key) + oracle.philox4x64(c2, key) == raw


def test_white_noise_is_standard_normal():
    scipy_stats = pytest.importorskip("scipy.stats")
    w = oracle.white_noise(64, 42).reshape(-1)
    n = w.size
    assert abs(w.mean()) < 5 / math.sqrt(n)
    assert abs(w.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert scipy_stats.kstest(w, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(w[:-1], w[1:])[0, 1]) < 5 / math.sqrt(n)
    assert not np.array_equal(w, oracle.white_noise(64, 43).reshape(-1))
    assert np.array_equal(w, oracle.white_noise(64, 42).reshape(-1))


def test_linear_field_power_and_variance():
    ng, L, slope = 64, 500.0, -1.5
    G, gk, amp = oracle.linear_field(ng, L, slope, 11, variance=1.0)
    assert abs(G.var() - 1.0) < 0.05
    kf = 2 * math.pi / L
    f = np.fft.fftfreq(ng, 1.0 / ng)
    fz = np.fft.rfftfreq(ng, 1.0 / ng)
    m = (f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2)
    ok = (m > 0) & (fz[None, None, :] > 0) & (fz[None, None, :] < ng // 2)
    ratio = (np.abs(gk) ** 2 * L ** 3 / ng ** 6)[ok] / (amp * (kf * kf * m[ok]) ** (0.5 * slope))
    shell = np.floor(np.sqrt(m[ok]) / 4).astype(int)
    for s in np.unique(shell)[:6]:
        r = ratio[shell == s]
        assert abs(r.mean() - 1.0) < 5 / math.sqrt(r.size), (s, r.mean(), r.size)


def test_displacement_of_a_plane_wave():
    ng, L = 16, 100.0
    gk = np.zeros((ng, ng, ng // 2 + 1), complex)
    i0, j0, l0 = 3, ng - 2, 5
    gk[i0, j0, l0] = ng ** 3 / 2.0                    # G = cos(k . x)
    kf = 2 * math.pi / L
    k = kf * np.array([3.0, -2.0, 5.0])
    x = np.arange(ng) * L / ng
    phase = k[0] * x[:, None, None] + k[1] * x[None, :, None] + k[2] * x[None, None, :]
    assert np.allclose(np.fft.irfftn(gk, s=(ng,) * 3), np.cos(phase), atol=1e-12)
    psi = oracle.displacement_z(gk, L)
    assert np.allclose(psi, -(k[2] / (k @ k)) * np.sin(phase), atol=1e-12)


def test_lognormal_weights_average_to_one():
    G, _, _ = oracle.linear_field(64, 1000.0, -1.5, 5)
    q = oracle.lognormal_weights(G)
    assert q.dtype == np.int64 and q.min() >= 0
    w = q / 2.0 ** 30
    sig2 = G.var()
    assert np.max(np.abs(w - np.exp(G - 0.5 * sig2))) <= 2.0 ** -31 * (1 + 1e-9)
    assert abs(w.mean() - 1.0) < 0.02


def test_placement_is_multinomial_and_inside_cells():
    scipy_stats = pytest.importorskip("scipy.stats")
    ng, L = 2, 10.0
    q = np.array([0, 3, 0, 5, 2, 0, 1, 9], np.int64).reshape(2, 2, 2) * 1000
    n = 200000
    pos = oracle.place(q, L, None, 0.0, 99, n)
    assert pos.shape == (n, 3)
    cell = np.floor(pos / (L / ng)).astype(int)
    flat = (cell[:, 0] * ng + cell[:, 1]) * ng + cell[:, 2]
    counts = np.bincount(flat, minlength=8)
    assert np.all(counts[q.reshape(-1) == 0] == 0)
    p = q.reshape(-1) / q.sum()
    nz = p > 0
    chi2 = np.sum((counts[nz] - n * p[nz]) ** 2 / (n * p[nz]))
    assert scipy_stats.chi2.sf(chi2, nz.sum() - 1) > 1e-4
    # offsets inside the cell are uniform
    frac = pos / (L / ng) - cell
    assert np.all((frac > 0) & (frac < 1))
    assert abs(frac.mean() - 0.5) < 5 * math.sqrt(1 / 12 / (3 * n))


def test_placement_applies_the_z_shift_and_wraps():
    ng, L, f = 8, 80.0, 0.75
    rng = np.random.default_rng(3)
    q = rng.integers(1, 100, (ng, ng, ng)).astype(np.int64)
    psi = rng.normal(0, 30.0, (ng, ng, ng))
    p0 = oracle.place(q, L, None, 0.0, 17, 5000)
    p1 = oracle.place(q, L, psi, f, 17, 5000)
    assert np.array_equal(p0[:, :2], p1[:, :2])
    cell = np.floor(p0 / (L / ng)).astype(int)
    shift = f * psi[cell[:, 0], cell[:, 1], cell[:, 2]]
    assert np.allclose(np.mod(p0[:, 2] + shift, L), p1[:, 2], atol=1e-9)
    assert p1.min() >= 0 and p1.max() < L


def test_catalog_is_seeded_and_sized():
    a = oracle.lognormal_catalog(3000, 200.0, 16, 8)
    b = oracle.lognormal_catalog(3000, 200.0, 16, 8)
    c = oracle.lognormal_catalog(3000, 200.0, 16, 9)
    assert a.shape == (3000, 3) and np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0 and a.max() < 200.0
