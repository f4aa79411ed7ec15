"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties one step of the oracle to a fact fixed by the paper or by
mathematics (arXiv:1712.05834 Sec. 3.3.1 painting, Sec. 3.3.2 windows,
interlacing and Eq. window-deconvolution, Sec. 3.4.1 FFTPower):

* the r2c transform equals a brute-force DFT (sign, normalization, halved axis);
* painting conserves mass and matches a per-cell brute-force evaluation;
* the node / half-node window weights equal the B-spline values (golden file);
* averaging over sub-cell offsets gives exactly sinc^p (the compensated window);
* a uniform random catalog gives the analytic aliased shot noise, which pins
  the normalization, the shot noise, the compensation and the interlacing sign
  (a planted wrong-direction interlace is rejected);
* Gaussian fields of known P(k), with and without a Kaiser factor, are
  recovered in P(k) and in P_0, P_2, P_4 within cosmic variance;
* a unit-amplitude field gives exact rational Legendre averages;
* half-grid weighted mode counts equal a full-grid integer enumeration;
* the mu-bin rule on the worked edge cases;
* the whole pipeline equals a fully brute-force full-grid computation on 8^3.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fftfreq_int(N):
    return np.where(np.arange(N) < N // 2, np.arange(N), np.arange(N) - N)


# ---------------------------------------------------------------- FFT step --

def brute_dft_r2c(mesh):
    """O(N^6) DFT, F(n) = sum_c F[c] exp(-2 pi i c.n / N), last axis halved."""
    N = mesh.shape[0]
    c = np.arange(N)
    E = np.exp(-2j * np.pi * np.outer(c, c) / N)          # E[n, c]
    out = np.zeros((N, N, N // 2 + 1), complex)
    for n0 in range(N):
        for n1 in range(N):
            for n2 in range(N // 2 + 1):
                ph = E[n0][:, None, None] * E[n1][None, :, None] * E[n2][None, None, :]
                out[n0, n1, n2] = np.sum(mesh * ph)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 11, 12, 22, 33, 48, 64, 66])
def test_dft_line_equals_direct_sum(oracle, n):
    """The oracle's mixed-radix 1D transform (radix 2, 3 and a direct sum for
    any other prime factor, as N = 40, 48, 528 need) equals the O(n^2)
    definition X[k] = sum_j x[j] exp(-2 pi i j k / n) written out."""
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    ref = np.array([np.sum(x * np.exp(-2j * np.pi * j * k / n)) for k in range(n)])
    got = oracle.dft(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("N", [6, 8, 12, 16])
def test_r2c_equals_bruteforce_dft_and_parseval(oracle, N):
    rng = np.random.default_rng(7 + N)
    mesh = rng.standard_normal((N, N, N))
    F = oracle.r2c(mesh)
    ref = brute_dft_r2c(mesh)
    assert F.shape == (N, N, N // 2 + 1)
    assert np.max(np.abs(F - ref)) <= 1e-12 * np.max(np.abs(ref))
    # Parseval over the full grid: the half grid counts l = 0, N/2 once, others twice
    h = np.full(N // 2 + 1, 2.0)
    h[0] = 1.0
    h[N // 2] = 1.0
    full = np.sum(h[None, None, :] * np.abs(F) ** 2)
    assert abs(np.sum(mesh ** 2) - full / N ** 3) <= 1e-12 * np.sum(mesh ** 2)


# -------------------------------------------------------------- paint step --

def load_golden_weights():
    rows = {}
    with open(os.path.join(GOLDEN, "window_node_weights.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[(parts[0], parts[1])] = [Fraction(x) for x in parts[2:]]
    return rows


@pytest.mark.parametrize("window", ["cic", "tsc", "pcs"])
def test_node_and_half_node_weights(oracle, window):
    g = load_golden_weights()
    N, L = 16, 16.0                        # H = 1: positions are in cells
    for kind, x, first in (("node", 5.0, 3), ("half", 5.5, 4)):
        mesh = oracle.paint(np.array([[x, 8.0, 8.0]]), None, L, N, window)
        line = mesh[:, 8, 8] / mesh[:, 8, 8].sum()
        # the y and z axes sit on a node; their node weight multiplies the x line
        want = [float(v) for v in g[(window, kind)]]
        got = line[first:first + len(want)]
        assert np.allclose(got, want, rtol=0, atol=1e-15), (window, kind, got, want)
        assert abs(np.sum(line) - 1.0) < 1e-15
        assert np.sum(np.abs(np.delete(line, range(first, first + len(want))))) == 0.0
    # the node weight on the y, z axes themselves
    node = [float(v) for v in g[(window, "node")]]
    mesh = oracle.paint(np.array([[5.0, 8.0, 8.0]]), None, L, N, window)
    assert abs(mesh[5, 8, 8] - node[2] ** 3) < 1e-15


def brute_paint(pos, w, L, N, p, shift, oracle):
    """Per-cell evaluation with minimum-image distances (no loop bounds to get wrong)."""
    mesh = np.zeros((N, N, N))
    s = (pos - L * np.floor(pos / L)) * N / L + shift
    cells = np.arange(N)
    for q in range(pos.shape[0]):
        ws = []
        for a in range(3):
            d = s[q, a] - cells
            d = d - N * np.round(d / N)              # minimum image in index space
            ws.append(np.array([oracle.window_weight(p, x) for x in d]))
        mesh += (1.0 if w is None else w[q]) * ws[0][:, None, None] * ws[1][None, :, None] * ws[2][None, None, :]
    return mesh


@pytest.mark.parametrize("window,shift", [("cic", 0.0), ("tsc", 0.5), ("pcs", 0.0), ("pcs", 0.5)])
def test_paint_equals_per_cell_bruteforce(oracle, window, shift):
    rng = np.random.default_rng(11)
    N, L = 8, 20.0
    pos = rng.uniform(-L, 2 * L, size=(25, 3))     # outside the box too: wrapped
    pos[0] = [0.0, L - 1e-12, 19.999]              # edges of the box
    w = rng.uniform(0.5, 2.0, 25)
    got = oracle.paint(pos, w, L, N, window, shift)
    ref = brute_paint(pos, w, L, N, oracle.WINDOW_ORDER[window], shift, oracle)
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("window", ["cic", "tsc", "pcs"])
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_paint_conserves_mass(oracle, window, shift):
    rng = np.random.default_rng(3)
    L, N = 100.0, 32
    pos = rng.uniform(0, L, size=(5000, 3))
    w = rng.exponential(1.0, 5000)
    mesh = oracle.paint(pos, w, L, N, window, shift)
    assert abs(mesh.sum() - w.sum()) <= 1e-13 * w.sum()


@pytest.mark.parametrize("window,p", [("cic", 2), ("tsc", 3), ("pcs", 4)])
def test_window_transform_averages_to_sinc_p(oracle, window, p):
    """E_x0[F~(n) exp(+i k x0)] = sinc^p(pi n / N): the function that
    Eq. window-deconvolution divides out.  Gauss-Legendre quadrature over the
    sub-cell offset on pieces where the window is a polynomial."""
    N, L = 16, 16.0
    xg, wg = np.polynomial.legendre.leggauss(12)
    breaks = np.linspace(0.0, 1.0, 3)                # pieces [0, 1/2], [1/2, 1]
    xs, ws = [], []
    for a, b in zip(breaks[:-1], breaks[1:]):
        xs.append(0.5 * (b - a) * xg + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * wg)
    xs, ws = np.concatenate(xs), np.concatenate(ws)
    pos = np.stack([4.0 + xs, np.full_like(xs, 8.0), np.full_like(xs, 8.0)], axis=1)
    acc = np.zeros(N // 2 + 1, complex)
    for x0, wq in zip(pos, ws):
        mesh = oracle.paint(x0[None, :], None, L, N, window)
        line = mesh.sum(axis=(1, 2))                 # partition of unity on y, z
        Fn = np.fft.rfft(line)
        acc += wq * Fn * np.exp(2j * np.pi * np.arange(N // 2 + 1) * x0[0] / N)
    n = np.arange(N // 2 + 1)
    want = np.sinc(n / N) ** p                       # np.sinc(x) = sin(pi x)/(pi x)
    assert np.max(np.abs(acc - want)) < 1e-10


# ---------------------------------------------------- Poisson shot noise --

def alias_factor(N, p, interlaced, M=64):
    """Per-axis alias sums A(n) = sum_n' f, B(n) = sum_n' (-1)^n' f, with
    f = sinc^{2p}(pi (n/N + n')) / sinc^{2p}(pi n / N), n = fftfreq index."""
    n = fftfreq_int(N).astype(float)
    nprime = np.arange(-M, M + 1, dtype=float)
    f = np.sinc(n[:, None] / N + nprime[None, :]) ** (2 * p) / np.sinc(n / N)[:, None] ** (2 * p)
    A = f.sum(axis=1)
    B = (f * np.where(nprime % 2 == 0, 1.0, -1.0)[None, :]).sum(axis=1)
    return A, B


def stored_modes(N):
    ip = fftfreq_int(N)
    l = np.arange(N // 2 + 1)
    I, J, Lz = np.meshgrid(ip, ip, l, indexing="ij")
    m = I ** 2 + J ** 2 + Lz ** 2
    h = np.where((Lz == 0) | (Lz == N // 2), 1.0, 2.0)
    return I, J, Lz, m, h


def kbins_of(m, L, kmin, dk, nk):
    kF = (2.0 * math.pi) / L
    b = np.floor((kF * np.sqrt(m.astype(float)) - kmin) / dk).astype(np.int64)
    ok = (m > 0) & (b >= 0) & (b < nk)
    return b, ok


def expected_shot(N, L, p, interlaced, dk, nk):
    """Bin means of E[P_raw] / (L^3 sum w^2 / (sum w)^2) and their variance factor."""
    A, B = alias_factor(N, p, interlaced)
    I, J, Lz, m, h = stored_modes(N)
    ix, jx = I % N, J % N
    if interlaced:
        S = 0.5 * (A[ix] * A[jx] * A[Lz] + B[ix] * B[jx] * B[Lz])
    else:
        S = A[ix] * A[jx] * A[Lz]
    b, ok = kbins_of(m, L, 0.0, dk, nk)
    Eb = np.zeros(nk)
    E2 = np.zeros(nk)
    H = np.zeros(nk)
    np.add.at(Eb, b[ok], (h * S)[ok])
    np.add.at(E2, b[ok], (h * S * S)[ok])
    np.add.at(H, b[ok], h[ok])
    return Eb / H, 2.0 * E2 / H ** 2


def shot_chi2(oracle, window, interlaced, seeds, second_shift=0.5):
    from scipy import stats
    N, L, Np = 32, 500.0, 40000
    p = oracle.WINDOW_ORDER[window]
    kF = 2 * math.pi / L
    dk = 2 * kF
    nk = oracle.nbins(L, N, dk)
    Eb, var = expected_shot(N, L, p, interlaced, dk, nk)
    chi2, dof, zmax = 0.0, 0, 0.0
    for seed in seeds:
        rng = np.random.default_rng(seed)
        pos = rng.uniform(0, L, size=(Np, 3))
        w = rng.uniform(0.5, 1.5, Np)
        F1 = oracle.r2c(oracle.paint(pos, w, L, N, window, 0.0))
        F2 = oracle.r2c(oracle.paint(pos, w, L, N, window, second_shift)) if interlaced else None
        sums = oracle.bin_modes(F1, F2, L, window, True, w.sum(), dk)
        shot = L ** 3 * np.sum(w * w) / w.sum() ** 2
        res = oracle.finalize(sums, shot, subtract_shot=False)
        ratio = res["power"] / shot
        z = (ratio - Eb) / np.sqrt(var)
        chi2 += float(np.sum(z ** 2))
        dof += nk
        zmax = max(zmax, float(np.max(np.abs(z))))
    return chi2, dof, zmax, stats.chi2.sf(chi2, dof)


@pytest.mark.parametrize("window,interlaced", [("cic", False), ("tsc", False), ("pcs", False),
                                                ("cic", True), ("tsc", True), ("pcs", True)])
def test_uniform_catalog_gives_aliased_shot_noise(oracle, window, interlaced):
    chi2, dof, zmax, pval = shot_chi2(oracle, window, interlaced, seeds=[101, 102, 103])
    assert zmax < 5.0 and pval > 1e-4, (chi2, dof, zmax, pval)


def test_planted_wrong_interlace_direction_is_rejected(oracle):
    """Negative control: paint the second mesh at x - H/2 (the opposite of the
    exp(+i k H/2) phase) and the same statistic must fail."""
    chi2, dof, zmax, pval = shot_chi2(oracle, "cic", True, seeds=[101, 102, 103], second_shift=-0.5)
    assert pval < 1e-8, (chi2, dof, zmax, pval)


def test_cic_alias_sum_matches_closed_form():
    """Cross-check of the test's own alias helper against the closed form
    sum_n' sinc^4(pi(x + n')) = 1 - (2/3) sin^2(pi x) for CIC (not assumed)."""
    N = 32
    A, _ = alias_factor(N, 2, False, M=400)
    n = fftfreq_int(N)
    closed = (1 - 2.0 / 3.0 * np.sin(np.pi * n / N) ** 2) / np.sinc(n / N) ** 4
    assert np.max(np.abs(A / closed - 1)) < 1e-9


# --------------------------------------------------- Gaussian / Kaiser field --

def gaussian_half_grid(N, L, seed, amp, slope, f_kaiser):
    rng = np.random.default_rng(seed)
    G = np.fft.rfftn(rng.standard_normal((N, N, N)))      # E|G|^2 = N^3
    I, J, Lz, m, h = stored_modes(N)
    k = (2 * math.pi / L) * np.sqrt(m.astype(float))
    k[m == 0] = 1.0
    Pk = amp * k ** slope
    mu2 = np.where(m > 0, Lz ** 2 / np.maximum(m, 1), 0.0)
    kaiser = (1.0 + f_kaiser * mu2)
    delta = G * np.sqrt(Pk / (L ** 3 * N ** 3)) * kaiser
    return delta, Pk * kaiser ** 2, mu2, m, h


@pytest.mark.parametrize("f_kaiser", [0.0, 0.75])
def test_gaussian_field_power_and_multipoles(oracle, f_kaiser):
    from scipy import stats
    N, L = 48, 1000.0
    dk = 3 * 2 * math.pi / L
    nk = oracle.nbins(L, N, dk)
    chi2, dof = 0.0, 0
    for seed in (5, 6):
        delta, Emode, mu2, m, h = gaussian_half_grid(N, L, seed, 2.0e4, -1.5, f_kaiser)
        sums = oracle.bin_modes(delta, None, L, "cic", False, 1.0, dk, nmu=5)
        res = oracle.finalize(sums, 0.0, subtract_shot=False)
        b, ok = kbins_of(m, L, 0.0, dk, nk)
        Lpoly = [np.ones_like(mu2), 0.5 * (3 * mu2 - 1), (35 * mu2 ** 2 - 30 * mu2 + 3) / 8]
        H = np.zeros(nk)
        np.add.at(H, b[ok], h[ok])
        for ell, Lp in zip((0, 2, 4), Lpoly):
            E = np.zeros(nk)
            V = np.zeros(nk)
            np.add.at(E, b[ok], (h * Emode * Lp)[ok])
            np.add.at(V, b[ok], (h * (Emode * Lp) ** 2)[ok])
            E = (2 * ell + 1) * E / H
            V = (2 * ell + 1) ** 2 * 2 * V / H ** 2
            z = (res["poles"][ell // 2] - E) / np.sqrt(V)
            assert np.max(np.abs(z)) < 5.0, (ell, z)
            chi2 += float(np.sum(z ** 2))
            dof += nk
    assert stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof)


def test_unit_field_gives_exact_legendre_averages(oracle):
    """|delta|^2 = 1 on every mode: P_0 = L^3 exactly and P_2, P_4 equal exact
    rational averages over the integer mode triples (mu^2 = l^2 / m)."""
    N, L = 12, 7.0
    dk = 2 * math.pi / L
    nk = oracle.nbins(L, N, dk)
    F = np.ones((N, N, N // 2 + 1), complex)
    sums = oracle.bin_modes(F, None, L, "cic", False, 1.0, dk, nmu=3)
    res = oracle.finalize(sums, 0.0, subtract_shot=False)
    acc = [[Fraction(0)] * nk for _ in range(3)]
    cnt = [0] * nk
    for i in fftfreq_int(N):
        for j in fftfreq_int(N):
            for l in range(N // 2 + 1):
                m = int(i * i + j * j + l * l)
                if m == 0:
                    continue
                b = oracle.kbin(m, L, 0.0, dk)
                if not 0 <= b < nk:
                    continue
                h = 1 if l in (0, N // 2) else 2
                mu2 = Fraction(l * l, m)
                cnt[b] += h
                acc[0][b] += h
                acc[1][b] += h * Fraction(5, 2) * (3 * mu2 - 1)
                acc[2][b] += h * Fraction(9, 8) * (35 * mu2 * mu2 - 30 * mu2 + 3)
    for b in range(nk):
        if cnt[b] == 0:                      # bin 0 holds only DC here: empty
            assert np.all(np.isnan(res["poles"][:, b]))
            continue
        for ell in range(3):
            want = float(acc[ell][b] / cnt[b]) * L ** 3
            got = res["poles"][ell][b]
            assert abs(got - want) <= 1e-12 * L ** 3, (b, ell, got, want)
    assert np.all(res["modes"] == np.array(cnt))


# ------------------------------------------------------------ mode counts --

@pytest.mark.parametrize("N,L,dk,nmu", [(16, 100.0, 0.07, 4), (18, 3.0, 0.5, 10), (20, 1000.0, 0.01, 7)])
def test_half_grid_counts_equal_full_grid_enumeration(oracle, N, L, dk, nmu):
    nk = oracle.nbins(L, N, dk)
    F = np.ones((N, N, N // 2 + 1), complex)
    sums = oracle.bin_modes(F, None, L, "cic", False, 1.0, dk, nmu=nmu)
    c1 = np.zeros(nk, np.int64)
    c2 = np.zeros((nk, nmu), np.int64)
    f = fftfreq_int(N)
    for i in f:
        for j in f:
            for l in f:                      # the full grid, every mode weight 1
                m = int(i * i + j * j + l * l)
                if m == 0:
                    continue
                b = int(math.floor(((2.0 * math.pi) / L * math.sqrt(m) - 0.0) / dk))
                if not 0 <= b < nk:
                    continue
                q = 0
                while q + 1 <= nmu and (q + 1) ** 2 * m <= nmu * nmu * l * l:
                    q += 1
                q = min(q, nmu - 1)
                c1[b] += 1
                c2[b, q] += 1
    assert np.array_equal(sums["modes1d"], c1)
    assert np.array_equal(sums["modes2d"].reshape(nk, nmu), c2)


def test_mu_bin_worked_examples(oracle):
    # (i', j', l) = (3, 0, 4): m = 25, mu = 0.8 exactly -> lower edge of bin 8 of 10
    assert oracle.mubin(25, 4, 10) == 8
    # (4, 0, 3): mu = 0.6 exactly -> bin 6
    assert oracle.mubin(25, 3, 10) == 6
    # mu = 1 (mode along the line of sight) -> last bin
    assert oracle.mubin(49, 7, 10) == 9
    # l = 0 -> mu = 0 -> bin 0
    assert oracle.mubin(5, 0, 10) == 0
    # mu = 1/sqrt(2) = 0.7071 -> bin 7
    assert oracle.mubin(2, 1, 10) == 7


# ------------------------------------------------- full brute-force pipeline --

@pytest.mark.parametrize("window,interlaced,compensated", [("tsc", True, True), ("cic", False, True),
                                                           ("pcs", True, False)])
def test_pipeline_equals_full_grid_bruteforce(oracle, window, interlaced, compensated):
    rng = np.random.default_rng(21)
    N, L, nmu = 8, 10.0, 4
    p = oracle.WINDOW_ORDER[window]
    pos = rng.uniform(0, L, size=(30, 3))
    w = rng.uniform(0.2, 3.0, 30)
    kF = 2 * math.pi / L
    dk = 0.8 * kF
    res = oracle.fft_power(pos, w, L, N, window, interlaced, compensated, dk=dk, nmu=nmu)
    # brute force: per-cell paint, O(N^6) full complex DFT, full-grid mode loop
    c = np.arange(N)
    E = np.exp(-2j * np.pi * np.outer(c, c) / N)
    meshes = [brute_paint(pos, w, L, N, p, 0.0, oracle)]
    if interlaced:
        meshes.append(brute_paint(pos, w, L, N, p, 0.5, oracle))
    full = [np.einsum("ai,bj,ck,ijk->abc", E, E, E, M) for M in meshes]
    f = fftfreq_int(N)
    nk = oracle.nbins(L, N, dk)
    S0, S2, S4, Hc = np.zeros(nk), np.zeros(nk), np.zeros(nk), np.zeros(nk)
    S2d, H2d = np.zeros((nk, nmu)), np.zeros((nk, nmu))
    for a in range(N):
        for b_ in range(N):
            for cz in range(N):
                n = np.array([f[a], f[b_], f[cz]])
                m = int(np.sum(n * n))
                if m == 0:
                    continue
                kb = int(math.floor((kF * math.sqrt(m) - 0.0) / dk))
                if not 0 <= kb < nk:
                    continue
                d = full[0][a, b_, cz]
                if interlaced:
                    d = 0.5 * (d + full[1][a, b_, cz] * np.exp(1j * np.pi * n.sum() / N))
                if compensated:
                    d = d / np.prod(np.sinc(n / N) ** p)
                P = L ** 3 * abs(d / w.sum()) ** 2
                mu2 = n[2] ** 2 / m
                S0[kb] += P
                S2[kb] += P * 0.5 * (3 * mu2 - 1)
                S4[kb] += P * (35 * mu2 ** 2 - 30 * mu2 + 3) / 8
                Hc[kb] += 1
                q = min(int(math.floor(nmu * abs(n[2]) / math.sqrt(m) + 1e-12)), nmu - 1)
                S2d[kb, q] += P
                H2d[kb, q] += 1
    shot = L ** 3 * np.sum(w * w) / w.sum() ** 2
    assert np.array_equal(res["modes"], Hc.astype(np.int64))
    np.testing.assert_allclose(res["power"], S0 / Hc - shot, rtol=1e-10, atol=1e-10 * shot)
    np.testing.assert_allclose(res["poles"][1], 5 * S2 / Hc, rtol=1e-9, atol=1e-10 * shot)
    np.testing.assert_allclose(res["poles"][2], 9 * S4 / Hc, rtol=1e-9, atol=1e-10 * shot)
    with np.errstate(invalid="ignore"):
        np.testing.assert_allclose(res["power2d"], S2d / H2d - shot, rtol=1e-10, atol=1e-10 * shot)


# ------------------------------------------- block paint and mode counts --

@pytest.mark.parametrize("window,shift", [("pcs", 0.5), ("tsc", 0.0), ("cic", 0.5)])
def test_paint_block_equals_per_cell_bruteforce(oracle, window, shift):
    """The block-restricted paint equals the per-cell brute force on blocks
    inside the box and blocks that wrap around its periodic faces."""
    rng = np.random.default_rng(31)
    N, L = 12, 30.0
    pos = rng.uniform(0, L, size=(400, 3))
    w = rng.uniform(0.5, 1.5, 400)
    full = brute_paint(pos, w, L, N, oracle.WINDOW_ORDER[window], shift, oracle)
    for c0, B in (((2, 3, 4), 5), ((10, 11, 9), 4), ((0, 0, 0), 12)):
        got = oracle.paint_block(pos, w, L, N, window, c0, B, shift)
        idx = [(np.arange(B) + c) % N for c in c0]
        ref = full[np.ix_(*idx)]
        assert np.max(np.abs(got - ref)) < 1e-13, (c0, B)


@pytest.mark.parametrize("N,L,dk,nmu", [(16, 100.0, 0.07, 4), (14, 5.0, 0.6, 3)])
def test_mode_counts_equal_full_grid_enumeration(oracle, N, L, dk, nmu):
    c1, c2 = oracle.mode_counts(N, L, dk, nmu=nmu)
    nk = oracle.nbins(L, N, dk)
    r1 = np.zeros(nk, np.int64)
    r2 = np.zeros((nk, nmu), np.int64)
    f = fftfreq_int(N)
    for i in f:
        for j in f:
            for l in f:
                m = int(i * i + j * j + l * l)
                if m == 0:
                    continue
                b = int(math.floor(((2.0 * math.pi) / L * math.sqrt(m) - 0.0) / dk))
                if not 0 <= b < nk:
                    continue
                q = min(int(math.isqrt(nmu * nmu * l * l // m)) if l else 0, nmu - 1)
                while q + 1 <= nmu - 1 and (q + 1) ** 2 * m <= nmu * nmu * l * l:
                    q += 1
                while q > 0 and q * q * m > nmu * nmu * l * l:
                    q -= 1
                r1[b] += 1
                r2[b, q] += 1
    assert np.array_equal(c1, r1)
    assert np.array_equal(c2, r2)
