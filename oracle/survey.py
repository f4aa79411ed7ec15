"""FP64 CPU oracle of the survey power-spectrum multipoles (ConvolvedFFTPower,
Sec. 3.4.1: multipoles of data given as right ascension, declination and
redshift, with a line of sight that points from the observer to each point).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` may import it.  It shares no code
with the CUDA library.

The paper states the estimator by reference only (the FFT-based estimator of
Hand et al. 2017, 2l + 1 FFTs per multipole l, improving on Bianchi et al.
2015 and Scoccimarro 2015, after Feldman, Kaiser & Peacock 1994 and Yamamoto
et al. 2006).  What it computes, written out here:

  FKP field     F(x) = n_d(x) - alpha n_r(x), each object painted with
                w = w_comp w_fkp; alpha = sum_d w_comp / sum_r w_comp.
  multipole     A_l(k) = sum_c F(x_c) exp(-i k.x_c) L_l(k^.x^_c), x_c the
  fields        observer-frame position of mesh node c, x^ = x / |x|.
  estimator     P_l(k) = (2l + 1) / I < Re[A_l(k) A_0(k)^*] / W^2(k) >_bin
                         - [l = 0] S
                with W(k) the window's transform (1 when not compensated),
                I = alpha sum_r nbar w_comp w_fkp^2 (the normalization from
                the randoms) and S = (sum_d w^2 + alpha^2 sum_r w^2) / I.

Two routes to A_l are written here.  ``multipoles_direct`` is the definition
summed over cells for every mode (tiny meshes only).  ``multipole_fields``
expands the Legendre polynomial in powers of k^.x^ (the Cartesian moments of
Bianchi et al. and Scoccimarro): (k^.x^)^2 = sum_ij k^_i k^_j x^_i x^_j, so
A_2 and A_4 come from the FFTs of F x^_i x^_j (6 fields) and of
F x^_i x^_j x^_k x^_l (15 fields).  The CUDA path uses the third route, the
spherical-harmonic addition theorem (2l + 1 FFTs per l); all three agree up to
rounding.

Readings where the paper is silent:
  * the common phase exp(-i k.x_0) of the box origin x_0 is dropped (it
    cancels in A_l A_0^*): A_l is the DFT over node indices;
  * a node exactly at the observer has no line of sight; it contributes to
    A_0 only;
  * interlacing combines the two painted meshes in Fourier space,
    (F~_1 + F~_2 exp(i k.(H/2)(1,1,1))) / 2, and the multipole fields are
    built from the inverse transform of that combination, without the modes
    that have an index at N/2 (their half-cell phase has no sign that keeps
    the combination Hermitian, and they lie at |k| >= k_N, outside every
    bin); the window compensation divides the binned products by W^2(k);
  * k bins, the mode weights h (1 on the l_z = 0 and N/2 planes, else 2) and
    the exclusion of k = 0 follow the periodic-box estimator of this oracle;
  * distances: flat LambdaCDM without radiation, chi(z) = (c / H0)
    int_0^z dz' / E(z'), E = sqrt(Om (1 + z)^3 + 1 - Om), in Mpc/h
    (c / H0 = 2997.92458 Mpc/h); RA and Dec in degrees.
"""
from __future__ import annotations

import math

import numpy as np

from . import WINDOW_ORDER, kbin, nbins, paint

C_OVER_H0 = 2997.92458          # Mpc/h: 299792.458 km/s over 100 h km/s/Mpc
ELLS = (0, 2, 4)


# ------------------------------------------------------------- distances --

def comoving_distance(z, omega_m: float, nodes: int = 64):
    """Line-of-sight comoving distance chi(z) in Mpc/h (flat LambdaCDM),
    Gauss-Legendre quadrature of 1 / E over [0, z] with `nodes` points."""
    z = np.asarray(z, dtype=np.float64)
    x, wq = np.polynomial.legendre.leggauss(int(nodes))
    flat = z.reshape(-1)
    out = np.empty_like(flat)
    for a in range(0, flat.size, 65536):
        zz = flat[a:a + 65536]
        zs = 0.5 * zz[:, None] * (x[None, :] + 1.0)
        E = np.sqrt(omega_m * (1.0 + zs) ** 3 + (1.0 - omega_m))
        out[a:a + 65536] = C_OVER_H0 * 0.5 * zz * np.sum(wq[None, :] / E, axis=1)
    return out.reshape(z.shape)


def sky_to_cartesian(ra_deg, dec_deg, z, omega_m: float):
    """Observer-frame Cartesian positions (n, 3) in Mpc/h: RA about +z from
    +x, Dec from the xy plane, radius chi(z)."""
    ra = np.radians(np.asarray(ra_deg, dtype=np.float64))
    dec = np.radians(np.asarray(dec_deg, dtype=np.float64))
    chi = comoving_distance(z, omega_m)
    return np.stack([chi * np.cos(dec) * np.cos(ra), chi * np.cos(dec) * np.sin(ra), chi * np.sin(dec)],
                    axis=-1)


# ------------------------------------------------------------ FKP sums --

def catalog_sums(wcomp, wfkp, nbar, n: int) -> dict:
    """sum w_comp, sum (w_comp w_fkp)^2 and sum nbar w_comp w_fkp^2 of one
    catalog (None columns are 1; nbar None gives no normalization sum)."""
    wc = np.ones(n) if wcomp is None else np.asarray(wcomp, dtype=np.float64)
    wf = np.ones(n) if wfkp is None else np.asarray(wfkp, dtype=np.float64)
    out = {"n": n, "wsum": float(np.sum(wc)), "w2sum": float(np.sum((wc * wf) ** 2))}
    out["nsum"] = None if nbar is None else float(np.sum(np.asarray(nbar, dtype=np.float64) * wc * wf * wf))
    return out


def fkp_constants(data_sums: dict, rand_sums: dict) -> dict:
    """alpha, the normalization I and the shot noise S (FKP, Yamamoto)."""
    alpha = data_sums["wsum"] / rand_sums["wsum"]
    norm = alpha * rand_sums["nsum"]
    shot = (data_sums["w2sum"] + alpha * alpha * rand_sums["w2sum"]) / norm
    return {"alpha": alpha, "norm": norm, "shot_noise": shot}


def fkp_weights(nbar, p0: float):
    """w_fkp = 1 / (1 + nbar P0)."""
    return 1.0 / (1.0 + np.asarray(nbar, dtype=np.float64) * float(p0))


# ----------------------------------------------------------- the field --

def fkp_meshes(data_pos, data_w, rand_pos, rand_w, alpha: float, box_size: float, box_origin, nmesh: int,
               window, interlaced: bool):
    """F = D - alpha R painted on the (N, N, N) mesh whose node c sits at
    box_origin + c H (observer frame); a second mesh shifted by H/2 when
    interlaced.  Positions are observer-frame (n, 3) arrays."""
    o = np.asarray(box_origin, dtype=np.float64).reshape(1, 3)
    dp = np.asarray(data_pos, dtype=np.float64).reshape(-1, 3) - o
    rp = np.asarray(rand_pos, dtype=np.float64).reshape(-1, 3) - o
    out = []
    for shift in ((0.0, 0.5) if interlaced else (0.0,)):
        D = paint(dp, data_w, box_size, nmesh, window, shift)
        R = paint(rp, rand_w, box_size, nmesh, window, shift)
        out.append(D - alpha * R)
    return out


def interlaced_field(F1, F2):
    """Real field whose transform is (F~_1 + F~_2 exp(i pi (n_x + n_y + n_z) / N)) / 2
    on every mode with no index at N/2 (those set to zero)."""
    if F2 is None:
        return np.asarray(F1, dtype=np.float64)
    N = F1.shape[0]
    f = np.fft.fftfreq(N, 1.0 / N)
    fz = np.fft.rfftfreq(N, 1.0 / N)
    ph = np.exp(1j * math.pi * (f[:, None, None] + f[None, :, None] + fz[None, None, :]) / N)
    C = 0.5 * (np.fft.rfftn(F1) + np.fft.rfftn(F2) * ph)
    h = N // 2
    C[h, :, :] = 0.0
    C[:, h, :] = 0.0
    C[:, :, h] = 0.0
    return np.fft.irfftn(C, s=F1.shape, axes=(0, 1, 2))


def node_directions(nmesh: int, box_size: float, box_origin):
    """Unit vectors x^ of the mesh nodes (3, N, N, N) and the mask of nodes
    not at the observer."""
    H = box_size / nmesh
    c = np.arange(nmesh, dtype=np.float64) * H
    o = np.asarray(box_origin, dtype=np.float64)
    X, Y, Z = np.meshgrid(o[0] + c, o[1] + c, o[2] + c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    away = r > 0.0
    rs = np.where(away, r, 1.0)
    return np.stack([X / rs * away, Y / rs * away, Z / rs * away]), away


def _half_grid_khat(N: int):
    """k^ on the stored half grid (3, N, N, N/2 + 1), zero at k = 0, and m = |n|^2."""
    f = np.fft.fftfreq(N, 1.0 / N)
    fz = np.arange(N // 2 + 1, dtype=np.float64)
    I, J, K = np.meshgrid(f, f, fz, indexing="ij")
    m = I * I + J * J + K * K
    kn = np.sqrt(np.where(m > 0, m, 1.0))
    return np.stack([I / kn, J / kn, K / kn]), (I * I + J * J + K * K).astype(np.int64)


def multipole_fields(F, box_size: float, box_origin, ells=ELLS) -> dict:
    """A_l on the stored half grid through the Cartesian moments of x^."""
    N = F.shape[0]
    xh, away = node_directions(N, box_size, box_origin)
    khat, _ = _half_grid_khat(N)
    A0 = np.fft.rfftn(F)
    out = {0: A0}
    if not any(l > 0 for l in ells):
        return out
    Fa = np.fft.rfftn(F * away)              # nodes with a line of sight
    S2 = np.zeros_like(A0)
    for i in range(3):
        for j in range(i, 3):
            mult = 1.0 if i == j else 2.0
            S2 += mult * khat[i] * khat[j] * np.fft.rfftn(F * xh[i] * xh[j])
    if 2 in ells:
        out[2] = 0.5 * (3.0 * S2 - Fa)
    if 4 in ells:
        S4 = np.zeros_like(A0)
        for a in range(5):
            for b in range(5 - a):
                c = 4 - a - b
                mult = math.factorial(4) / (math.factorial(a) * math.factorial(b) * math.factorial(c))
                mono = xh[0] ** a * xh[1] ** b * xh[2] ** c
                S4 += mult * khat[0] ** a * khat[1] ** b * khat[2] ** c * np.fft.rfftn(F * mono)
        out[4] = (35.0 * S4 - 30.0 * S2 + 3.0 * Fa) / 8.0
    for ell in out:
        if ell > 0:
            out[ell][0, 0, 0] = 0.0          # k = 0 has no direction (and is never binned)
    return out


def multipoles_direct(F, box_size: float, box_origin, ells=ELLS) -> dict:
    """A_l on the stored half grid by the definition: for every mode, the sum
    over nodes of F exp(-2 pi i c.n / N) L_l(k^.x^_c) (Legendre polynomials
    from numpy).  O(N^6): meshes of a few thousand nodes only."""
    N = F.shape[0]
    xh, away = node_directions(N, box_size, box_origin)
    khat, m = _half_grid_khat(N)
    c = np.arange(N, dtype=np.float64)
    Ci, Cj, Ck = np.meshgrid(c, c, c, indexing="ij")
    f = np.fft.fftfreq(N, 1.0 / N)
    Fv = F.reshape(-1)
    xv = xh.reshape(3, -1)
    out = {l: np.zeros((N, N, N // 2 + 1), np.complex128) for l in ells}
    for a in range(N):
        for b in range(N):
            for l in range(N // 2 + 1):
                ph = np.exp(-2j * math.pi * (Ci * f[a] + Cj * f[b] + Ck * l) / N).reshape(-1)
                if m[a, b, l] == 0:
                    out[0][a, b, l] = np.sum(Fv * ph)
                    continue
                mu = khat[0, a, b, l] * xv[0] + khat[1, a, b, l] * xv[1] + khat[2, a, b, l] * xv[2]
                for ell in ells:
                    coef = np.zeros(ell + 1)
                    coef[ell] = 1.0
                    Lw = np.polynomial.legendre.legval(mu, coef)
                    if ell > 0:
                        Lw = Lw * away.reshape(-1)
                    out[ell][a, b, l] = np.sum(Fv * ph * Lw)
    return out


# -------------------------------------------------------------- binning --

def bin_multipoles(A: dict, box_size: float, window, compensated: bool, dk: float, kmin: float = 0.0,
                   kmax=None) -> dict:
    """Bin sums over the stored half grid: modes sum h, ksum sum h k and, per
    l, sum h Re[A_l A_0^*] / W^2 (k = 0 excluded; exact k bins)."""
    A0 = A[0]
    N = A0.shape[0]
    _, m = _half_grid_khat(N)
    nk = nbins(box_size, N, dk, kmin, kmax)
    b = np.full(m.shape, -1, np.int64)
    for mv in np.unique(m):
        if mv > 0:
            b[m == mv] = kbin(int(mv), box_size, kmin, dk)
    ok = (m > 0) & (b >= 0) & (b < nk)
    lz = np.arange(N // 2 + 1)
    h = np.where((lz == 0) | (lz == N // 2), 1.0, 2.0)[None, None, :] * np.ones(m.shape)
    cw = np.ones(m.shape)
    if compensated:
        p = WINDOW_ORDER[window] if isinstance(window, str) else int(window)
        f = np.fft.fftfreq(N, 1.0 / N)
        fz = np.arange(N // 2 + 1, dtype=np.float64)
        W = (np.sinc(f[:, None, None] / N) * np.sinc(f[None, :, None] / N) * np.sinc(fz[None, None, :] / N)) ** p
        cw = 1.0 / (W * W)
    kF = 2.0 * math.pi / box_size
    out = {"nk": nk,
           "modes": np.bincount(b[ok], weights=h[ok], minlength=nk).round().astype(np.int64),
           "ksum": np.bincount(b[ok], weights=(h * kF * np.sqrt(m.astype(np.float64)))[ok], minlength=nk),
           "sums": {}}
    for ell, Al in A.items():
        v = h * cw * np.real(Al * np.conj(A0))
        out["sums"][ell] = np.bincount(b[ok], weights=v[ok], minlength=nk)
    return out


# ---------------------------------------------------------- whole path --

def convolved_power(data: dict, randoms: dict, box_size: float, box_origin, nmesh: int, window="cic",
                    interlaced: bool = False, compensated: bool = True, dk=None, kmin: float = 0.0,
                    kmax=None, poles=ELLS, subtract_shot: bool = True, omega_m=None, p0_fkp: float = 0.0):
    """Survey multipoles in FP64.  Each catalog is a dict with either 'pos'
    (observer-frame (n, 3), Mpc/h) or 'ra', 'dec', 'z' (degrees, redshift;
    needs omega_m), and optional 'wcomp', 'wfkp', 'nbar' columns.  With
    p0_fkp > 0 the FKP weights are 1 / (1 + nbar P0)."""
    cats = []
    for cat in (data, randoms):
        if "pos" in cat:
            pos = np.asarray(cat["pos"], dtype=np.float64).reshape(-1, 3)
        else:
            pos = sky_to_cartesian(cat["ra"], cat["dec"], cat["z"], omega_m)
        n = pos.shape[0]
        wfkp = cat.get("wfkp")
        if p0_fkp > 0:
            wfkp = fkp_weights(cat["nbar"], p0_fkp)
        sums = catalog_sums(cat.get("wcomp"), wfkp, cat.get("nbar"), n)
        wc = np.ones(n) if cat.get("wcomp") is None else np.asarray(cat["wcomp"], dtype=np.float64)
        wf = np.ones(n) if wfkp is None else np.asarray(wfkp, dtype=np.float64)
        cats.append((pos, wc * wf, sums))
    (dpos, dw, dsum), (rpos, rw, rsum) = cats
    const = fkp_constants(dsum, rsum)
    meshes = fkp_meshes(dpos, dw, rpos, rw, const["alpha"], box_size, box_origin, nmesh, window, interlaced)
    F = interlaced_field(meshes[0], meshes[1] if interlaced else None)
    ells = tuple(sorted(set((0,) + tuple(poles))))
    A = multipole_fields(F, box_size, box_origin, ells)
    sums = bin_multipoles(A, box_size, window, compensated, dk, kmin, kmax)
    modes = sums["modes"].astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        res = {"k": sums["ksum"] / modes, "modes": sums["modes"], "nk": sums["nk"],
               "power_raw": sums["sums"][0] / modes / const["norm"], "poles": {}}
        for ell in poles:
            P = (2 * ell + 1) * sums["sums"][ell] / modes / const["norm"]
            if ell == 0 and subtract_shot:
                P = P - const["shot_noise"]
            res["poles"][ell] = P
    res.update(const)
    res["data_sums"], res["rand_sums"] = dsum, rsum
    return res
