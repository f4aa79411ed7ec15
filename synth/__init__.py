"""Seeded synthetic catalogs for tests and benchmarks.

Shared by the oracle side (tests) and the CUDA side (tests, bench).  Holds none
of the estimator's arithmetic (no painting, no windows, no binning): it only
draws object positions with the structure of the paper's workloads --
uniform random catalogs, Poisson-sampled log-normal fields with a linear
redshift-space displacement (the kind of LogNormalCatalog the paper's tests
and benchmarks use, Sec. 3.2 and Sec. 3.3.2) and Zel'dovich-displaced
lattices.  Gaussian fields are drawn with torch (CPU or CUDA) from a seeded
generator; positions come back as torch tensors on the requested device.

Gaussian field convention: for white noise W on an N^3 grid (E|W~|^2 = N^3),
G~(n) = W~(n) sqrt(P(k) N^3 / L^3) gives a grid field whose variance is
(1/L^3) sum_{k != 0} P(k).
"""
from __future__ import annotations

import math

import numpy as np
import torch

SEED_BASE = 20171215


def seed_for(config: int, mock: int = 0) -> int:
    """Seed of mock `mock` of workload `config`: 20171215 + 1000 config + mock."""
    return SEED_BASE + 1000 * int(config) + int(mock)


def uniform_catalog(n: int, box_size: float, seed: int, dtype=np.float64) -> np.ndarray:
    """n objects uniform in [0, L)^3 (numpy PCG64), shape (n, 3)."""
    rng = np.random.default_rng(seed)
    return (rng.random((n, 3)) * box_size).astype(dtype)


def _kgrid(ng: int, box_size: float, device):
    kf = 2.0 * math.pi / box_size
    f = torch.fft.fftfreq(ng, d=1.0 / ng, device=device, dtype=torch.float64) * kf
    fz = torch.fft.rfftfreq(ng, d=1.0 / ng, device=device, dtype=torch.float64) * kf
    return f[:, None, None], f[None, :, None], fz[None, None, :]


def gaussian_field_k(ng: int, box_size: float, slope: float, seed: int, device="cpu",
                     amp: float | None = None, variance: float = 1.0):
    """Half-grid transform G~ of a Gaussian field with P(k) = A k^slope.

    If amp is None, A is set so the grid variance (1/L^3) sum_{k!=0} P(k)
    equals `variance`.  Returns (G~ complex64 on device, A)."""
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    w = torch.randn((ng, ng, ng), generator=gen, device=device, dtype=torch.float32)
    wk = torch.fft.rfftn(w)
    del w
    kx, ky, kz = _kgrid(ng, box_size, device)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    shape = (k2 ** (0.5 * slope))
    shape[0, 0, 0] = 0.0
    if amp is None:
        # full-grid sum of k^slope: the half grid counts planes 0 and ng/2 once
        h = torch.full((ng // 2 + 1,), 2.0, dtype=torch.float64, device=device)
        h[0] = 1.0
        if ng % 2 == 0:
            h[-1] = 1.0
        total = float((shape * h[None, None, :]).sum())
        amp = variance * box_size ** 3 / total
    scale = torch.sqrt(amp * shape * (ng ** 3) / box_size ** 3).to(torch.float32)
    return wk * scale, amp


def _displacement(gk, box_size: float, axis: int):
    """Linear displacement psi_a = IFFT(i k_a / k^2 G~) on the grid (Mpc/h)."""
    ng = gk.shape[0]
    kx, ky, kz = _kgrid(ng, box_size, gk.device)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    ka = (kx, ky, kz)[axis]
    fac = (ka / k2).to(torch.float32)
    psi_k = gk * (1j * fac)
    psi_k[0, 0, 0] = 0.0
    return torch.fft.irfftn(psi_k, s=(ng, ng, ng))


def _cell_cdf(rho, ngrid: int):
    """Running sum of the cell weights in cell order.  On the CPU a plain
    cumsum (sequential, the same every run).  On a GPU a 1-D cumsum is a
    single-pass scan whose floating-point summation order depends on the
    timing of its blocks, so two processes could draw different cells for
    the same seed; there each z row is summed on its own (one row per
    thread block, a fixed order) and the row totals are summed on the host."""
    if rho.device.type == "cpu":
        return torch.cumsum(rho, 0)
    rows = torch.cumsum(rho.reshape(ngrid * ngrid, ngrid), 1)
    start = torch.cumsum(rows[:, -1].cpu(), 0) - rows[:, -1].cpu()
    return (rows + start.to(rho.device)[:, None]).reshape(-1)


def lognormal_catalog(n: int, box_size: float, ngrid: int, seed: int, slope: float = -1.5,
                      variance: float = 1.0, f_rsd: float = 0.75, device="cpu",
                      dtype=torch.float32):
    """n objects Poisson-sampled from a log-normal field on an ngrid^3 grid.

    1 + delta = exp(G - sigma_G^2 / 2) with G Gaussian, P_G(k) = A k^slope and A
    chosen so sigma_G^2 = `variance` at the cell scale.  Exactly n objects are
    drawn by inverse-CDF sampling of cells with probability proportional to
    1 + delta (a multinomial draw), placed uniformly inside their cell, then
    displaced along z by f_rsd * psi_z with psi the linear displacement of G
    (redshift-space distortion), and wrapped into [0, L).  Shape (n, 3)."""
    gk, _ = gaussian_field_k(ngrid, box_size, slope, seed, device, variance=variance)
    g = torch.fft.irfftn(gk, s=(ngrid, ngrid, ngrid))
    sig2 = float(g.double().var())
    rho = torch.exp(g.double() - 0.5 * sig2).reshape(-1)
    del g
    cdf = _cell_cdf(rho, ngrid)
    del rho
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) + 1)
    u = torch.rand(n, generator=gen, device=device, dtype=torch.float64) * float(cdf[-1])
    cell = torch.searchsorted(cdf, u).clamp_(max=ngrid ** 3 - 1)
    del cdf, u
    H = box_size / ngrid
    ix = cell // (ngrid * ngrid)
    iy = (cell // ngrid) % ngrid
    iz = cell % ngrid
    off = torch.rand((n, 3), generator=gen, device=device, dtype=torch.float64)
    pos = torch.stack([ix, iy, iz], dim=1).to(torch.float64).add_(off).mul_(H)
    del off
    if f_rsd:
        psi_z = _displacement(gk, box_size, 2).reshape(-1)
        pos[:, 2] += f_rsd * psi_z[cell].to(torch.float64)
        del psi_z
        pos[:, 2] = torch.remainder(pos[:, 2], box_size)
    return pos.to(dtype)


def zeldovich_lattice(nside: int, box_size: float, seed: int, slope: float = -2.0,
                      rms_frac: float = 0.25, device="cpu", dtype=torch.float32):
    """nside^3 objects on a lattice (spacing L / nside) displaced by the linear
    (Zel'dovich) displacement of a Gaussian field with P(k) ~ k^slope, scaled
    so the rms displacement is rms_frac lattice spacings; wrapped into [0, L).
    Shape (nside^3, 3)."""
    gk, _ = gaussian_field_k(nside, box_size, slope, seed, device, variance=1.0)
    spacing = box_size / nside
    psis = [_displacement(gk, box_size, a) for a in range(3)]
    rms = math.sqrt(sum(float((p.double() ** 2).mean()) for p in psis))
    scale = rms_frac * spacing / rms
    del gk
    out = torch.empty((nside ** 3, 3), device=device, dtype=dtype)
    q = torch.arange(nside, device=device, dtype=torch.float64) * spacing
    for a in range(3):
        shape = [1, 1, 1]
        shape[a] = nside
        qa = q.reshape(shape).expand(nside, nside, nside)
        x = torch.remainder(qa + scale * psis[a].double(), box_size)
        out[:, a] = x.reshape(-1).to(dtype)
        psis[a] = None
        del x
    return out


def mock_set_specs(n_mocks: int, seed: int, n_lo: float = 2e5, n_hi: float = 4e6,
                   meshes=(128, 192, 256), windows=("cic", "tsc")) -> list:
    """Specs of a covariance mock set: per mock an object count log-uniform in
    [n_lo, n_hi], a mesh size and a window drawn uniformly from the choices,
    and the mock's own seed.  numpy PCG64 from `seed`."""
    rng = np.random.default_rng(seed)
    logn = rng.uniform(math.log(n_lo), math.log(n_hi), n_mocks)
    ns = np.floor(np.exp(logn)).astype(np.int64)
    nm = rng.choice(np.asarray(meshes), n_mocks)
    wi = rng.integers(0, len(windows), n_mocks)
    return [{"n": int(ns[i]), "nmesh": int(nm[i]), "window": windows[int(wi[i])],
             "seed": int(seed) + 1 + i} for i in range(n_mocks)]


# ----------------------------------------------------------------------
# Survey-like catalogs (the ConvolvedFFTPower workload, Sec. 3.4.1): an
# observer at the origin, objects in a shell octant with a radial selection,
# randoms drawn from the same selection.  Columns only: positions, the
# selection's expected density `nbar`, completeness weights.
# ----------------------------------------------------------------------

def radial_selection(r, r_min: float, r_max: float):
    """Selection probability of a survey shell: a smooth bump peaking at the
    shell's middle, zero outside [r_min, r_max]."""
    r = np.asarray(r, dtype=np.float64)
    mid, half = 0.5 * (r_min + r_max), 0.5 * (r_max - r_min)
    s = np.exp(-((r - mid) / (0.6 * half)) ** 2)
    return np.where((r >= r_min) & (r <= r_max), s, 0.0)


def _thin_to_shell(pos: np.ndarray, r_min: float, r_max: float, rng, n_keep: int):
    """Keep objects with probability radial_selection(|x|), the first n_keep."""
    r = np.sqrt(np.sum(pos * pos, axis=1))
    keep = rng.random(len(pos)) < radial_selection(r, r_min, r_max)
    out = pos[keep]
    return out[:n_keep]


def survey_catalogs(n_data: int, n_randoms: int, extent: float, seed: int, ngrid: int = 64,
                    clustered: bool = True, device="cpu") -> dict:
    """Data and randoms of a synthetic survey in observer-frame Cartesian
    coordinates (Mpc/h): the octant x, y, z in [0, extent) with radii in
    [0.2, 0.95] extent and the radial_selection bump.  Data: a log-normal
    catalog (no RSD) of the cube, thinned by the selection (clustered=False:
    uniform instead); randoms: uniform in the cube, thinned the same way.
    Returns float64 numpy arrays: data / randoms (n, 3), their nbar (the
    expected data density n0 sel(r) with n0 the cube's density before
    thinning), data completeness weights in [0.8, 1.2], and the radii."""
    rng = np.random.default_rng(seed)
    r_min, r_max = 0.2 * extent, 0.95 * extent
    probe = rng.random((200000, 3)) * extent
    eff = float(np.mean(radial_selection(np.sqrt(np.sum(probe * probe, axis=1)), r_min, r_max)))
    n_gen_d = int(math.ceil(1.15 * n_data / eff)) + 1000
    n_gen_r = int(math.ceil(1.15 * n_randoms / eff)) + 1000
    if clustered:
        d = lognormal_catalog(n_gen_d, extent, ngrid, seed, f_rsd=0.0, device=device,
                              dtype=torch.float64).cpu().numpy()
    else:
        d = rng.random((n_gen_d, 3)) * extent
    data = _thin_to_shell(d, r_min, r_max, rng, n_data)
    rand = _thin_to_shell(rng.random((n_gen_r, 3)) * extent, r_min, r_max, rng, n_randoms)
    n0 = n_gen_d / extent ** 3
    nbar = lambda p: n0 * radial_selection(np.sqrt(np.sum(p * p, axis=1)), r_min, r_max)
    return {"data": data, "randoms": rand, "data_nbar": nbar(data), "rand_nbar": nbar(rand),
            "data_wcomp": rng.uniform(0.8, 1.2, len(data)), "extent": extent,
            "r_min": r_min, "r_max": r_max}


def survey_sky(n: int, seed: int, ra=(10.0, 80.0), dec=(5.0, 55.0), z=(0.15, 0.7)) -> dict:
    """Sky coordinates of n objects: RA uniform (degrees), uniform on the
    sphere in Dec (sin Dec uniform), redshift with density growing as z^2
    over the range; plus a stand-in n(z) column (a smooth positive function
    of z, 1e-4 to 4e-4) and completeness weights in [0.8, 1.2]."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(ra[0], ra[1], n)
    s0, s1 = math.sin(math.radians(dec[0])), math.sin(math.radians(dec[1]))
    d = np.degrees(np.arcsin(rng.uniform(s0, s1, n)))
    zz = (rng.uniform(z[0] ** 3, z[1] ** 3, n)) ** (1.0 / 3.0)
    nz = 1e-4 * (2.5 + 1.5 * np.cos(2 * math.pi * (zz - z[0]) / (z[1] - z[0])))
    return {"ra": r, "dec": d, "z": zz, "nbar": nz, "wcomp": rng.uniform(0.8, 1.2, n)}
