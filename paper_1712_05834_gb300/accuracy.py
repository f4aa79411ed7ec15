"""Window and interlacing accuracy study (Sec. 3.3.2 and its comparison of
interlaced CIC / TSC / PCS painting against a finer reference mesh).

One catalog is painted on a coarse mesh with each window, with and without
interlacing, always compensated by Eq. window-deconvolution, and on a mesh
twice as fine with PCS + interlacing (the reference).  Both use the same k
bins up to the coarse mesh's Nyquist wavenumber k_N, where the two meshes hold
exactly the same Fourier modes, so the ratio P / P_ref of each bin measures
only the aliasing and window errors of the coarse estimate (sample variance
cancels).  Powers are compared before shot-noise subtraction.

Host orchestration only: every evaluation runs through the C ABI.
"""
from __future__ import annotations

import math

import numpy as np

from . import make_config, pk_compute, pk_destroy, pk_paint, pk_plan, pk_result

SCHEMES = [(w, il) for w in ("cic", "tsc", "pcs") for il in (False, True)]


def scheme_name(window: str, interlaced: bool) -> str:
    return window + ("+interlacing" if interlaced else "")


def _raw_power(pos, box_size, nmesh, window, interlaced, dk, kmax, stream, precision="f32"):
    cfg = make_config(box_size, nmesh, window, interlaced=interlaced, dk=dk, kmax=kmax, subtract_shot=False,
                      precision=precision)
    plan = pk_plan(cfg, stream)
    try:
        pk_paint(plan, pos)
        pk_compute(plan)
        return pk_result(plan, 0)
    finally:
        pk_destroy(plan)


def window_study(pos, box_size: float, nmesh: int, ref_nmesh: int | None = None, dk: float | None = None,
                 fractions=(0.5, 0.75, 1.0), stream=None, precision: str = "f32") -> dict:
    """Ratios P / P_ref per k bin for every (window, interlacing) scheme on an
    nmesh^3 mesh against PCS + interlacing on ref_nmesh^3 (default 2 nmesh),
    every spectrum in the given mesh precision ("f32" or "f64").

    Returns k (bin means), k / k_N, the mode counts, the ratio per scheme and
    max |ratio - 1| over the bins with k < f k_N for each f in `fractions`."""
    ref_nmesh = ref_nmesh or 2 * nmesh
    kF = 2.0 * math.pi / box_size
    kN = math.pi * nmesh / box_size
    dk = dk if dk is not None else 2.0 * kF
    nk = int(math.floor(kN / dk))
    kmax = nk * dk                                   # bins [0, kmax) with kmax <= k_N
    ref = _raw_power(pos, box_size, ref_nmesh, "pcs", True, dk, kmax, stream, precision)
    ok = ref["modes"] > 0
    out = {"k": ref["k"][ok], "k_over_kN": ref["k"][ok] / kN, "modes": ref["modes"][ok],
           "nmesh": nmesh, "ref_nmesh": ref_nmesh, "box_size": box_size, "dk": dk,
           "ratio": {}, "max_abs_dev": {}}
    for window, il in SCHEMES:
        r = _raw_power(pos, box_size, nmesh, window, il, dk, kmax, stream, precision)
        if not np.array_equal(r["modes"], ref["modes"]):
            raise RuntimeError("coarse and reference meshes binned different modes")
        ratio = r["power"][ok] / ref["power"][ok]
        name = scheme_name(window, il)
        out["ratio"][name] = ratio
        out["max_abs_dev"][name] = {
            "k<%.2fkN" % f: float(np.max(np.abs(ratio[out["k_over_kN"] < f] - 1.0)))
            for f in fractions}
    return out
