"""GB300 FFT power-spectrum path: Python binding of ``libpk.so``.

The estimator is nbodykit's FFTPower (Hand, Feng et al., arXiv:1712.05834):
paint a catalog onto a mesh with a CIC / TSC / PCS window, optionally
interlaced (Sec. 3.3.1-3.3.2), r2c FFT, window compensation
(Eq. window-deconvolution), and |delta(k)|^2 binned in k, (k, mu) and Legendre
multipoles (Sec. 3.4.1).  Every step runs in the CUDA kernels of ``libpk.so``;
this module only marshals arguments to the C ABI declared in
``include/pk.h`` and keeps its names: ``pk_plan``, ``pk_paint``,
``pk_paint_many``, ``pk_compute``, ``pk_result``, ``pk_mesh``, ``pk_destroy``.

The survey multipoles of ConvolvedFFTPower (Sec. 3.4.1) use the same library
through ``pk_survey_plan``, ``pk_survey_paint``, ``pk_survey_compute``,
``pk_survey_result`` (and ``pk_survey_bounds`` / ``survey_box`` to choose the
mesh box), e.g.::

    lo, hi = pk_survey_bounds(survey_catalog(randoms_radecz, "sky", nbar=nz_r))
    L, origin = survey_box(lo, hi, pad=0.02)
    with ConvolvedFFTPower(make_survey_config(L, origin, 512, "tsc", True)) as cp:
        res = cp.run(survey_catalog(data_radecz, "sky", wcomp=wc, nbar=nz_d),
                     survey_catalog(randoms_radecz, "sky", nbar=nz_r))
    res["poles"]      # P_0, P_2, P_4 per k bin

There is no fallback: if the library is missing or no GPU is present the calls
raise.  ``build()`` compiles the library in-tree (nvcc, sm_103a).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from .build import LIB as LIB_PATH
from .build import build

__all__ = [
    "PK_CIC", "PK_TSC", "PK_PCS", "PK_F32", "PK_F64", "PK_F32X4", "PK_MESH_F32", "PK_MESH_F64",
    "PK_PAINT_SORT", "PK_PAINT_ATOMIC",
    "PkError", "pk_config", "pk_config_default", "make_config", "pk_plan", "pk_paint",
    "pk_paint_many", "pk_compute", "pk_result", "pk_mesh", "pk_destroy", "pk_status_string",
    "pk_last_error", "pk_enable_timing", "pk_stage_times", "pk_launch_count", "pk_use_own_fft", "FFTPower", "load",
    "build", "make_survey_config", "survey_catalog", "pk_survey_plan", "pk_survey_paint", "pk_survey_compute",
    "pk_survey_result", "pk_survey_ylm", "pk_survey_destroy", "ConvolvedFFTPower", "pk_survey_bounds",
    "survey_box",
]

PK_OK, PK_EINVAL, PK_ENOMEM, PK_ECUDA, PK_ECUFFT, PK_EOVERFLOW, PK_ETIMEOUT, PK_ESTATE = range(8)
PK_CIC, PK_TSC, PK_PCS = 2, 3, 4
PK_F32, PK_F64, PK_F32X4 = 0, 1, 2
PK_MESH_F32, PK_MESH_F64 = 0, 1
PK_PAINT_SORT, PK_PAINT_ATOMIC = 0, 1
VARIANTS = {"sort": PK_PAINT_SORT, "atomic": PK_PAINT_ATOMIC}
WINDOWS = {"cic": PK_CIC, "tsc": PK_TSC, "pcs": PK_PCS}
EXPORTED = ["pk_config_default", "pk_plan", "pk_paint", "pk_paint_many", "pk_compute",
            "pk_result", "pk_mesh", "pk_destroy", "pk_status_string", "pk_last_error",
            "pk_plan_error", "pk_enable_timing", "pk_stage_times", "pk_launch_count", "pk_use_own_fft",
            "pk_bin_static", "pk_cross", "pk_cross_result", "pk_paint_values", "pk_projected", "pk_lognormal_plan", "pk_lognormal_field", "pk_lognormal_draw",
            "pk_lognormal_amp", "pk_lognormal_launch_count", "pk_lognormal_error", "pk_lognormal_destroy",
            "pk_survey_config_default", "pk_survey_plan", "pk_survey_paint", "pk_survey_compute",
            "pk_survey_result", "pk_survey_ylm", "pk_survey_launch_count", "pk_survey_error",
            "pk_survey_destroy", "pk_survey_enable_timing", "pk_survey_stage_times", "pk_survey_bounds"]
STAGES = ["sort", "paint", "fft", "bin", "final"]


class pk_config(ctypes.Structure):
    _fields_ = [
        ("box_size", ctypes.c_double), ("nmesh", ctypes.c_int), ("window", ctypes.c_int),
        ("interlaced", ctypes.c_int), ("compensated", ctypes.c_int), ("kmin", ctypes.c_double),
        ("kmax", ctypes.c_double), ("dk", ctypes.c_double), ("nmu", ctypes.c_int),
        ("poles_mask", ctypes.c_uint), ("los_axis", ctypes.c_int), ("precision", ctypes.c_int),
        ("subtract_shot", ctypes.c_int), ("fixed_scale_log2", ctypes.c_int), ("batch", ctypes.c_int),
        ("tile", ctypes.c_int), ("paint_variant", ctypes.c_int), ("capacity", ctypes.c_int64),
    ]


class pk_survey_config(ctypes.Structure):
    _fields_ = [
        ("box_size", ctypes.c_double), ("box_origin", ctypes.c_double * 3), ("nmesh", ctypes.c_int),
        ("window", ctypes.c_int), ("interlaced", ctypes.c_int), ("compensated", ctypes.c_int),
        ("kmin", ctypes.c_double), ("kmax", ctypes.c_double), ("dk", ctypes.c_double),
        ("poles_mask", ctypes.c_uint), ("precision", ctypes.c_int), ("subtract_shot", ctypes.c_int),
        ("omega_m", ctypes.c_double), ("zmax", ctypes.c_double), ("p0_fkp", ctypes.c_double),
        ("max_batch", ctypes.c_int), ("capacity", ctypes.c_int64),
    ]


class pk_survey_catalog(ctypes.Structure):
    _fields_ = [
        ("pos", ctypes.c_void_p), ("dtype", ctypes.c_int), ("coord", ctypes.c_int),
        ("wcomp", ctypes.c_void_p), ("wfkp", ctypes.c_void_p), ("nbar", ctypes.c_void_p),
        ("n", ctypes.c_int64),
    ]


class pk_lognormal_config(ctypes.Structure):
    _fields_ = [
        ("box_size", ctypes.c_double), ("ngrid", ctypes.c_int), ("slope", ctypes.c_double),
        ("amp", ctypes.c_double), ("variance", ctypes.c_double), ("f_rsd", ctypes.c_double),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_up = ctypes.POINTER(ctypes.c_uint64)


class pk_result_view(ctypes.Structure):
    _fields_ = [
        ("nk", ctypes.c_int), ("nmu", ctypes.c_int), ("npoles", ctypes.c_int),
        ("k_edges", _dp), ("mu_edges", _dp), ("k_mean", _dp), ("pk", _dp), ("poles", _dp),
        ("modes", _up), ("k_mean2d", _dp), ("mu_mean2d", _dp), ("pkmu", _dp), ("modes2d", _up),
        ("shot_noise", ctypes.c_double), ("wsum", ctypes.c_double), ("w2sum", ctypes.c_double),
    ]


class pk_projected_view(ctypes.Structure):
    _fields_ = [
        ("nk", ctypes.c_int), ("ndim", ctypes.c_int), ("k_edges", _dp), ("k_mean", _dp), ("pk", _dp),
        ("modes", _up), ("shot_noise", ctypes.c_double), ("wsum", ctypes.c_double),
    ]


class pk_survey_result_view(ctypes.Structure):
    _fields_ = [
        ("nk", ctypes.c_int), ("npoles", ctypes.c_int), ("k_edges", _dp), ("k_mean", _dp), ("poles", _dp),
        ("modes", _up), ("alpha", ctypes.c_double), ("norm", ctypes.c_double), ("shot_noise", ctypes.c_double),
        ("data_wsum", ctypes.c_double), ("randoms_wsum", ctypes.c_double), ("data_w2sum", ctypes.c_double),
        ("randoms_w2sum", ctypes.c_double), ("randoms_nsum", ctypes.c_double), ("n_data", ctypes.c_int64),
        ("n_randoms", ctypes.c_int64), ("n_outside", ctypes.c_int64), ("n_rejected", ctypes.c_int64),
    ]


class PkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (pk_status_string(status), msg))
        self.status = status


_lib = None


def load():
    """Load libpk.so (built by ``build()``); raises if it is not there."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpk.so is not built: call paper_1712_05834_gb300.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.pk_config_default.argtypes = [ctypes.POINTER(pk_config)]
        lib.pk_config_default.restype = None
        lib.pk_plan.argtypes = [ctypes.POINTER(pk_config), vp, ctypes.POINTER(vp)]
        lib.pk_plan.restype = i
        lib.pk_paint.argtypes = [vp, vp, i, vp, i64, i]
        lib.pk_paint.restype = i
        lib.pk_paint_many.argtypes = [vp, vp, i, vp, ctypes.POINTER(ctypes.c_int64), i]
        lib.pk_paint_many.restype = i
        lib.pk_paint_values.argtypes = [vp, vp, i, vp, vp, ctypes.POINTER(ctypes.c_int64), i]
        lib.pk_paint_values.restype = i
        lib.pk_compute.argtypes = [vp]
        lib.pk_compute.restype = i
        lib.pk_result.argtypes = [vp, i, ctypes.POINTER(pk_result_view)]
        lib.pk_result.restype = i
        lib.pk_cross.argtypes = [vp, i, i]
        lib.pk_cross.restype = i
        lib.pk_cross_result.argtypes = [vp, ctypes.POINTER(pk_result_view)]
        lib.pk_cross_result.restype = i
        lib.pk_projected.argtypes = [vp, i, ctypes.c_uint, ctypes.POINTER(pk_projected_view)]
        lib.pk_projected.restype = i
        lib.pk_mesh.argtypes = [vp, i, i, vp]
        lib.pk_mesh.restype = i
        lib.pk_destroy.argtypes = [vp]
        lib.pk_destroy.restype = i
        lib.pk_status_string.argtypes = [i]
        lib.pk_status_string.restype = ctypes.c_char_p
        lib.pk_last_error.argtypes = [vp]
        lib.pk_last_error.restype = ctypes.c_char_p
        lib.pk_plan_error.argtypes = []
        lib.pk_plan_error.restype = ctypes.c_char_p
        lib.pk_enable_timing.argtypes = [vp, i]
        lib.pk_enable_timing.restype = i
        lib.pk_use_own_fft.argtypes = [vp, i]
        lib.pk_use_own_fft.restype = i
        lib.pk_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.pk_stage_times.restype = i
        lib.pk_launch_count.argtypes = [vp]
        lib.pk_launch_count.restype = ctypes.c_longlong
        lib.pk_bin_static.argtypes = [ctypes.POINTER(pk_config), vp, vp, vp, vp, ctypes.c_char_p, ctypes.c_size_t]
        lib.pk_bin_static.restype = i
        lib.pk_lognormal_plan.argtypes = [ctypes.POINTER(pk_lognormal_config), vp, ctypes.POINTER(vp)]
        lib.pk_lognormal_plan.restype = i
        lib.pk_lognormal_field.argtypes = [vp, ctypes.c_uint64, vp]
        lib.pk_lognormal_field.restype = i
        lib.pk_lognormal_draw.argtypes = [vp, ctypes.c_uint64, i64, vp]
        lib.pk_lognormal_draw.restype = i
        lib.pk_lognormal_amp.argtypes = [vp]
        lib.pk_lognormal_amp.restype = ctypes.c_double
        lib.pk_lognormal_launch_count.argtypes = [vp]
        lib.pk_lognormal_launch_count.restype = ctypes.c_longlong
        lib.pk_lognormal_error.argtypes = [vp]
        lib.pk_lognormal_error.restype = ctypes.c_char_p
        lib.pk_lognormal_destroy.argtypes = [vp]
        lib.pk_lognormal_destroy.restype = i
        lib.pk_survey_config_default.argtypes = [ctypes.POINTER(pk_survey_config)]
        lib.pk_survey_config_default.restype = None
        lib.pk_survey_plan.argtypes = [ctypes.POINTER(pk_survey_config), vp, ctypes.POINTER(vp)]
        lib.pk_survey_plan.restype = i
        lib.pk_survey_paint.argtypes = [vp, ctypes.POINTER(pk_survey_catalog), ctypes.POINTER(pk_survey_catalog)]
        lib.pk_survey_paint.restype = i
        lib.pk_survey_compute.argtypes = [vp]
        lib.pk_survey_compute.restype = i
        lib.pk_survey_result.argtypes = [vp, ctypes.POINTER(pk_survey_result_view)]
        lib.pk_survey_result.restype = i
        lib.pk_survey_ylm.argtypes = [i, i, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.pk_survey_ylm.restype = ctypes.c_double
        lib.pk_survey_launch_count.argtypes = [vp]
        lib.pk_survey_launch_count.restype = ctypes.c_longlong
        lib.pk_survey_error.argtypes = [vp]
        lib.pk_survey_error.restype = ctypes.c_char_p
        lib.pk_survey_bounds.argtypes = [ctypes.POINTER(pk_survey_catalog), ctypes.c_double, ctypes.c_double, vp,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.pk_survey_bounds.restype = i
        lib.pk_survey_enable_timing.argtypes = [vp, i]
        lib.pk_survey_enable_timing.restype = i
        lib.pk_survey_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.pk_survey_stage_times.restype = i
        lib.pk_survey_destroy.argtypes = [vp]
        lib.pk_survey_destroy.restype = i
        _lib = lib
    return _lib


def pk_status_string(status: int) -> str:
    return load().pk_status_string(int(status)).decode()


def pk_last_error(plan) -> str:
    return load().pk_last_error(plan).decode()


def _check(status, plan=None):
    if status != PK_OK:
        msg = load().pk_plan_error().decode() if plan is None else pk_last_error(plan)
        raise PkError(status, msg)


def pk_config_default() -> pk_config:
    c = pk_config()
    load().pk_config_default(ctypes.byref(c))
    return c


def make_config(box_size, nmesh, window="cic", interlaced=False, compensated=True, dk=None,
                kmin=0.0, kmax=None, nmu=0, poles=(0, 2, 4), precision="f32",
                subtract_shot=True, fixed_scale_log2=0, batch=1, tile=0, paint_variant="sort",
                capacity=0) -> pk_config:
    """pk_config from keyword arguments that follow the paper's ``to_mesh`` /
    ``FFTPower`` options (Sec. 3.3.2, Sec. 3.4.1).  dk defaults to 2 kF.
    ``paint_variant`` ("sort" / "atomic"), ``tile`` and ``capacity`` (objects
    reserved at plan time) only change speed and allocation, not results."""
    c = pk_config_default()
    c.box_size = float(box_size)
    c.nmesh = int(nmesh)
    c.window = WINDOWS[window] if isinstance(window, str) else int(window)
    c.interlaced = int(bool(interlaced))
    c.compensated = int(bool(compensated))
    c.kmin = float(kmin)
    c.kmax = 0.0 if kmax is None else float(kmax)
    c.dk = float(dk) if dk is not None else 2.0 * (2.0 * math.pi) / float(box_size)
    c.nmu = int(nmu)
    c.poles_mask = sum({0: 1, 2: 2, 4: 4}[ell] for ell in poles)
    c.los_axis = 2
    c.precision = {"f32": PK_MESH_F32, "f64": PK_MESH_F64}[precision] if isinstance(precision, str) else int(precision)
    c.subtract_shot = int(bool(subtract_shot))
    c.fixed_scale_log2 = int(fixed_scale_log2)
    c.batch = int(batch)
    c.tile = int(tile)
    c.paint_variant = VARIANTS[paint_variant] if isinstance(paint_variant, str) else int(paint_variant)
    c.capacity = int(capacity)
    return c


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def pk_plan(cfg: pk_config, stream=None):
    """Create a plan (device = the current CUDA device).  ``stream`` is a
    torch.cuda.Stream, a raw cudaStream_t integer, or None (default stream)."""
    h = ctypes.c_void_p()
    _check(load().pk_plan(ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(h)))
    return h


def _array_info(a):
    """(pointer, dtype code, n) of a position array: torch tensor or numpy array."""
    shape = tuple(a.shape)
    if len(shape) != 2 or shape[1] not in (3, 4):
        raise ValueError("positions must have shape (n, 3) or (n, 4)")
    if hasattr(a, "data_ptr"):                      # torch tensor
        if not a.is_contiguous():
            raise ValueError("positions must be contiguous")
        name = str(a.dtype)
        ptr = a.data_ptr()
    else:
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("positions must be C-contiguous")
        name = str(a.dtype)
        ptr = a.ctypes.data
    if shape[1] == 4:
        if "float32" not in name:
            raise ValueError("(n, 4) positions must be float32 xyzw")
        return ptr, PK_F32X4, shape[0]
    if "float32" in name:
        return ptr, PK_F32, shape[0]
    if "float64" in name:
        return ptr, PK_F64, shape[0]
    raise ValueError("positions must be float32 or float64")


def _weights_ptr(w, n):
    if w is None:
        return None
    if tuple(w.shape) != (n,):
        raise ValueError("weights must have shape (n,)")
    if hasattr(w, "data_ptr"):
        if str(w.dtype) != "torch.float32" or not w.is_contiguous():
            raise ValueError("weights must be contiguous float32")
        return w.data_ptr()
    if w.dtype != np.float32 or not w.flags["C_CONTIGUOUS"]:
        raise ValueError("weights must be contiguous float32")
    return w.ctypes.data


def pk_paint(plan, pos, weights=None, accumulate=False):
    """Paint one catalog (device or host array) onto the plan's mesh(es)."""
    ptr, code, n = _array_info(pos)
    _check(load().pk_paint(plan, ptr, code, _weights_ptr(weights, n), n, int(bool(accumulate))), plan)


def pk_paint_many(plan, pos, offsets, weights=None):
    """Paint catalogs stored back to back; offsets has nitems + 1 entries."""
    ptr, code, n = _array_info(pos)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if off[-1] != n:
        raise ValueError("offsets[-1] must equal the number of objects")
    _check(load().pk_paint_many(plan, ptr, code, _weights_ptr(weights, n),
                                off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(off) - 1), plan)


def pk_paint_values(plan, pos, values, offsets=None, weights=None):
    """Paint the field value V of every object (e.g. a velocity component:
    the momentum field); normalization by sum W, deposits W V."""
    ptr, code, n = _array_info(pos)
    off = np.ascontiguousarray(np.asarray([0, n] if offsets is None else offsets, dtype=np.int64))
    if off[-1] != n:
        raise ValueError("offsets[-1] must equal the number of objects")
    _check(load().pk_paint_values(plan, ptr, code, _weights_ptr(weights, n), _weights_ptr(values, n),
                                  off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(off) - 1), plan)


def pk_compute(plan):
    _check(load().pk_compute(plan), plan)


def _arr(ptr, n, dtype=np.float64):
    if not ptr or n == 0:
        return None
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def _view_dict(v) -> dict:
    nk, nmu = v.nk, v.nmu
    out = {
        "nk": nk, "nmu": nmu,
        "k_edges": _arr(v.k_edges, nk + 1),
        "k": _arr(v.k_mean, nk),
        "power": _arr(v.pk, nk),
        "poles": _arr(v.poles, 3 * nk).reshape(3, nk),
        "modes": _arr(v.modes, nk, np.int64),
        "shot_noise": v.shot_noise, "wsum": v.wsum, "w2sum": v.w2sum,
    }
    if nmu > 0:
        out["mu_edges"] = _arr(v.mu_edges, nmu + 1)
        out["k2d"] = _arr(v.k_mean2d, nk * nmu).reshape(nk, nmu)
        out["mu2d"] = _arr(v.mu_mean2d, nk * nmu).reshape(nk, nmu)
        out["power2d"] = _arr(v.pkmu, nk * nmu).reshape(nk, nmu)
        out["modes2d"] = _arr(v.modes2d, nk * nmu, np.int64).reshape(nk, nmu)
    return out


def pk_result(plan, item=0) -> dict:
    """Result of catalog ``item`` of the last compute, copied into numpy arrays."""
    v = pk_result_view()
    _check(load().pk_result(plan, int(item), ctypes.byref(v)), plan)
    return _view_dict(v)


def pk_cross(plan, item_a, item_b) -> dict:
    """Cross power of two catalogs of the last compute (no shot noise), as a
    dict like pk_result's (wsum: catalog a's sum of weights, w2sum: b's)."""
    _check(load().pk_cross(plan, int(item_a), int(item_b)), plan)
    v = pk_result_view()
    _check(load().pk_cross_result(plan, ctypes.byref(v)), plan)
    return _view_dict(v)


AXES = {"x": 1, "y": 2, "z": 4}


def pk_projected(plan, item=0, axes=(0, 1)) -> dict:
    """Power of catalog ``item`` projected onto ``axes`` (indices 0-2 or
    names "x", "y", "z"; one or two axes), after pk_compute."""
    mask = 0
    for a in axes:
        mask |= AXES[a] if isinstance(a, str) else (1 << int(a))
    v = pk_projected_view()
    _check(load().pk_projected(plan, int(item), mask, ctypes.byref(v)), plan)
    return {"nk": v.nk, "ndim": v.ndim, "k_edges": _arr(v.k_edges, v.nk + 1), "k": _arr(v.k_mean, v.nk),
            "power": _arr(v.pk, v.nk), "modes": _arr(v.modes, v.nk, np.int64), "shot_noise": v.shot_noise,
            "wsum": v.wsum}


def pk_mesh(plan, item, mesh, nmesh, f64=False):
    """Dense (N, N, N) numpy copy of a painted mesh (before pk_compute)."""
    out = np.empty((nmesh, nmesh, nmesh), dtype=np.float64 if f64 else np.float32)
    _check(load().pk_mesh(plan, int(item), int(mesh), out.ctypes.data), plan)
    return out


def pk_enable_timing(plan, on=True):
    _check(load().pk_enable_timing(plan, int(bool(on))), plan)


def pk_use_own_fft(plan, on=True):
    """Select the r2c transform of the next pk_compute: the library's own FFT
    kernels (y and x passes, then z fused into the bin pass) or cuFFT's R2C."""
    _check(load().pk_use_own_fft(plan, int(bool(on))), plan)


def pk_stage_times(plan) -> dict:
    """Device ms per stage of the last timed pk_paint / pk_compute."""
    ms = (ctypes.c_double * len(STAGES))()
    _check(load().pk_stage_times(plan, ms), plan)
    return dict(zip(STAGES, list(ms)))


def pk_launch_count(plan) -> int:
    return int(load().pk_launch_count(plan))


def pk_destroy(plan):
    if plan:
        _check(load().pk_destroy(plan))


class FFTPower:
    """Plan-owning convenience wrapper: ``FFTPower(cfg).run(pos, weights)``."""

    def __init__(self, cfg: pk_config, stream=None):
        self.cfg = cfg
        self.plan = pk_plan(cfg, stream)

    def run(self, pos, weights=None):
        pk_paint(self.plan, pos, weights)
        pk_compute(self.plan)
        return pk_result(self.plan, 0)

    def close(self):
        if self.plan:
            pk_destroy(self.plan)
            self.plan = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- log-normal mock catalogs on the device (pk_lognormal_*) ----

def _check_ln(status, gen):
    if status != PK_OK:
        raise PkError(status, load().pk_lognormal_error(gen).decode())


def pk_lognormal_plan(box_size, ngrid, slope=-1.5, amp=0.0, variance=1.0, f_rsd=0.75, stream=None):
    """Generator of log-normal catalogs on an ngrid^3 field (see include/pk.h)."""
    c = pk_lognormal_config(float(box_size), int(ngrid), float(slope), float(amp or 0.0), float(variance),
                            float(f_rsd))
    h = ctypes.c_void_p()
    _check(load().pk_lognormal_plan(ctypes.byref(c), _stream_ptr(stream), ctypes.byref(h)))
    return h


def pk_lognormal_field(gen, seed, out):
    """The Gaussian linear field of `seed` into `out` (torch tensor or numpy
    array of ngrid^3 float32, device or host)."""
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    _check_ln(load().pk_lognormal_field(gen, int(seed), ptr), gen)


def pk_lognormal_draw(gen, seed, n, out):
    """Draw n objects of `seed` into `out`, a contiguous (>= n, 3) float32 device tensor."""
    if tuple(out.shape[1:]) != (3,) or out.shape[0] < n or str(out.dtype) != "torch.float32" \
            or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous (>= n, 3) float32 CUDA tensor")
    _check_ln(load().pk_lognormal_draw(gen, int(seed), int(n), out.data_ptr()), gen)


def pk_lognormal_amp(gen) -> float:
    return float(load().pk_lognormal_amp(gen))


def pk_lognormal_destroy(gen):
    if gen:
        _check(load().pk_lognormal_destroy(gen))


class LogNormalCatalog:
    """Device-resident log-normal mocks (the paper's LogNormalCatalog source):
    ``LogNormalCatalog(L, ngrid).draw(seed, n)`` returns an (n, 3) float32 CUDA
    tensor of positions in [0, L), generated wholly by the library's kernels."""

    def __init__(self, box_size, ngrid, slope=-1.5, amp=0.0, variance=1.0, f_rsd=0.75, stream=None):
        import torch
        self.torch = torch
        self.box_size, self.ngrid = float(box_size), int(ngrid)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.gen = pk_lognormal_plan(box_size, ngrid, slope, amp, variance, f_rsd, self.stream)

    @property
    def amp(self) -> float:
        return pk_lognormal_amp(self.gen)

    def draw(self, seed, n, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty((int(n), 3), dtype=torch.float32, device="cuda")
        pk_lognormal_draw(self.gen, seed, n, out)
        return out[: int(n)]

    def field(self, seed):
        torch = self.torch
        out = torch.empty((self.ngrid,) * 3, dtype=torch.float32, device="cuda")
        pk_lognormal_field(self.gen, seed, out)
        return out

    def close(self):
        if self.gen:
            pk_lognormal_destroy(self.gen)
            self.gen = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- survey multipoles (pk_survey_*: the ConvolvedFFTPower of Sec. 3.4.1) ----

PK_COORD_CARTESIAN, PK_COORD_SKY = 0, 1


def _check_sv(status, plan):
    if status != PK_OK:
        raise PkError(status, load().pk_survey_error(plan).decode())


def make_survey_config(box_size, box_origin, nmesh, window="cic", interlaced=False, compensated=True, dk=None,
                       kmin=0.0, kmax=None, poles=(0, 2, 4), precision="f32", subtract_shot=True, omega_m=0.31,
                       zmax=5.0, p0_fkp=0.0, max_batch=0, capacity=0) -> pk_survey_config:
    """pk_survey_config from keywords (the ConvolvedFFTPower options: mesh,
    window, interlacing, k bins, poles, FKP P0; omega_m for sky input)."""
    c = pk_survey_config()
    load().pk_survey_config_default(ctypes.byref(c))
    c.box_size = float(box_size)
    for a in range(3):
        c.box_origin[a] = float(box_origin[a])
    c.nmesh = int(nmesh)
    c.window = WINDOWS[window] if isinstance(window, str) else int(window)
    c.interlaced = int(bool(interlaced))
    c.compensated = int(bool(compensated))
    c.dk = float(dk) if dk is not None else 2.0 * (2.0 * math.pi) / float(box_size)
    c.kmin = float(kmin)
    c.kmax = 0.0 if kmax is None else float(kmax)
    c.poles_mask = sum({0: 1, 2: 2, 4: 4}[ell] for ell in poles) | 1
    c.precision = {"f32": PK_MESH_F32, "f64": PK_MESH_F64}[precision] if isinstance(precision, str) else int(precision)
    c.subtract_shot = int(bool(subtract_shot))
    c.omega_m = float(omega_m)
    c.zmax = float(zmax)
    c.p0_fkp = float(p0_fkp)
    c.max_batch = int(max_batch)
    c.capacity = int(capacity)
    return c


def pk_survey_plan(cfg: pk_survey_config, stream=None):
    h = ctypes.c_void_p()
    _check(load().pk_survey_plan(ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(h)))
    return h


def _ptr_f32(a, n, name):
    if a is None:
        return None
    if tuple(a.shape) != (n,):
        raise ValueError("%s must have shape (n,)" % name)
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != "torch.float32" or not a.is_contiguous():
            raise ValueError("%s must be contiguous float32" % name)
        return a.data_ptr()
    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("%s must be contiguous float32" % name)
    return a.ctypes.data


def survey_catalog(pos, coord="cartesian", wcomp=None, wfkp=None, nbar=None) -> pk_survey_catalog:
    """pk_survey_catalog of an (n, 3) float32/float64 array (torch or numpy,
    device or host): x, y, z (coord "cartesian") or RA, Dec, z ("sky")."""
    ptr, code, n = _array_info(pos)
    if code == PK_F32X4:
        raise ValueError("survey positions must have shape (n, 3)")
    cat = pk_survey_catalog(ptr, code, {"cartesian": PK_COORD_CARTESIAN, "sky": PK_COORD_SKY}[coord],
                            _ptr_f32(wcomp, n, "wcomp"), _ptr_f32(wfkp, n, "wfkp"), _ptr_f32(nbar, n, "nbar"), n)
    cat._arrays = (pos, wcomp, wfkp, nbar)      # the struct holds raw pointers: keep the arrays alive
    return cat


def pk_survey_paint(plan, data: pk_survey_catalog, randoms: pk_survey_catalog | None = None):
    """Paint the data and (unless None: keep the last ones) the randoms."""
    _check_sv(load().pk_survey_paint(plan, ctypes.byref(data), None if randoms is None else ctypes.byref(randoms)),
              plan)


def pk_survey_compute(plan):
    _check_sv(load().pk_survey_compute(plan), plan)


def pk_survey_result(plan) -> dict:
    v = pk_survey_result_view()
    _check_sv(load().pk_survey_result(plan, ctypes.byref(v)), plan)
    nk = v.nk
    return {"nk": nk, "k_edges": _arr(v.k_edges, nk + 1), "k": _arr(v.k_mean, nk),
            "poles": _arr(v.poles, 3 * nk).reshape(3, nk), "modes": _arr(v.modes, nk, np.int64),
            "alpha": v.alpha, "norm": v.norm, "shot_noise": v.shot_noise, "data_wsum": v.data_wsum,
            "randoms_wsum": v.randoms_wsum, "data_w2sum": v.data_w2sum, "randoms_w2sum": v.randoms_w2sum,
            "randoms_nsum": v.randoms_nsum, "n_data": v.n_data, "n_randoms": v.n_randoms,
            "n_outside": v.n_outside, "n_rejected": v.n_rejected}


def pk_survey_ylm(l, m, x, y, z) -> float:
    return float(load().pk_survey_ylm(int(l), int(m), float(x), float(y), float(z)))


def pk_survey_bounds(cat: pk_survey_catalog, omega_m=0.31, zmax=5.0, stream=None):
    """Per-axis (min, max) of a catalog's observer-frame Cartesian positions
    (sky input converted on the device as the survey paint converts it)."""
    lo = (ctypes.c_double * 3)()
    hi = (ctypes.c_double * 3)()
    status = load().pk_survey_bounds(ctypes.byref(cat), float(omega_m), float(zmax), _stream_ptr(stream), lo, hi)
    _check(status)
    return np.array(list(lo)), np.array(list(hi))


def survey_box(lo, hi, pad=0.02):
    """Cubic mesh box enclosing [lo, hi]: edge (1 + pad) times the largest
    extent, centred on the middle of the range.  Returns (box_size, origin)."""
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    size = float(np.max(hi - lo)) * (1.0 + float(pad))
    if not size > 0.0:
        raise ValueError("empty or degenerate range")
    origin = 0.5 * (lo + hi) - 0.5 * size
    return size, tuple(float(v) for v in origin)


SURVEY_STAGES = ["prep", "paint", "fft", "field", "bin", "final"]


def pk_survey_enable_timing(plan, on=True):
    _check_sv(load().pk_survey_enable_timing(plan, int(bool(on))), plan)


def pk_survey_stage_times(plan) -> dict:
    """Device ms per stage of the last timed pk_survey_paint / pk_survey_compute."""
    ms = (ctypes.c_double * len(SURVEY_STAGES))()
    _check_sv(load().pk_survey_stage_times(plan, ms), plan)
    return dict(zip(SURVEY_STAGES, list(ms)))


def pk_survey_launch_count(plan) -> int:
    return int(load().pk_survey_launch_count(plan))


def pk_survey_destroy(plan):
    if plan:
        _check(load().pk_survey_destroy(plan))


class ConvolvedFFTPower:
    """Survey multipoles: ``ConvolvedFFTPower(cfg).run(data, randoms)`` with
    catalogs made by ``survey_catalog``; randoms=None reuses the last ones."""

    def __init__(self, cfg: pk_survey_config, stream=None):
        self.cfg = cfg
        self.plan = pk_survey_plan(cfg, stream)

    def run(self, data, randoms=None):
        pk_survey_paint(self.plan, data, randoms)
        pk_survey_compute(self.plan)
        return pk_survey_result(self.plan)

    def close(self):
        if self.plan:
            pk_survey_destroy(self.plan)
            self.plan = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
