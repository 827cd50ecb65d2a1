"""ctypes binding of the C ABI in include/salt.h (argument marshalling only).

Every computation runs in libsalt_b300.so; this module only builds the C
structs from numpy arrays or torch CUDA tensors and checks status codes. If the
shared library is missing, importing a handle raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsalt_b300.so")

SALT_OK = 0
SALT_PENDING = 1
SALT_ERR_INVALID = -1
SALT_ERR_OOM = -2
SALT_ERR_CUDA = -3
SALT_ERR_TIMEOUT = -4
SALT_ERR_NOT_FOUND = -5
SALT_ERR_CANCELLED = -6
SALT_ERR_DATA = -7

SALT_OPT_KERNEL = 1
SALT_OPT_TILE_SAMPLES = 2
SALT_OPT_GRAPHS = 3
SALT_OPT_SERVE_CHUNK = 4
SALT_OPT_LAST_KERNEL = 5

SALT_KERNEL_AUTO = 0
SALT_KERNEL_DIRECT = 1
SALT_KERNEL_FACTORISED = 2
SALT_KERNEL_BANDWARP = 3
SALT_KERNEL_UNIT = 4

# Every symbol include/salt.h declares (checked by the ABI test).
EXPORTS = [
    "salt_init_model", "salt_destroy", "salt_plan_create", "salt_plan_destroy",
    "salt_bandflux_offsets", "salt_bandflux", "salt_chi2", "salt_chi2_grad", "salt_check",
    "salt_set_option", "salt_get_option", "salt_serve_submit", "salt_serve_poll",
    "salt_serve_cancel", "salt_serve_stats_get", "salt_status_str", "salt_last_error",
    "salt_chi2_grad_noalloc", "salt_fit", "salt_register_band", "salt_band_load", "salt_nested",
    "salt_measure_peaks",
]

# Fitting (salt_fit): parameter bits, outcome codes.
SALT_FIT_Z, SALT_FIT_T0, SALT_FIT_X0, SALT_FIT_X1, SALT_FIT_C = 1, 2, 4, 8, 16
SALT_FIT_DEFAULT_MASK = SALT_FIT_T0 | SALT_FIT_X0 | SALT_FIT_X1 | SALT_FIT_C
SALT_FIT_MAXITER, SALT_FIT_LINESEARCH, SALT_FIT_INVALID, SALT_FIT_FLAT = -1, -2, -3, -4

# Scratch bytes of the no-allocation call (SALT_NOALLOC_SCRATCH_BYTES).
SALT_NOALLOC_SCRATCH_BYTES = 16 << 20


class SaltError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"salt status {code}: {msg}")
        self.code = code


class ModelDesc(C.Structure):
    _fields_ = [("n_phase", C.c_int32), ("n_wave", C.c_int32),
                ("phase0", C.c_double), ("dphase", C.c_double),
                ("wave0", C.c_double), ("dwave", C.c_double),
                ("m0", C.c_void_p), ("m1", C.c_void_p),
                ("n_cl", C.c_int32), ("cl", C.c_void_p),
                ("cl_lo", C.c_double), ("cl_hi", C.c_double),
                ("phase_nodes", C.c_void_p), ("wave_nodes", C.c_void_p)]


class BandDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("wave", C.c_void_p), ("trans", C.c_void_p)]


class BatchDesc(C.Structure):
    _fields_ = [("n_sn", C.c_int64), ("obs_off", C.c_void_p), ("par_off", C.c_void_p),
                ("mjd", C.c_void_p), ("band", C.c_void_p), ("flux", C.c_void_p),
                ("fluxerr", C.c_void_p), ("zp", C.c_void_p), ("t0", C.c_void_p),
                ("z", C.c_void_p), ("x0", C.c_void_p), ("x1", C.c_void_p), ("c", C.c_void_p),
                ("plan", C.c_void_p), ("validate", C.c_int32)]


class FitOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("max_evals", C.c_int32), ("history", C.c_int32),
                ("free_mask", C.c_int32), ("gtol", C.c_double), ("ftol", C.c_double)]


class NestedOpts(C.Structure):
    _fields_ = [("n_live", C.c_int32), ("n_batch", C.c_int32), ("n_steps", C.c_int32),
                ("max_iter", C.c_int32), ("free_mask", C.c_int32), ("reserved", C.c_int32),
                ("seed", C.c_uint64), ("dlogz", C.c_double)]


class Request(C.Structure):
    _fields_ = [("n_obs", C.c_int32), ("n_par", C.c_int32), ("want_grad", C.c_int32),
                ("mjd", C.c_void_p), ("band", C.c_void_p), ("flux", C.c_void_p),
                ("fluxerr", C.c_void_p), ("zp", C.c_void_p), ("t0", C.c_void_p),
                ("z", C.c_void_p), ("x0", C.c_void_p), ("x1", C.c_void_p), ("c", C.c_void_p)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("cancelled", C.c_uint64),
                ("rejected", C.c_uint64), ("launches", C.c_uint64), ("queued", C.c_uint64),
                ("active", C.c_uint64), ("mem_in_use", C.c_size_t), ("mem_limit", C.c_size_t),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


class Peaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("l2_read_gbs", C.c_double), ("smem_read_gbs", C.c_double),
                ("sm_clock_max_mhz", C.c_double), ("num_sms", C.c_int32)]


class ReplayStats(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("submit_s", C.c_double), ("completed", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


class PlainStats(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("completed", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


CLIENT_EXPORTS = ("salt_client_replay", "salt_client_plain")
_client = None


def client():
    """Load libsalt_client.so, the native load generator over the C ABI
    (salt_client.h); raises if it has not been built."""
    global _client
    if _client is not None:
        return _client
    lib()  # the client links the library: load it (and its checks) first
    path = os.path.join(os.path.dirname(LIB_PATH), "libsalt_client.so")
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_2504_08081_b300/build.py")
    L = C.CDLL(path)
    p = C.c_void_p
    L.salt_client_replay.argtypes = [p, p, C.c_int32, p, p, p, p, C.POINTER(ReplayStats)]
    L.salt_client_replay.restype = C.c_int
    L.salt_client_plain.argtypes = [p, p, C.c_int32, C.c_double, C.c_size_t, p, C.POINTER(PlainStats)]
    L.salt_client_plain.restype = C.c_int
    _client = L
    return L


_lib = None


def lib():
    """Load libsalt_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2504_08081_b300/build.py "
                          "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    p, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    L.salt_init_model.argtypes = [C.POINTER(ModelDesc), C.POINTER(BandDesc), i32, i32, C.c_size_t,
                                  C.POINTER(p)]
    L.salt_destroy.argtypes = [p]
    L.salt_destroy.restype = None
    L.salt_plan_create.argtypes = [p, i64, p, p, C.POINTER(p)]
    L.salt_plan_destroy.argtypes = [p]
    L.salt_plan_destroy.restype = None
    L.salt_bandflux_offsets.argtypes = [i64, p, p, p]
    L.salt_bandflux.argtypes = [p, C.POINTER(BatchDesc), p, p]
    L.salt_chi2.argtypes = [p, C.POINTER(BatchDesc), p, p]
    L.salt_chi2_grad.argtypes = [p, C.POINTER(BatchDesc), p, p, p]
    L.salt_chi2_grad_noalloc.argtypes = [p, C.POINTER(BatchDesc), p, p, p]
    L.salt_fit.argtypes = [p, C.POINTER(BatchDesc), p, p, C.POINTER(FitOpts), p, p, p, p]
    L.salt_nested.argtypes = [p, C.POINTER(BatchDesc), p, p, C.POINTER(NestedOpts), p, p, p, p, p, p]
    L.salt_register_band.argtypes = [p, C.POINTER(BandDesc), C.POINTER(i32)]
    L.salt_band_load.argtypes = [p, C.c_char_p, C.c_double, C.c_double, p, p, i32, C.POINTER(i32)]
    L.salt_measure_peaks.argtypes = [p, C.POINTER(Peaks)]
    L.salt_check.argtypes = [p, p]
    L.salt_set_option.argtypes = [p, i32, i64]
    L.salt_get_option.argtypes = [p, i32, C.POINTER(i64)]
    L.salt_serve_submit.argtypes = [p, C.POINTER(Request), C.POINTER(u64)]
    L.salt_serve_poll.argtypes = [p, u64, i32, p, p]
    L.salt_serve_cancel.argtypes = [p, u64]
    L.salt_serve_stats_get.argtypes = [p, C.POINTER(ServeStats)]
    L.salt_status_str.argtypes = [C.c_int]
    L.salt_status_str.restype = C.c_char_p
    L.salt_last_error.argtypes = [p]
    L.salt_last_error.restype = C.c_char_p
    void_fns = ("salt_destroy", "salt_plan_destroy")
    str_fns = ("salt_status_str", "salt_last_error")
    for name in EXPORTS:
        if name not in void_fns + str_fns:
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(x):
    """Address of a numpy array or a torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Context:
    """Owns a salt_ctx: the model grids and bandpasses on one CUDA device."""

    def __init__(self, model, bands, device: int = 0, serve_mem_bytes: int = 0):
        L = lib()
        m0 = np.ascontiguousarray(model.m0, dtype=np.float32)
        m1 = np.ascontiguousarray(model.m1, dtype=np.float32)
        cl = np.ascontiguousarray(model.cl, dtype=np.float64)
        nodes = [getattr(model, k, None) for k in ("phase_nodes", "wave_nodes")]
        nodes = [None if v is None else np.ascontiguousarray(v, dtype=np.float64) for v in nodes]
        md = ModelDesc(model.n_phase, model.n_wave, model.phase0, model.dphase, model.wave0,
                       model.dwave, m0.ctypes.data, m1.ctypes.data, len(cl), cl.ctypes.data,
                       model.cl_lo, model.cl_hi, *[None if v is None else v.ctypes.data for v in nodes])
        keep = [v for v in nodes if v is not None]
        arr = (BandDesc * max(1, len(bands)))()
        for b, band in enumerate(bands):
            w = np.ascontiguousarray(band.wave, dtype=np.float64)
            t = np.ascontiguousarray(band.trans, dtype=np.float64)
            keep += [w, t]
            arr[b] = BandDesc(len(w), w.ctypes.data, t.ctypes.data)
        h = C.c_void_p()
        rc = L.salt_init_model(C.byref(md), arr, len(bands), device, serve_mem_bytes, C.byref(h))
        if rc != SALT_OK:
            raise SaltError(rc, L.salt_status_str(rc).decode())
        self.h = h
        self.device = device
        self.n_bands = len(bands)

    def close(self):
        if getattr(self, "h", None):
            lib().salt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc: int):
        if rc != SALT_OK:
            msg = lib().salt_last_error(self.h).decode() if self.h else ""
            raise SaltError(rc, msg or lib().salt_status_str(rc).decode())
        return rc

    def set_option(self, opt: int, value: int):
        self.check(lib().salt_set_option(self.h, opt, int(value)))

    def get_option(self, opt: int) -> int:
        v = C.c_int64()
        self.check(lib().salt_get_option(self.h, opt, C.byref(v)))
        return v.value

    def device_check(self, stream=None):
        return lib().salt_check(self.h, stream)


class Plan:
    def __init__(self, ctx: Context, obs_off: np.ndarray, par_off: np.ndarray):
        self.obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
        self.par_off = np.ascontiguousarray(par_off, dtype=np.int64)
        h = C.c_void_p()
        ctx.check(lib().salt_plan_create(ctx.h, len(self.obs_off) - 1, self.obs_off.ctypes.data,
                                         self.par_off.ctypes.data, C.byref(h)))
        self.h = h
        self.ctx = ctx

    def close(self):
        if getattr(self, "h", None):
            lib().salt_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bandflux_offsets(obs_off, par_off) -> np.ndarray:
    oo = np.ascontiguousarray(obs_off, dtype=np.int64)
    po = np.ascontiguousarray(par_off, dtype=np.int64)
    out = np.zeros(len(oo), dtype=np.int64)
    rc = lib().salt_bandflux_offsets(len(oo) - 1, oo.ctypes.data, po.ctypes.data, out.ctypes.data)
    if rc != SALT_OK:
        raise SaltError(rc, "bad offsets")
    return out


def batch_desc(obs_off, par_off, dev: dict, plan: Plan | None = None, validate: bool = False):
    """dev: device tensors mjd, band, flux, fluxerr, zp, t0, z, x0, x1, c."""
    return BatchDesc(len(obs_off) - 1, _ptr(obs_off), _ptr(par_off), _ptr(dev["mjd"]),
                     _ptr(dev["band"]), _ptr(dev["flux"]), _ptr(dev["fluxerr"]), _ptr(dev["zp"]),
                     _ptr(dev["t0"]), _ptr(dev["z"]), _ptr(dev["x0"]), _ptr(dev["x1"]),
                     _ptr(dev["c"]), plan.h.value if plan is not None else None,
                     1 if validate else 0)


def load_band(path: str, step: float = 5.0, wave_scale: float = 1.0):
    """salt_band_load: (wave, trans) float64 arrays from a bandpass text file,
    resampled at multiples of `step` Angstrom (0 keeps the file's samples)."""
    n = C.c_int32()
    rc = lib().salt_band_load(None, str(path).encode(), wave_scale, step, None, None, 0, C.byref(n))
    if rc != SALT_OK:
        raise SaltError(rc, f"cannot load bandpass {path}")
    wave = np.empty(n.value)
    trans = np.empty(n.value)
    rc = lib().salt_band_load(None, str(path).encode(), wave_scale, step, wave.ctypes.data,
                              trans.ctypes.data, n.value, C.byref(n))
    if rc != SALT_OK:
        raise SaltError(rc, f"cannot load bandpass {path}")
    return wave, trans
