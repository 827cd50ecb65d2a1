"""FP64 CPU oracle for batched SALT synthetic photometry (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
bench's CPU-baseline leg, never by the library. The arithmetic lives in
salt_oracle.c (plain C, double precision, host libm); this module only
marshals numpy arrays into it. See salt_oracle.c for the definitions followed
(SALT model form, Eq. 1; bandflux integral, Eq. 2; trapezoidal rule) and the
readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build

_lib = None


class _Model(C.Structure):
    _fields_ = [("n_phase", C.c_int32), ("n_wave", C.c_int32),
                ("phase0", C.c_double), ("dphase", C.c_double),
                ("wave0", C.c_double), ("dwave", C.c_double),
                ("m0", C.POINTER(C.c_double)), ("m1", C.POINTER(C.c_double)),
                ("cl", C.c_double * 4), ("cl_lo", C.c_double), ("cl_hi", C.c_double),
                ("pnode", C.POINTER(C.c_double)), ("wnode", C.POINTER(C.c_double))]


class _Band(C.Structure):
    _fields_ = [("n", C.c_int32), ("wave", C.POINTER(C.c_double)),
                ("trans", C.POINTER(C.c_double))]


class _Batch(C.Structure):
    _fields_ = [("n_sn", C.c_int64), ("obs_off", C.POINTER(C.c_int64)),
                ("mjd", C.POINTER(C.c_double)), ("band", C.POINTER(C.c_int32)),
                ("flux", C.POINTER(C.c_double)), ("fluxerr", C.POINTER(C.c_double)),
                ("zp", C.POINTER(C.c_double)), ("par_off", C.POINTER(C.c_int64)),
                ("t0", C.POINTER(C.c_double)), ("z", C.POINTER(C.c_double)),
                ("x0", C.POINTER(C.c_double)), ("x1", C.POINTER(C.c_double)),
                ("c", C.POINTER(C.c_double))]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i32, i64, p = C.c_double, C.c_int32, C.c_int64, C.c_void_p
        _lib.om_axis_taps_nodes.restype = C.c_int
        _lib.om_axis_taps_nodes.argtypes = [d, p, i32, C.POINTER(i32), p, p]
        _lib.om_axis_taps.restype = C.c_int
        _lib.om_axis_taps.argtypes = [d, d, d, i32, C.POINTER(i32), p, p]
        _lib.om_surface.restype = d
        _lib.om_surface.argtypes = [C.POINTER(_Model), p, d, d, C.POINTER(d), C.POINTER(d)]
        _lib.om_colorlaw.restype = d
        _lib.om_colorlaw.argtypes = [p, d, d, d, C.POINTER(d)]
        _lib.om_flux_obs.restype = d
        _lib.om_flux_obs.argtypes = [C.POINTER(_Model), d, d, p, p]
        _lib.om_trapz.restype = d
        _lib.om_trapz.argtypes = [i32, p, p]
        _lib.om_band_ab_flux.restype = d
        _lib.om_band_ab_flux.argtypes = [C.POINTER(_Band)]
        _lib.om_bandflux_one.restype = d
        _lib.om_bandflux_one.argtypes = [C.POINTER(_Model), C.POINTER(_Band), d, d, p, p]
        _lib.om_bandflux_batch.restype = None
        _lib.om_bandflux_batch.argtypes = [C.POINTER(_Model), C.POINTER(_Band), C.POINTER(_Batch), p, p]
        _lib.om_chi2_batch.restype = None
        _lib.om_chi2_batch.argtypes = [C.POINTER(_Model), C.POINTER(_Band), C.POINTER(_Batch), p, p]
        _lib.om_set_threads.argtypes = [C.c_int]
        _lib.om_get_max_threads.restype = C.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Oracle:
    """Holds FP64 copies of a model and its bands for repeated evaluation."""

    def __init__(self, model, bands, threads: int | None = None):
        L = lib()
        self._keep = []
        self.m0 = np.ascontiguousarray(model.m0, dtype=np.float64)
        self.m1 = np.ascontiguousarray(model.m1, dtype=np.float64)
        cl = (C.c_double * 4)(*[float(v) for v in model.cl])
        nodes = []
        for name in ("phase_nodes", "wave_nodes"):
            v = getattr(model, name, None)
            v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
            self._keep.append(v)
            nodes.append(None if v is None else _dp(v))
        self.model = _Model(model.n_phase, model.n_wave, model.phase0, model.dphase,
                            model.wave0, model.dwave, _dp(self.m0), _dp(self.m1), cl,
                            model.cl_lo, model.cl_hi, nodes[0], nodes[1])
        nb = len(bands)
        self.bands = (_Band * max(nb, 1))()
        for b, band in enumerate(bands):
            w = np.ascontiguousarray(band.wave, dtype=np.float64)
            t = np.ascontiguousarray(band.trans, dtype=np.float64)
            self._keep += [w, t]
            self.bands[b] = _Band(len(w), _dp(w), _dp(t))
        self.threads = threads if threads else max(1, os.cpu_count() or 1)
        L.om_set_threads(self.threads)

    # -- pieces ------------------------------------------------------------
    def surface(self, which: int, p: float, lam: float):
        dp_, dl_ = C.c_double(), C.c_double()
        G = self.m0 if which == 0 else self.m1
        v = lib().om_surface(C.byref(self.model), G.ctypes.data, p, lam, C.byref(dp_), C.byref(dl_))
        return v, dp_.value, dl_.value

    def colorlaw(self, lam: float):
        d = C.c_double()
        cl = np.ascontiguousarray(np.array(self.model.cl[:]), dtype=np.float64)
        v = lib().om_colorlaw(cl.ctypes.data, self.model.cl_lo, self.model.cl_hi, lam, C.byref(d))
        return v, d.value

    def flux_obs(self, lam_obs, mjd, par, grad=False):
        par = np.ascontiguousarray(par, dtype=np.float64)
        d = np.zeros(5)
        v = lib().om_flux_obs(C.byref(self.model), lam_obs, mjd, par.ctypes.data,
                              d.ctypes.data if grad else None)
        return (v, d) if grad else v

    def band_ab_flux(self, b: int) -> float:
        return lib().om_band_ab_flux(C.byref(self.bands[b]))

    def bandflux_one(self, band: int, mjd: float, zp: float, par, grad=False):
        par = np.ascontiguousarray(par, dtype=np.float64)
        g = np.zeros(5)
        v = lib().om_bandflux_one(C.byref(self.model), C.byref(self.bands[band]), mjd, zp,
                                  par.ctypes.data, g.ctypes.data if grad else None)
        return (v, g) if grad else v

    # -- batched -----------------------------------------------------------
    def _batch(self, bt):
        arrs = dict(obs_off=np.ascontiguousarray(bt.obs_off, dtype=np.int64),
                    mjd=np.ascontiguousarray(bt.mjd, dtype=np.float64),
                    band=np.ascontiguousarray(bt.band, dtype=np.int32),
                    flux=np.ascontiguousarray(bt.flux, dtype=np.float64),
                    fluxerr=np.ascontiguousarray(bt.fluxerr, dtype=np.float64),
                    zp=np.ascontiguousarray(bt.zp, dtype=np.float64),
                    par_off=np.ascontiguousarray(bt.par_off, dtype=np.int64),
                    t0=np.ascontiguousarray(bt.t0, dtype=np.float64),
                    z=np.ascontiguousarray(bt.z, dtype=np.float64),
                    x0=np.ascontiguousarray(bt.x0, dtype=np.float64),
                    x1=np.ascontiguousarray(bt.x1, dtype=np.float64),
                    c=np.ascontiguousarray(bt.c, dtype=np.float64))
        i64p = lambda a: a.ctypes.data_as(C.POINTER(C.c_int64))
        s = _Batch(len(arrs["obs_off"]) - 1, i64p(arrs["obs_off"]), _dp(arrs["mjd"]),
                   arrs["band"].ctypes.data_as(C.POINTER(C.c_int32)), _dp(arrs["flux"]),
                   _dp(arrs["fluxerr"]), _dp(arrs["zp"]), i64p(arrs["par_off"]),
                   _dp(arrs["t0"]), _dp(arrs["z"]), _dp(arrs["x0"]), _dp(arrs["x1"]),
                   _dp(arrs["c"]))
        return s, arrs

    @staticmethod
    def bandflux_offsets(bt) -> np.ndarray:
        n = np.diff(np.asarray(bt.obs_off, dtype=np.int64))
        s = np.diff(np.asarray(bt.par_off, dtype=np.int64))
        off = np.zeros(len(n) + 1, dtype=np.int64)
        off[1:] = np.cumsum(n * s)
        return off

    def bandflux(self, bt) -> np.ndarray:
        s, keep = self._batch(bt)
        off = self.bandflux_offsets(bt)
        out = np.zeros(int(off[-1]))
        lib().om_set_threads(self.threads)
        lib().om_bandflux_batch(C.byref(self.model), self.bands, C.byref(s), off.ctypes.data,
                                out.ctypes.data)
        return out

    def chi2(self, bt, grad=False):
        s, keep = self._batch(bt)
        n_par = int(bt.par_off[-1])
        chi2 = np.zeros(n_par)
        g = np.zeros((n_par, 5)) if grad else None
        lib().om_set_threads(self.threads)
        lib().om_chi2_batch(C.byref(self.model), self.bands, C.byref(s), chi2.ctypes.data,
                            g.ctypes.data if grad else None)
        return (chi2, g) if grad else chi2
