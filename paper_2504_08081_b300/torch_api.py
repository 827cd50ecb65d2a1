"""torch front end of the C ABI: device-resident batches, batch calls on the
current CUDA stream, and chi^2 with its hand-written adjoint as an autograd
Function. Only marshalling happens here; every step runs in libsalt_b300.so."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import Context, Plan, SaltError

OBS_FIELDS = (("mjd", torch.float64), ("band", torch.int32), ("flux", torch.float32),
              ("fluxerr", torch.float32), ("zp", torch.float32))
PAR_FIELDS = (("t0", torch.float64), ("z", torch.float32), ("x0", torch.float32),
              ("x1", torch.float32), ("c", torch.float32))


class DeviceBatch:
    """A ragged batch resident on one CUDA device: host CSR offsets plus device
    tensors for the observation and parameter arrays."""

    def __init__(self, obs_off, par_off, tensors: dict, plan: Plan | None = None):
        self.obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
        self.par_off = np.ascontiguousarray(par_off, dtype=np.int64)
        self.t = tensors
        self.plan = plan

    @property
    def n_sn(self):
        return len(self.obs_off) - 1

    @property
    def n_par(self):
        return int(self.par_off[-1])

    @property
    def n_obs(self):
        return int(self.obs_off[-1])

    def with_params(self, **params) -> "DeviceBatch":
        t = dict(self.t)
        t.update(params)
        return DeviceBatch(self.obs_off, self.par_off, t, self.plan)


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Salt:
    """One model (grids + bandpasses) on one device."""

    def __init__(self, model, bands, device: int = 0, serve_mem_bytes: int = 0):
        self.device = torch.device("cuda", device)
        self.ctx = Context(model, bands, device=device, serve_mem_bytes=serve_mem_bytes)

    def close(self):
        self.ctx.close()

    # -- data movement -------------------------------------------------------
    def upload(self, batch, plan: bool = True, pin: bool = False) -> DeviceBatch:
        """Copy a host batch (workloads.Batch-like: numpy arrays) to the device."""
        t = {}
        for name, dt in OBS_FIELDS + PAR_FIELDS:
            a = torch.from_numpy(np.ascontiguousarray(getattr(batch, name)))
            a = a.to(dt)
            if pin:
                a = a.pin_memory()
            t[name] = a.to(self.device, non_blocking=pin)
        db = DeviceBatch(batch.obs_off, batch.par_off, t)
        if plan:
            db.plan = Plan(self.ctx, db.obs_off, db.par_off)
        return db

    def plan(self, db: DeviceBatch) -> Plan:
        db.plan = Plan(self.ctx, db.obs_off, db.par_off)
        return db.plan

    def _desc(self, db: DeviceBatch, validate: bool):
        for name, dt in OBS_FIELDS + PAR_FIELDS:
            x = db.t[name]
            if x.dtype != dt or not x.is_cuda or not x.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous {dt} CUDA tensor")
        return _abi.batch_desc(db.obs_off, db.par_off, db.t, db.plan, validate)

    # -- batch calls ---------------------------------------------------------
    def bandflux_offsets(self, db: DeviceBatch) -> np.ndarray:
        return _abi.bandflux_offsets(db.obs_off, db.par_off)

    def bandflux(self, db: DeviceBatch, out: torch.Tensor | None = None, validate=False):
        n = int(self.bandflux_offsets(db)[-1])
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=self.device)
        d = self._desc(db, validate)
        self.ctx.check(_abi.lib().salt_bandflux(self.ctx.h, C.byref(d), out.data_ptr(),
                                                _stream(self.device)))
        return out

    def chi2(self, db: DeviceBatch, out: torch.Tensor | None = None, validate=False):
        if out is None:
            out = torch.empty(db.n_par, dtype=torch.float64, device=self.device)
        d = self._desc(db, validate)
        self.ctx.check(_abi.lib().salt_chi2(self.ctx.h, C.byref(d), out.data_ptr(),
                                            _stream(self.device)))
        return out

    def chi2_grad(self, db: DeviceBatch, chi2: torch.Tensor | None = None,
                  grad: torch.Tensor | None = None, validate=False):
        if chi2 is None:
            chi2 = torch.empty(db.n_par, dtype=torch.float64, device=self.device)
        if grad is None:
            grad = torch.empty((db.n_par, 5), dtype=torch.float32, device=self.device)
        d = self._desc(db, validate)
        self.ctx.check(_abi.lib().salt_chi2_grad(self.ctx.h, C.byref(d), chi2.data_ptr(),
                                                 grad.data_ptr(), _stream(self.device)))
        return chi2, grad

    def chi2_grad_noalloc(self, db: DeviceBatch, chi2: torch.Tensor, grad: torch.Tensor,
                          validate=False):
        """chi2_grad through the no-allocation entry point, into caller-owned
        outputs (float64 [n_par], float32 [n_par, 5] on this device)."""
        if chi2.dtype != torch.float64 or grad.dtype != torch.float32 or \
                chi2.numel() < db.n_par or grad.numel() < 5 * db.n_par or \
                not chi2.is_contiguous() or not grad.is_contiguous():
            raise ValueError("chi2/grad: contiguous float64 [n_par] / float32 [n_par, 5] tensors")
        d = self._desc(db, validate)
        self.ctx.check(_abi.lib().salt_chi2_grad_noalloc(self.ctx.h, C.byref(d), chi2.data_ptr(),
                                                         grad.data_ptr(), _stream(self.device)))
        return chi2, grad

    def fit(self, db: DeviceBatch, lower: torch.Tensor | None = None, upper: torch.Tensor | None = None,
            free_mask: int = 0, max_iter: int = 0, max_evals: int = 0, history: int = 0,
            gtol: float = 0.0, ftol: float = 0.0):
        """Fit every supernova's parameters (one starting sample per supernova in
        db). lower/upper: float64 [n_sn, 5] device tensors (z, t0, x0, x1, c) or
        None. Returns theta float64 [n_sn, 5], chi2 float64 [n_sn] and status
        int32 [n_sn] (device tensors)."""
        n = db.n_sn
        for b in (lower, upper):
            if b is not None and (b.dtype != torch.float64 or not b.is_cuda or not b.is_contiguous()
                                  or b.numel() != 5 * n):
                raise ValueError("bounds: contiguous float64 [n_sn, 5] CUDA tensors")
        theta = torch.empty((n, 5), dtype=torch.float64, device=self.device)
        chi2 = torch.empty(n, dtype=torch.float64, device=self.device)
        status = torch.empty(n, dtype=torch.int32, device=self.device)
        opts = _abi.FitOpts(max_iter, max_evals, history, free_mask, gtol, ftol)
        d = self._desc(db, False)
        self.ctx.check(_abi.lib().salt_fit(
            self.ctx.h, C.byref(d), lower.data_ptr() if lower is not None else None,
            upper.data_ptr() if upper is not None else None, C.byref(opts), theta.data_ptr(),
            chi2.data_ptr(), status.data_ptr(), _stream(self.device)))
        return theta, chi2, status

    def nested(self, db: DeviceBatch, lower: torch.Tensor, upper: torch.Tensor, free_mask: int = 0,
               n_live: int = 0, n_batch: int = 0, n_steps: int = 0, max_iter: int = 0, seed: int = 1,
               dlogz: float = 0.0):
        """Nested sampling per supernova (one sample per supernova in db holds
        the values of the parameters not sampled). lower/upper: float64
        [n_sn, 5] device tensors, the uniform prior box. Returns logz, logz_err
        (float64 [n_sn]), mean, std (float64 [n_sn, 5]), status (int32 [n_sn])."""
        n = db.n_sn
        for b in (lower, upper):
            if b.dtype != torch.float64 or not b.is_cuda or not b.is_contiguous() or b.numel() != 5 * n:
                raise ValueError("prior box: contiguous float64 [n_sn, 5] CUDA tensors")
        f64 = dict(dtype=torch.float64, device=self.device)
        logz, err = torch.empty(n, **f64), torch.empty(n, **f64)
        mean, std = torch.empty((n, 5), **f64), torch.empty((n, 5), **f64)
        status = torch.empty(n, dtype=torch.int32, device=self.device)
        opts = _abi.NestedOpts(n_live, n_batch, n_steps, max_iter, free_mask, 0, seed, dlogz)
        d = self._desc(db, False)
        self.ctx.check(_abi.lib().salt_nested(
            self.ctx.h, C.byref(d), lower.data_ptr(), upper.data_ptr(), C.byref(opts), logz.data_ptr(),
            err.data_ptr(), mean.data_ptr(), std.data_ptr(), status.data_ptr(), _stream(self.device)))
        return logz, err, mean, std, status

    def check(self):
        """Synchronise and raise if a kernel met invalid batch data."""
        self.ctx.check(self.ctx.device_check(_stream(self.device)))

    def set_kernel(self, which: int):
        self.ctx.set_option(_abi.SALT_OPT_KERNEL, which)

    def set_tile(self, tile: int):
        self.ctx.set_option(_abi.SALT_OPT_TILE_SAMPLES, tile)

    def register_band(self, wave, trans) -> int:
        """Add a bandpass (wavelength [A], transmission) to this context; returns its id."""
        w = np.ascontiguousarray(wave, np.float64)
        t = np.ascontiguousarray(trans, np.float64)
        if w.shape != t.shape or w.ndim != 1:
            raise ValueError("wave and trans: 1-D arrays of one length")
        bd = _abi.BandDesc(len(w), w.ctypes.data, t.ctypes.data)
        bid = C.c_int32()
        self.ctx.check(_abi.lib().salt_register_band(self.ctx.h, C.byref(bd), C.byref(bid)))
        return bid.value

    def set_graphs(self, on: bool):
        self.ctx.set_option(_abi.SALT_OPT_GRAPHS, 1 if on else 0)

    def last_kernel(self) -> tuple[int, int]:
        """(SALT_KERNEL_* family, samples per tile) of the last batch launch."""
        v = self.ctx.get_option(_abi.SALT_OPT_LAST_KERNEL)
        return v // 32, v % 32

    def measure_peaks(self) -> dict:
        """FP32 FMA rate, L2 and shared-memory read bandwidth of this device
        (salt_measure_peaks microbenchmarks; synchronous)."""
        pk = _abi.Peaks()
        self.ctx.check(_abi.lib().salt_measure_peaks(self.ctx.h, C.byref(pk)))
        return {f: getattr(pk, f) for f, _ in _abi.Peaks._fields_}

    # -- serving -------------------------------------------------------------
    def submit(self, n_obs, mjd, band, flux, fluxerr, zp, t0, z, x0, x1, c, want_grad) -> int:
        arrs = [np.ascontiguousarray(mjd, np.float64), np.ascontiguousarray(band, np.int32),
                np.ascontiguousarray(flux, np.float32), np.ascontiguousarray(fluxerr, np.float32),
                np.ascontiguousarray(zp, np.float32), np.ascontiguousarray(t0, np.float64),
                np.ascontiguousarray(z, np.float32), np.ascontiguousarray(x0, np.float32),
                np.ascontiguousarray(x1, np.float32), np.ascontiguousarray(c, np.float32)]
        req = _abi.Request(int(n_obs), len(arrs[5]), 1 if want_grad else 0,
                           *[a.ctypes.data for a in arrs])
        tk = C.c_uint64()
        self.ctx.check(_abi.lib().salt_serve_submit(self.ctx.h, C.byref(req), C.byref(tk)))
        return tk.value

    def poll(self, ticket: int, n_par: int, want_grad: bool, wait_ms: int = -1):
        chi2 = np.empty(n_par, dtype=np.float64)
        grad = np.empty((n_par, 5), dtype=np.float32) if want_grad else None
        rc = _abi.lib().salt_serve_poll(self.ctx.h, ticket, wait_ms, chi2.ctypes.data,
                                        grad.ctypes.data if grad is not None else None)
        return rc, chi2, grad

    def cancel(self, ticket: int) -> int:
        return _abi.lib().salt_serve_cancel(self.ctx.h, ticket)

    def serve_stats(self) -> dict:
        st = _abi.ServeStats()
        self.ctx.check(_abi.lib().salt_serve_stats_get(self.ctx.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in _abi.ServeStats._fields_}


class SaltChi2(torch.autograd.Function):
    """chi^2 per parameter sample with d chi^2 / d(z, t0, x0, x1, c) from the
    library's adjoint kernel (one fused forward+adjoint launch)."""

    @staticmethod
    def forward(ctx, salt: Salt, db: DeviceBatch, z, t0, x0, x1, c):
        b = db.with_params(z=z.detach().contiguous(), t0=t0.detach().contiguous(),
                           x0=x0.detach().contiguous(), x1=x1.detach().contiguous(),
                           c=c.detach().contiguous())
        chi2, grad = salt.chi2_grad(b)
        ctx.save_for_backward(grad)
        return chi2

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        g = gout.to(torch.float32)[:, None] * grad
        return (None, None, g[:, 0].contiguous(), g[:, 1].to(torch.float64).contiguous(),
                g[:, 2].contiguous(), g[:, 3].contiguous(), g[:, 4].contiguous())


__all__ = ["Salt", "SaltChi2", "DeviceBatch", "SaltError"]
