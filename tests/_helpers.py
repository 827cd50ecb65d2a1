"""Shared test helpers: workloads with observed fluxes made by the FP64 oracle
at the truth (plus seeded noise), tolerances, and comparisons."""
import numpy as np

import oracle
import workloads as W

# Tolerances (FP32 kernel vs FP64 oracle).
BF_RTOL = 1e-5          # bandflux, relative
BF_FLOOR = 1e-3         # ... relative to max(|B|, BF_FLOOR * max |B| of the supernova)
GRAD_RTOL = 1e-3        # gradient, against the scaled gradient's inf-norm per sample
SCALES = (0.01, 1.0, None, 1.0, 0.1)  # z, t0, x0 (-> |x0|), x1, c


def with_oracle_flux(wl, seed=11, noiseless=False):
    """Fill observed fluxes with oracle model values at the truth + 5% noise."""
    o = oracle.Oracle(wl.model, wl.bands)
    tb = W.truth_batch(wl.batch)
    m = o.bandflux(tb)
    W.add_noise(wl.batch, m, np.random.default_rng(seed), noiseless=noiseless)
    return o


def bf_scale(batch, ref):
    """Per-bandflux comparison scale max(|B|, floor * max |B| over its SN)."""
    scale = np.abs(ref).astype(np.float64)
    off = oracle.Oracle.bandflux_offsets(batch)
    for s in range(batch.n_sn):
        lo, hi = off[s], off[s + 1]
        if hi > lo:
            scale[lo:hi] = np.maximum(scale[lo:hi], BF_FLOOR * np.abs(ref[lo:hi]).max())
    return scale


def assert_bandflux_close(batch, got, ref, rtol=BF_RTOL):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref) / np.maximum(bf_scale(batch, ref), 1e-300)
    assert np.all(np.isfinite(got))
    worst = float(err.max()) if err.size else 0.0
    assert worst <= rtol, f"max relative bandflux error {worst:.3e} > {rtol}"
    return worst


def chi2_bound(batch, bf_ref, rtol=BF_RTOL):
    """|dchi2| <= sum_i 2|r_i| e_i + e_i^2 with e_i = rtol * scale_i / sigma_i."""
    off = oracle.Oracle.bandflux_offsets(batch)
    scale = bf_scale(batch, bf_ref)
    out = np.zeros(batch.n_par)
    for s in range(batch.n_sn):
        n = int(batch.obs_off[s + 1] - batch.obs_off[s])
        if n == 0:
            continue
        f = batch.flux[batch.obs_off[s]:batch.obs_off[s + 1]].astype(np.float64)
        sig = batch.fluxerr[batch.obs_off[s]:batch.obs_off[s + 1]].astype(np.float64)
        for jj, j in enumerate(range(batch.par_off[s], batch.par_off[s + 1])):
            sl = slice(off[s] + jj * n, off[s] + (jj + 1) * n)
            r = (f - bf_ref[sl]) / sig
            e = rtol * scale[sl] / sig
            out[j] = np.sum(2 * np.abs(r) * e + e * e)
    return out


def assert_chi2_close(batch, got, ref, bf_ref):
    got = np.asarray(got, dtype=np.float64)
    bound = chi2_bound(batch, bf_ref) + 1e-12 * np.abs(ref) + 1e-12
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"chi2 outside its bound at {bad[:5]}: {err[bad[:5]]} > {bound[bad[:5]]}"
    return float(np.max(err / np.maximum(bound, 1e-300))) if err.size else 0.0


def grad_scale(batch):
    return np.stack([np.full(batch.n_par, SCALES[0]), np.full(batch.n_par, SCALES[1]),
                     np.abs(batch.x0.astype(np.float64)), np.full(batch.n_par, SCALES[3]),
                     np.full(batch.n_par, SCALES[4])], 1)


FD_SCALES = (0.01, 1.0, None, 1.0, 0.1)  # FD step scale per parameter (x0: |x0|)


def bandflux_jacobian(o, batch):
    """d B / d(z, t0, x0, x1, c) of every bandflux by FP64 central differences
    of the oracle's bandflux, h = 1e-4 max(|theta|, scale)."""
    names = ("z", "t0", "x0", "x1", "c")
    n_bf = int(o.bandflux_offsets(batch)[-1])
    jac = np.zeros((n_bf, 5))
    for q, name in enumerate(names):
        base = np.asarray(getattr(batch, name), dtype=np.float64)
        scale = np.abs(base) if FD_SCALES[q] is None else np.full_like(base, FD_SCALES[q])
        h = 1e-4 * np.maximum(np.abs(base), scale)
        out = []
        for sign in (1.0, -1.0):
            b2 = W.Batch(**{k: getattr(batch, k) for k in ("obs_off", "mjd", "band", "flux", "fluxerr", "zp",
                                                         "par_off", "t0", "z", "x0", "x1", "c")})
            setattr(b2, name, base + sign * h)  # float64 copy: the oracle evaluates in FP64
            out.append(o.bandflux(b2))
        per_sample_h = np.repeat(h, _bf_per_sample(batch))
        jac[:, q] = (out[0] - out[1]) / (2 * per_sample_h)
    return jac


def _bf_per_sample(batch):
    n_obs = np.diff(batch.obs_off)
    n_par = np.diff(batch.par_off)
    return np.repeat(n_obs, n_par)  # bandfluxes of each sample, in bandflux order


def grad_bound(batch, bf_ref, jac, rtol=BF_RTOL):
    """Per sample and parameter: the change in d chi^2 / d theta that bandflux
    errors of rtol (on the comparison scale, as in chi2_bound) and derivative
    errors of rtol (relative) can make:
    sum_i 2 |dB_i/dtheta| (e_i / sigma_i^2 + rtol |r_i| / sigma_i)."""
    off = oracle.Oracle.bandflux_offsets(batch)
    scale = bf_scale(batch, bf_ref)
    out = np.zeros((batch.n_par, 5))
    for s in range(batch.n_sn):
        n = int(batch.obs_off[s + 1] - batch.obs_off[s])
        if n == 0:
            continue
        f = batch.flux[batch.obs_off[s]:batch.obs_off[s + 1]].astype(np.float64)
        sig = batch.fluxerr[batch.obs_off[s]:batch.obs_off[s + 1]].astype(np.float64)
        for jj, j in enumerate(range(batch.par_off[s], batch.par_off[s + 1])):
            sl = slice(off[s] + jj * n, off[s] + (jj + 1) * n)
            r = (f - bf_ref[sl]) / sig
            e = rtol * scale[sl]
            w = 2.0 * (e / sig ** 2 + rtol * np.abs(r) / sig)
            out[j] = np.abs(jac[sl]).T @ w
    return out


# Samples whose gradient may pass only through grad_bound (the fallback): at
# most FALLBACK_FRAC of a batch's samples, and at least FALLBACK_MIN allowed.
FALLBACK_FRAC = 0.01
FALLBACK_MIN = 2
# (test, samples compared, samples that needed the fallback) of every call
FALLBACK_LOG = []


def assert_grad_close(batch, got, ref, rtol=GRAD_RTOL, o=None, bf_ref=None, max_fallback=None):
    """Scaled gradient within rtol of its per-sample inf-norm; where that fails
    and the oracle `o` is given, within the larger of that and grad_bound (what
    the bandflux tolerance allows a gradient that is a sum with cancellation,
    near a minimum) -- the gradient counterpart of assert_chi2_close.

    At most `max_fallback` samples may pass through grad_bound alone
    (default: max(FALLBACK_MIN, ceil(FALLBACK_FRAC * samples))), so that a
    regression moving many gradients into the fallback fails. Returns
    (worst error as a fraction of its allowance, samples that needed the
    fallback); every call is recorded in FALLBACK_LOG."""
    import os
    s = grad_scale(batch)
    gs = np.asarray(got, np.float64) * s
    rs = np.asarray(ref, np.float64) * s
    assert np.all(np.isfinite(gs))
    norm = np.max(np.abs(rs), axis=1, keepdims=True)
    allowed = rtol * np.maximum(norm, 1e-300)
    err = np.abs(gs - rs) / allowed
    strict_fail = err.max(axis=1) > 1.0 if err.size else np.zeros(0, bool)
    n_fallback = 0
    if strict_fail.any() and o is not None:
        bf = o.bandflux(batch) if bf_ref is None else bf_ref
        bound = grad_bound(batch, bf, bandflux_jacobian(o, batch)) * s
        err = np.abs(gs - rs) / np.maximum(allowed, bound)
        n_fallback = int(np.sum(strict_fail & (err.max(axis=1) <= 1.0)))
    worst = float(err.max()) if err.size else 0.0
    n = int(gs.shape[0])
    FALLBACK_LOG.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], n, n_fallback))
    assert worst <= 1.0, f"scaled gradient error {worst:.3f} of its allowance (rtol {rtol})"
    limit = max(FALLBACK_MIN, int(np.ceil(FALLBACK_FRAC * n))) if max_fallback is None else max_fallback
    assert n_fallback <= limit, \
        f"{n_fallback} of {n} gradients pass only through the bandflux-derived bound (limit {limit})"
    return worst, n_fallback


DCHI2 = 2e-3  # fit parity: floor of the chi^2 excess allowed over the reference minimum


def dchi2_tol(o, start, theta):
    """Fit parity tolerance per supernova: max(DCHI2, the chi^2 change 1e-5
    relative bandflux errors can make at theta), theta [n_sn][5]."""
    out = np.empty(start.n_sn)
    for s in range(start.n_sn):
        one = W.subset(start, [s])
        one.t0 = np.array([theta[s, 1]])
        one.z, one.x0, one.x1, one.c = (np.array([theta[s, i]]) for i in (0, 2, 3, 4))
        out[s] = max(DCHI2, chi2_bound(one, o.bandflux(one))[0])
    return out
