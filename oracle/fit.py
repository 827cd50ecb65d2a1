"""Reference minimiser for the fitting path (TEST INFRASTRUCTURE ONLY: used by
the tests and the bench's CPU-baseline leg, never by the library).

The paper optimises the free SALT parameters x0, x1, t0 and c with L-BFGS-B
(Implementation, first paragraph). The reference here is that algorithm as a
library routine, scipy.optimize.minimize(method="L-BFGS-B"), applied to each
supernova separately on the FP64 oracle chi^2 and its analytic gradient, with
tight tolerances so that it lands on the constrained minimum. Variables are
scaled as in the device fit (z/0.01, t0/1 d, x0/|x0 start|, x1, c/0.1); the
minimiser's result does not depend on that choice, only its path does.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

PARAMS = ("z", "t0", "x0", "x1", "c")  # gradient order
MASK_Z, MASK_T0, MASK_X0, MASK_X1, MASK_C = 1, 2, 4, 8, 16
DEFAULT_MASK = MASK_T0 | MASK_X0 | MASK_X1 | MASK_C


def scales(theta0):
    """Variable scales of one supernova from its starting point."""
    x0 = abs(float(theta0[2]))
    return np.array([0.01, 1.0, x0 if x0 > 0 else 1e-5, 1.0, 0.1])


def _one_sn(batch, s):
    lo, hi = int(batch.obs_off[s]), int(batch.obs_off[s + 1])
    return SimpleNamespace(obs_off=np.array([0, hi - lo], np.int64), mjd=batch.mjd[lo:hi],
                           band=batch.band[lo:hi], flux=batch.flux[lo:hi],
                           fluxerr=batch.fluxerr[lo:hi], zp=batch.zp[lo:hi],
                           par_off=np.array([0, 1], np.int64))


def _with_theta(b1, theta):
    b1.t0 = np.array([theta[1]])
    b1.z, b1.x0, b1.x1, b1.c = (np.array([theta[i]]) for i in (0, 2, 3, 4))
    return b1


def start_point(batch, s):
    j = int(batch.par_off[s])
    return np.array([batch.z[j], batch.t0[j], batch.x0[j], batch.x1[j], batch.c[j]], np.float64)


def chi2_at(o, batch, theta):
    """FP64 oracle chi^2 of each supernova at theta[s] (n_sn x 5)."""
    out = np.empty(batch.n_sn if hasattr(batch, "n_sn") else len(batch.obs_off) - 1)
    for s in range(len(out)):
        out[s] = o.chi2(_with_theta(_one_sn(batch, s), theta[s]))[0]
    return out


def fit_one(o, batch, s, lower=None, upper=None, mask=DEFAULT_MASK, theta0=None,
            gtol=1e-10, ftol=1e-15, maxiter=2000):
    """Minimise supernova s's chi^2 over the masked parameters within the box.
    Returns (theta, chi2, scipy result)."""
    from scipy.optimize import minimize
    theta0 = start_point(batch, s) if theta0 is None else np.asarray(theta0, np.float64)
    sc = scales(theta0)
    free = [i for i in range(5) if (mask >> i) & 1]
    b1 = _one_sn(batch, s)
    lo = np.full(5, -np.inf) if lower is None else np.asarray(lower, np.float64)
    hi = np.full(5, np.inf) if upper is None else np.asarray(upper, np.float64)
    lo = lo.copy()
    if mask & MASK_Z:
        lo[0] = max(lo[0], -0.99)
    start = np.clip(theta0, lo, hi)

    def fun(v):
        th = start.copy()
        th[free] = v * sc[free]
        f, g = o.chi2(_with_theta(b1, th), grad=True)
        return float(f[0]), g[0][free] * sc[free]

    bounds = [(lo[i] / sc[i] if np.isfinite(lo[i]) else None,
               hi[i] / sc[i] if np.isfinite(hi[i]) else None) for i in free]
    res = minimize(fun, start[free] / sc[free], jac=True, method="L-BFGS-B", bounds=bounds,
                   options=dict(maxiter=maxiter, gtol=gtol, ftol=ftol, maxcor=10))
    th = start.copy()
    th[free] = res.x * sc[free]
    return th, float(res.fun), res


def fit_batch(o, batch, lower=None, upper=None, mask=DEFAULT_MASK, sns=None, **kw):
    """fit_one over the supernovae `sns` (default all); lower/upper n_sn x 5."""
    n = len(batch.obs_off) - 1
    sns = range(n) if sns is None else sns
    thetas, chi2s, nits = [], [], []
    for s in sns:
        th, f, res = fit_one(o, batch, s, None if lower is None else lower[s],
                             None if upper is None else upper[s], mask, **kw)
        thetas.append(th)
        chi2s.append(f)
        nits.append(res.nit)
    return np.array(thetas), np.array(chi2s), np.array(nits)
