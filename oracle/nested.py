"""Reference nested sampler for the nested-sampling path (TEST INFRASTRUCTURE
ONLY: used by the tests and the bench's CPU-baseline leg, never by the library).

The paper samples the SALT posterior by nested sampling (Implementation, first
paragraph: the ns.py example). It prints no algorithm, so the method here is
standard nested sampling (Skilling's evidence integration over a shrinking
prior volume), written step by step in the order the device path takes them,
on the FP64 oracle chi^2 (log L = -chi^2 / 2) and a uniform prior box:

  1. N live points drawn uniformly in the box of the free parameters.
  2. Each iteration: order the live points by log L (ties by index). If the
     live points could add less than dlogz to log Z (max log L + log X),
     stop. Otherwise remove the k lowest: removing the j-th of them (while
     N - j points are live) shrinks log X by 1/(N - j) (its expected log
     shrinkage) and adds weight X_before - X_after at its log L to the
     evidence and the posterior moments.
  3. Replace them: chain c starts at a surviving point picked uniformly and
     takes M random-walk steps theta' = theta + f sigma * n (n standard
     normal, sigma the survivors' standard deviation per parameter, f a
     common scale), accepting a proposal inside the box with log L above the
     k-th lowest removed log L; the chain's end state takes the place of the
     c-th removed point. After the iteration f is multiplied by
     exp(acceptance rate - 1/2) (clipped to [1e-3, 10]).
  4. At the stop the live points share the remaining volume equally.
Random numbers come from Philox4x32-10 (Salmon et al., SC'11), counter
(supernova, iteration or point, index, stream) and key (seed low/high 32
bits), so the device path draws the same numbers.
"""
from __future__ import annotations

import math
from types import SimpleNamespace

import numpy as np

from .fit import PARAMS, DEFAULT_MASK, MASK_X0, start_point, _one_sn  # noqa: F401

_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
STREAM_INIT, STREAM_START, STREAM_STEP = 0, 1, 2


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds: 4 counter words, 2 key words -> 4 words."""
    c0, c1, c2, c3 = (int(v) & 0xFFFFFFFF for v in ctr)
    k0, k1 = (int(v) & 0xFFFFFFFF for v in key)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & 0xFFFFFFFF, p1 & 0xFFFFFFFF, \
                         ((p0 >> 32) ^ c3 ^ k1) & 0xFFFFFFFF, p0 & 0xFFFFFFFF
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def _u01(x):
    return (x + 0.5) * 2.0 ** -32


def _draw(seed, s, a, b, stream, part):
    return philox4x32_10((s, a, b, 4 * stream + part), (seed & 0xFFFFFFFF, seed >> 32))


def uniforms5(seed, s, a, b, stream):
    w = _draw(seed, s, a, b, stream, 0) + _draw(seed, s, a, b, stream, 1)
    return [_u01(w[i]) for i in range(5)]


def normals5(seed, s, a, b, stream):
    w = _draw(seed, s, a, b, stream, 0) + _draw(seed, s, a, b, stream, 1)
    out = []
    for q in range(3):  # Box-Muller on (w[2q], w[2q+1])
        r = math.sqrt(-2.0 * math.log(_u01(w[2 * q])))
        ang = 2.0 * math.pi * _u01(w[2 * q + 1])
        out += [r * math.cos(ang), r * math.sin(ang)]
    return out[:5]


def pick(seed, s, it, c, n):
    """Index in [0, n) from the first word of the START draw."""
    w = _draw(seed, s, it, c, STREAM_START, 0)[0]
    return (w * n) >> 32


class _Acc:
    """Running evidence and posterior moments in log space."""

    def __init__(self):
        self.m = -math.inf
        self.s0 = 0.0
        self.s1 = np.zeros(5)
        self.s2 = np.zeros(5)
        self.sl = 0.0

    def add(self, logw_l, theta, logl):
        if logw_l == -math.inf:
            return
        if logw_l > self.m:
            r = math.exp(self.m - logw_l) if self.m > -math.inf else 0.0
            self.s0 *= r
            self.s1 *= r
            self.s2 *= r
            self.sl *= r
            self.m = logw_l
        e = math.exp(logw_l - self.m)
        th = np.asarray(theta, np.float64)
        self.s0 += e
        self.s1 += e * th
        self.s2 += e * th * th
        self.sl += e * logl

    def log_z(self):
        return self.m + math.log(self.s0)


def _logl(o, b1, thetas):
    """log L = -chi^2 / 2 of one supernova at several parameter vectors."""
    n = len(thetas)
    b = SimpleNamespace(**vars(b1))
    b.par_off = np.array([0, n], np.int64)
    th = np.asarray(thetas, np.float64)
    b.z, b.t0, b.x0, b.x1, b.c = th[:, 0], th[:, 1], th[:, 2], th[:, 3], th[:, 4]
    x2 = o.chi2(b)
    return np.where(np.isfinite(x2), -0.5 * x2, -np.inf)


def run_one(o, batch, s, lower, upper, mask=DEFAULT_MASK, n_live=64, n_batch=16, n_steps=10,
            max_iter=100000, seed=1, dlogz=0.1):
    """Nested sampling of supernova s. Returns dict(logz, logz_err, mean, std,
    iterations, h)."""
    N, k, M = n_live, n_batch, n_steps
    ref = start_point(batch, s)
    free = [i for i in range(5) if (mask >> i) & 1]
    lo = np.where([(mask >> i) & 1 for i in range(5)], lower, ref)
    hi = np.where([(mask >> i) & 1 for i in range(5)], upper, ref)
    b1 = _one_sn(batch, s)
    live = np.empty((N, 5))
    for p in range(N):
        u = uniforms5(seed, s, 0, p, STREAM_INIT)
        live[p] = [lo[i] + u[i] * (hi[i] - lo[i]) if i in free else ref[i] for i in range(5)]
    live = _fp32(live)
    logl = _logl(o, b1, live)
    logx = 0.0
    acc = _Acc()
    f = 1.0
    it = 0
    while True:
        order = np.lexsort((np.arange(N), logl))  # by log L, ties by index
        z_now = acc.log_z() if acc.s0 > 0 else -math.inf
        remain = float(np.max(logl)) + logx
        if z_now > -math.inf and np.logaddexp(z_now, remain) - z_now < dlogz:
            break
        if it >= max_iter:
            break
        for j in range(k):
            n_alive = N - j
            logx_new = logx - 1.0 / n_alive
            logw = logx + math.log(-math.expm1(-1.0 / n_alive))
            p = order[j]
            acc.add(logw + logl[p], live[p], logl[p])
            logx = logx_new
        lstar = logl[order[k - 1]]
        surv = order[k:]
        sig = np.std(live[surv], axis=0)
        chains = np.array([live[surv[pick(seed, s, it, c, N - k)]] for c in range(k)])
        chain_l = np.array([logl[surv[pick(seed, s, it, c, N - k)]] for c in range(k)])
        n_acc = 0
        for m in range(M):
            prop = chains.copy()
            for c in range(k):
                nz = normals5(seed, s, it, m * k + c, STREAM_STEP)
                for i in free:
                    prop[c, i] = chains[c, i] + f * sig[i] * nz[i]
            prop = _fp32(prop)
            inbox = np.all((prop >= lo) & (prop <= hi), axis=1)
            lp = _logl(o, b1, prop)
            ok = inbox & (lp > lstar)
            chains[ok] = prop[ok]
            chain_l[ok] = lp[ok]
            n_acc += int(ok.sum())
        for c in range(k):
            live[order[c]] = chains[c]
            logl[order[c]] = chain_l[c]
        f = min(max(f * math.exp(n_acc / (k * M) - 0.5), 1e-3), 10.0)
        it += 1
    logw_live = logx - math.log(N)
    for p in range(N):
        acc.add(logw_live + logl[p], live[p], logl[p])
    logz = acc.log_z()
    h = acc.sl / acc.s0 - logz
    mean = acc.s1 / acc.s0
    var = np.maximum(acc.s2 / acc.s0 - mean * mean, 0.0)
    return dict(logz=logz, logz_err=math.sqrt(max(h, 0.0) / N), mean=mean, std=np.sqrt(var),
                iterations=it, h=h)


def _fp32(th):
    """The device evaluates z, x0, x1, c in FP32 (t0 in FP64): round the same."""
    th = np.array(th, np.float64)
    for i in (0, 2, 3, 4):
        th[..., i] = th[..., i].astype(np.float32).astype(np.float64)
    return th
