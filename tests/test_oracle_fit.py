"""Pins of the reference minimiser (scipy L-BFGS-B on the FP64 oracle chi^2,
oracle/fit.py) against facts that do not come from it: on noiseless data the
minimum is the truth; with only x0 free the minimum has the weighted
least-squares closed form; with a bound cutting off the unconstrained minimum
the result sits on the bound with the KKT sign conditions."""
import numpy as np
import pytest

import oracle
import oracle.fit as OF
import workloads as W
from tests import _helpers as H


@pytest.fixture(scope="module")
def noiseless():
    wl = W.config2(n_sn=3)
    o = H.with_oracle_flux(wl, noiseless=True)
    start = W.fit_start(wl.batch, np.random.default_rng(5))
    return wl, o, start


@pytest.fixture(scope="module")
def noisy():
    wl = W.config2(n_sn=3)
    o = H.with_oracle_flux(wl, seed=12)
    start = W.fit_start(wl.batch, np.random.default_rng(6))
    return wl, o, start


def test_noiseless_fit_recovers_the_truth(noiseless):
    wl, o, start = noiseless
    th, f, nit = OF.fit_batch(o, start)
    tb = W.truth_batch(wl.batch)
    truth = np.stack([tb.z, tb.t0, tb.x0, tb.x1, tb.c], axis=1).astype(np.float64)
    for s in range(start.n_sn):
        sc = OF.scales(OF.start_point(start, s))
        assert np.all(np.abs(th[s] - truth[s]) / sc <= 1e-5), (s, th[s], truth[s])
        assert f[s] <= 1e-8
        assert nit[s] > 1  # the start was away from the truth


def test_x0_only_fit_matches_the_weighted_least_squares_closed_form(noisy):
    wl, o, start = noisy
    th, f, _ = OF.fit_batch(o, start, mask=OF.MASK_X0)
    # bandflux is linear in x0: m = x0 * m1 with m1 the bandflux at x0 = 1
    for s in range(start.n_sn):
        lo, hi = start.obs_off[s], start.obs_off[s + 1]
        one = W.subset(start, [s])
        one.x0 = np.array([1.0])
        m1 = o.bandflux(one)
        sig = start.fluxerr[lo:hi].astype(np.float64)
        fl = start.flux[lo:hi].astype(np.float64)
        x0_star = np.sum(fl * m1 / sig**2) / np.sum(m1 * m1 / sig**2)
        assert abs(th[s, 2] - x0_star) <= 1e-8 * abs(x0_star)
        # the other parameters stay where they started
        assert np.array_equal(th[s, [0, 1, 3, 4]], OF.start_point(start, s)[[0, 1, 3, 4]])


def test_active_bound_satisfies_kkt(noisy):
    wl, o, start = noisy
    th_free, _, _ = OF.fit_batch(o, start)
    n = start.n_sn
    upper = np.full((n, 5), np.inf)
    upper[:, 4] = th_free[:, 4] - 0.05  # cut the colour below its unconstrained optimum
    th, f, _ = OF.fit_batch(o, start, upper=upper)
    for s in range(n):
        assert th[s, 4] == pytest.approx(upper[s, 4], abs=1e-12)
        b1 = OF._with_theta(OF._one_sn(start, s), th[s])
        _, g = o.chi2(b1, grad=True)
        sc = OF.scales(OF.start_point(start, s))
        gs = g[0] * sc
        assert gs[4] < 0  # chi^2 would fall by raising c past the bound
        assert np.all(np.abs(gs[[1, 2, 3]]) <= 1e-6 * np.abs(gs[4]) + 1e-6)
        assert f[s] > OF.chi2_at(o, start, th_free)[s]  # the bound costs chi^2
