"""Pins of the reference nested sampler (oracle/nested.py): the Philox4x32-10
generator against its published known-answer vectors, and the sampler's
evidence and posterior mean against the closed form of a case the model makes
Gaussian: with only x0 free the bandflux is linear in x0, so chi^2 is a
quadratic A x0^2 - 2 B x0 + C and, on a uniform prior [a, b],
Z = exp(-(C - B^2/A)/2) sqrt(pi/(2A)) [erf(sqrt(A/2)(b - mu)) - erf(sqrt(A/2)(a - mu))] / (b - a),
mu = B / A."""
import math

import numpy as np
import pytest

import oracle
import oracle.nested as NS
import oracle.fit as OF
import workloads as W
from tests import _helpers as H


@pytest.mark.parametrize("ctr,key,out", [
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
])
def test_philox_known_answers(ctr, key, out):
    assert NS.philox4x32_10(ctr, key) == out


def x0_closed_form(o, batch, s, a, b):
    """(log Z, posterior mean of x0) with only x0 free on the prior [a, b]."""
    lo, hi = batch.obs_off[s], batch.obs_off[s + 1]
    one = W.subset(batch, [s])
    one.x0 = np.array([1.0])
    m1 = o.bandflux(one)
    sig = batch.fluxerr[lo:hi].astype(np.float64)
    f = batch.flux[lo:hi].astype(np.float64)
    A = np.sum(m1 * m1 / sig**2)
    B = np.sum(f * m1 / sig**2)
    C = np.sum(f * f / sig**2)
    mu = B / A
    r = math.sqrt(A / 2.0)
    logz = -(C - B * B / A) / 2.0 + 0.5 * math.log(math.pi / (2.0 * A)) \
        + math.log(math.erf(r * (b - mu)) - math.erf(r * (a - mu))) - math.log(b - a)
    return logz, mu, 1.0 / math.sqrt(A)


@pytest.fixture(scope="module")
def one_sn():
    wl = W.config2(n_sn=12)
    n = np.diff(wl.batch.obs_off)
    wl.batch = W.subset(wl.batch, list(np.argsort(n)[:2]))  # the two shortest light curves
    o = H.with_oracle_flux(wl, seed=31)
    return wl, o


def test_x0_only_evidence_and_mean_match_the_closed_form(one_sn):
    wl, o = one_sn
    bt = wl.batch
    for s in range(bt.n_sn):
        x0 = float(bt.x0[s])
        a, b = 0.5 * x0, 1.5 * x0
        logz, mu, sd = x0_closed_form(o, bt, s, a, b)
        lower = np.full(5, -np.inf)
        upper = np.full(5, np.inf)
        lower[2], upper[2] = a, b
        r = NS.run_one(o, bt, s, lower, upper, mask=OF.MASK_X0, n_live=96, n_batch=24, n_steps=8,
                       seed=7 + s)
        assert abs(r["logz"] - logz) <= 4 * r["logz_err"] + 0.05, (r, logz)
        assert abs(r["mean"][2] - mu) <= 0.2 * sd, (r["mean"][2], mu, sd)
        assert r["std"][2] == pytest.approx(sd, rel=0.3)
