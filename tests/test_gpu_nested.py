"""GPU nested sampling (salt_nested) against the closed-form evidence of the
x0-only (Gaussian) case and against the reference sampler on the FP64 oracle
(oracle/nested.py, same algorithm and Philox streams; FP32 versus FP64 chi^2
makes the runs diverge, so the comparison is statistical: within the sum of
the two runs' log Z errors, sqrt(H / N) each)."""
import math

import numpy as np
import pytest

import oracle
import oracle.fit as OF
import oracle.nested as NS
import workloads as W
from tests import _helpers as H
from tests.test_oracle_nested import x0_closed_form

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _salt(wl):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    return Salt(wl.model, wl.bands)


@pytest.fixture(scope="module")
def short():
    wl = W.config2(n_sn=40)
    n = np.diff(wl.batch.obs_off)
    wl.batch = W.subset(wl.batch, list(np.argsort(n)[:6]))  # six short light curves
    o = H.with_oracle_flux(wl, seed=41)
    return wl, o


def _box(bt, mask, widths):
    n = bt.n_sn
    lo = np.full((n, 5), -np.inf)
    hi = np.full((n, 5), np.inf)
    ref = np.stack([bt.z, bt.t0, bt.x0, bt.x1, bt.c], axis=1).astype(np.float64)
    for i, (a, b) in widths.items():
        lo[:, i] = a(ref[:, i])
        hi[:, i] = b(ref[:, i])
    return lo, hi


def _run(wl, lo, hi, **kw):
    s = _salt(wl)
    db = s.upload(wl.batch)
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=s.device).contiguous()
    out = s.nested(db, T(lo), T(hi), **kw)
    s.check()
    return [t.cpu().numpy() for t in out]


def test_x0_only_evidence_matches_the_closed_form(short):
    wl, o = short
    bt = wl.batch
    lo, hi = _box(bt, OF.MASK_X0, {2: (lambda v: 0.5 * v, lambda v: 1.5 * v)})
    logz, err, mean, std, st = _run(wl, lo, hi, free_mask=OF.MASK_X0, n_live=256, n_batch=64,
                                    n_steps=12, seed=3)
    assert np.all(st >= 0), st
    for s in range(bt.n_sn):
        lz, mu, sd = x0_closed_form(o, bt, s, lo[s, 2], hi[s, 2])
        assert abs(logz[s] - lz) <= 4 * err[s] + 0.05, (s, logz[s], lz, err[s])
        assert abs(mean[s, 2] - mu) <= 0.2 * sd, (s, mean[s, 2], mu, sd)
        assert std[s, 2] == pytest.approx(sd, rel=0.25)


def test_four_parameters_agree_with_the_reference_sampler(short):
    wl, o = short
    bt = W.subset(wl.batch, [0, 1])
    wl2 = W.Workload(wl.name, wl.model, wl.bands, bt)
    widths = {1: (lambda v: v - 5.0, lambda v: v + 5.0), 2: (lambda v: 0.5 * v, lambda v: 1.5 * v),
              3: (lambda v: v * 0 - 3.0, lambda v: v * 0 + 3.0), 4: (lambda v: v * 0 - 0.3, lambda v: v * 0 + 0.3)}
    lo, hi = _box(bt, OF.DEFAULT_MASK, widths)
    kw = dict(n_live=96, n_batch=24, n_steps=8)
    logz, err, mean, std, st = _run(wl2, lo, hi, seed=11, **kw)
    assert np.all(st >= 0), st
    for s in range(bt.n_sn):
        r = NS.run_one(o, bt, s, lo[s], hi[s], seed=11, **kw)
        tol = 4 * math.hypot(err[s], r["logz_err"]) + 0.1
        assert abs(logz[s] - r["logz"]) <= tol, (s, logz[s], r["logz"], tol)
        for i in (1, 2, 3, 4):
            assert abs(mean[s, i] - r["mean"][i]) <= 0.5 * max(std[s, i], r["std"][i]), (s, i)


def test_a_seed_reproduces_a_run_and_bad_inputs_are_refused(short):
    from paper_2504_08081_b300 import _abi
    wl, o = short
    bt = wl.batch
    lo, hi = _box(bt, OF.MASK_X0, {2: (lambda v: 0.5 * v, lambda v: 1.5 * v)})
    a = _run(wl, lo, hi, free_mask=OF.MASK_X0, n_live=64, n_batch=16, n_steps=6, seed=5)
    b = _run(wl, lo, hi, free_mask=OF.MASK_X0, n_live=64, n_batch=16, n_steps=6, seed=5)
    c = _run(wl, lo, hi, free_mask=OF.MASK_X0, n_live=64, n_batch=16, n_steps=6, seed=6)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a[0], c[0])
    lo2, hi2 = lo.copy(), hi.copy()
    lo2[1, 2], hi2[1, 2] = hi[1, 2], lo[1, 2]  # empty box for SN 1
    r = _run(wl, lo2, hi2, free_mask=OF.MASK_X0, n_live=64, n_batch=16, n_steps=6, seed=5)
    assert r[4][1] == _abi.SALT_FIT_INVALID and np.all(np.delete(r[4], 1) >= 0)
    wl3 = W.config3(n_sn=2, n_samples=3)
    s3 = _salt(wl3)
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=s3.device).contiguous()
    with pytest.raises(_abi.SaltError):
        s3.nested(s3.upload(wl3.batch), T(np.zeros((2, 5))), T(np.ones((2, 5))))
