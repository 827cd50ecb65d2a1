"""Serving engine (continuous batching) through salt_serve_submit/poll/cancel:
results match the batch API and the oracle, are identical alone and in a mix,
memory admission completes a stream larger than the budget, and invalid,
oversized and cancelled requests get their status codes."""
import numpy as np
import pytest

import workloads as W
from tests import _helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _salt(wl, **kw):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    return Salt(wl.model, wl.bands, **kw)


@pytest.fixture(scope="module")
def stream():
    wl = W.config4(n_req=120, seed=4321)
    return wl


def _submit(s, rq):
    b = rq.batch
    return s.submit(b.n_obs, b.mjd, b.band, b.flux, b.fluxerr, b.zp, b.t0, b.z, b.x0, b.x1, b.c,
                    rq.want_grad)


def _result(s, tk, rq):
    rc, x2, g = s.poll(tk, rq.batch.n_par, rq.want_grad, wait_ms=60000)
    assert rc == 0, rc
    return x2, g


def test_alone_and_in_mix_identical(stream):
    reqs = stream.requests
    s = _salt(stream, serve_mem_bytes=256 << 20)
    probe = [3, 17, 42, 99]
    alone = {}
    for i in probe:
        alone[i] = _result(s, _submit(s, reqs[i]), reqs[i])
    tks = [_submit(s, rq) for rq in reqs]
    mixed = {i: _result(s, tks[i], reqs[i]) for i in range(len(reqs))}
    for i in probe:
        np.testing.assert_array_equal(alone[i][0], mixed[i][0])
        if reqs[i].want_grad:
            np.testing.assert_array_equal(alone[i][1], mixed[i][1])
    st = s.serve_stats()
    assert st["completed"] == len(reqs) + len(probe)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    s.close()


def test_serving_matches_batch_api(stream):
    reqs = stream.requests[:30]
    s = _salt(stream, serve_mem_bytes=128 << 20)
    tks = [_submit(s, rq) for rq in reqs]
    for rq, tk in zip(reqs, tks):
        x2, g = _result(s, tk, rq)
        db = s.upload(rq.batch)
        bx2, bg = s.chi2_grad(db)
        np.testing.assert_allclose(x2, bx2.cpu().numpy(), rtol=1e-6)
        if rq.want_grad:
            np.testing.assert_allclose(g, bg.cpu().numpy(), rtol=1e-5,
                                       atol=1e-5 * float(np.abs(bg.cpu().numpy()).max()))
    s.close()


def test_serving_matches_oracle():
    wl = W.config3(n_sn=3, n_samples=70, seed=99)
    o = H.with_oracle_flux(wl)
    s = _salt(wl, serve_mem_bytes=64 << 20)
    for sn in range(3):
        sub = W.subset(wl.batch, [sn])
        rq = W.Request(arrival_s=0.0, want_grad=True, batch=sub)
        x2, g = _result(s, _submit(s, rq), rq)
        ref_x2, ref_g = o.chi2(sub, grad=True)
        H.assert_chi2_close(sub, x2, ref_x2, o.bandflux(sub))
        H.assert_grad_close(sub, g, ref_g, o=o)
    s.close()


def test_admission_under_small_budget(stream):
    # a budget far below the stream's total forces requests to wait for memory
    reqs = stream.requests
    s = _salt(stream, serve_mem_bytes=4 << 20)
    tks = []
    for rq in reqs:
        try:
            tks.append((rq, _submit(s, rq)))
        except Exception as ex:  # a request larger than the whole budget
            assert getattr(ex, "code", None) == -2
    for rq, tk in tks:
        _result(s, tk, rq)
    st = s.serve_stats()
    assert st["completed"] == len(tks) and st["mem_in_use"] == 0
    s.close()


def test_invalid_oversized_cancelled_and_unknown(stream):
    from paper_2504_08081_b300 import SaltError
    rq = stream.requests[5]
    s = _salt(stream, serve_mem_bytes=1 << 20)
    b = rq.batch
    bad_band = b.band.copy()
    bad_band[0] = 99
    with pytest.raises(SaltError) as ei:
        s.submit(b.n_obs, b.mjd, bad_band, b.flux, b.fluxerr, b.zp, b.t0, b.z, b.x0, b.x1, b.c, False)
    assert ei.value.code == -1
    big = np.ones(200000)
    with pytest.raises(SaltError) as ei:
        s.submit(b.n_obs, b.mjd, b.band, b.flux, b.fluxerr, b.zp, 55000.0 + big, 0.1 * big,
                 1e-5 * big, 0 * big, 0 * big, False)
    assert ei.value.code == -2
    tk = _submit(s, rq)
    s.cancel(tk)
    rc, _, _ = s.poll(tk, b.n_par, rq.want_grad, wait_ms=60000)
    assert rc in (0, -6)
    rc, _, _ = s.poll(tk, b.n_par, rq.want_grad, wait_ms=0)
    assert rc == -5  # released after it was collected
    s.close()


def test_burst_with_cancels_accounts_for_every_request():
    """A burst of 20 000 requests under a 64 MB budget with 2 % cancelled right
    after submission: every request ends DONE or CANCELLED, the counters add
    up, the arenas drain back to empty, and sampled results agree with the
    batch API's on the same request (to FP32 summation order: the batch call
    may pick another kernel family or tile)."""
    import ctypes as C
    from paper_2504_08081_b300 import _abi, serving as SV
    wl = W.config4(n_req=20000, seed=4242)
    reqs = wl.requests
    s = _salt(wl, serve_mem_bytes=64 << 20)
    prep = SV._prepared(reqs)
    L = _abi.lib()
    rng = np.random.default_rng(1)
    cancel = rng.random(len(reqs)) < 0.02
    tks = []
    for i in range(len(reqs)):
        req, _, _, _, tk = prep[i]
        assert L.salt_serve_submit(s.ctx.h, C.byref(req), C.byref(tk)) == _abi.SALT_OK
        tks.append(tk.value)
        if cancel[i]:
            L.salt_serve_cancel(s.ctx.h, tk.value)
    n_ok = n_cancel = 0
    for i in range(len(reqs)):
        _, _, chi2, grad, _ = prep[i]
        rc = L.salt_serve_poll(s.ctx.h, tks[i], 60000, chi2.ctypes.data,
                               grad.ctypes.data if grad is not None else None)
        assert rc in (_abi.SALT_OK, _abi.SALT_ERR_CANCELLED), (i, rc)
        n_ok += rc == _abi.SALT_OK
        n_cancel += rc == _abi.SALT_ERR_CANCELLED
    st = s.serve_stats()
    assert n_ok + n_cancel == len(reqs) and n_cancel <= int(cancel.sum())
    assert st["completed"] == n_ok and st["submitted"] == len(reqs)
    assert st["queued"] == 0 and st["active"] == 0 and st["mem_in_use"] == 0
    for i in [i for i in rng.choice(len(reqs), 200, replace=False) if not cancel[i]][:100]:
        x2, g = s.chi2_grad(s.upload(reqs[i].batch, plan=False))
        np.testing.assert_allclose(prep[i][2], x2.cpu().numpy(), rtol=1e-6)
        if reqs[i].want_grad:
            ref = g.cpu().numpy()
            scale = np.abs(ref).max(axis=1, keepdims=True)
            assert np.all(np.abs(prep[i][3] - ref) <= 1e-5 * scale)
    s.close()


def test_native_client_replay_and_plain(stream):
    """The native load generator (salt_client.h): a replay submitted all at
    once and one on Poisson arrivals give bitwise the results the engine gives
    through the Python client, every request completes, and the plain
    per-request loop over the C ABI runs the same requests."""
    from paper_2504_08081_b300 import serving as SV
    reqs = stream.requests
    s = _salt(stream, serve_mem_bytes=256 << 20)
    ref = {}
    for i in (0, 7, 33, 119):
        ref[i] = _result(s, _submit(s, reqs[i]), reqs[i])
    for arrivals in (None, np.cumsum(np.random.default_rng(5).exponential(1e-4, len(reqs)))):
        wall, res, st, cs = SV.replay_native(s, reqs, arrivals, collect=True)
        assert cs["completed"] == len(reqs) and wall > 0 and cs["client_p99_ms"] >= cs["client_p50_ms"] > 0
        for i, (x2, g) in ref.items():
            np.testing.assert_array_equal(res[i][0], x2)
            if reqs[i].want_grad:
                np.testing.assert_array_equal(res[i][1], g)
    k, wall, p50, p99 = SV.plain_native(s, reqs, limit_s=30.0)
    assert k == len(reqs) and p99 >= p50 > 0
    s.close()
