"""Host logic of the benchmark (CPU): the algorithmic FLOP count behind
`roofline.achieved` against a brute-force count of the same definition, and
the error measures of `error_vs_oracle`."""
import numpy as np

import bench
import workloads as W


def _first_tap(i, n):
    return 0 if i == 0 else (n - 4 if i == n - 2 else i - 1)


def _brute_force_flops(wl, grad):
    """Per (sample, band): in-grid band samples, the distinct phase rows the
    band's observations touch (4 per in-grid observation) and the window of
    columns from the first to the last in-grid band sample's taps, counted one
    element at a time."""
    m, bt = wl.model, wl.batch
    kf, rc, cc, ob = ((bench.FLOP_K_GRAD, bench.FLOP_RC_GRAD, bench.FLOP_C_GRAD, bench.FLOP_OBS_GRAD) if grad
                      else (bench.FLOP_K_FWD, bench.FLOP_RC_FWD, 0, bench.FLOP_OBS_FWD))
    total = 0
    for s in range(bt.n_sn):
        for j in range(bt.par_off[s], bt.par_off[s + 1]):
            a = 1.0 / (1.0 + float(bt.z[j]))
            for b in range(len(wl.bands)):
                rows, n_obs_b = set(), 0
                for i in range(bt.obs_off[s], bt.obs_off[s + 1]):
                    if bt.band[i] != b:
                        continue
                    n_obs_b += 1
                    p = (bt.mjd[i] - bt.t0[j]) * a
                    if m.phase0 <= p <= m.phase_max:
                        iv = min(max(int(np.floor((p - m.phase0) / m.dphase)), 0), m.n_phase - 2)
                        f = _first_tap(iv, m.n_phase)
                        rows.update(range(f, f + 4))
                if n_obs_b == 0:
                    continue
                lr = [w * a for w in wl.bands[b].wave if m.wave0 <= w * a <= m.wave_max]
                cols = 0
                if lr:
                    ivs = [min(max(int(np.floor((x - m.wave0) / m.dwave)), 0), m.n_wave - 2) for x in (lr[0], lr[-1])]
                    cols = _first_tap(ivs[1], m.n_wave) + 3 - _first_tap(ivs[0], m.n_wave) + 1
                total += kf * len(lr) + rc * len(rows) * cols + cc * cols + ob * n_obs_b
    return total


def test_flop_count_matches_brute_force():
    for wl in (W.config1(), W.config2(n_sn=12), W.config3(n_sn=2, n_samples=3)):
        for grad in (True, False):
            assert bench.algorithmic_flops(wl, grad=grad) == _brute_force_flops(wl, grad)


def test_error_measures():
    wl = W.config2(n_sn=3)
    bt = wl.batch
    rng = np.random.default_rng(0)
    n_bf = bt.n_bandflux()
    ref = (rng.uniform(1, 2, bt.n_par), rng.normal(size=(bt.n_par, 5)), rng.uniform(1, 2, n_bf))
    same = bench.error_vs_oracle(bt, (ref[0].copy(), ref[1].astype(np.float32), ref[2].astype(np.float32)), ref)
    assert same["chi2_max_rel"] == 0.0 and same["bandflux_max_rel"] < 1e-7 and same["grad_max_scaled"] < 1e-6
    x2 = ref[0].copy()
    x2[1] *= 1 + 3e-4
    bf = ref[2].copy()
    bf[5] *= 1 + 2e-3
    worse = bench.error_vs_oracle(bt, (x2, ref[1], bf), ref)
    np.testing.assert_allclose(worse["chi2_max_rel"], 3e-4, rtol=1e-6)
    assert worse["bandflux_max_rel"] >= 2e-3 * 0.99


def test_sampled_oracle_pairs_and_errors(monkeypatch):
    """The CPU-baseline leg for batches too large for the oracle: the seeded
    pairs include the batch's first and last sample, each pair's bandfluxes
    are taken from the right positions of a full-batch bandflux array, and the
    error measures see exactly the planted differences. The library is
    replaced by the oracle's own full-batch results (no GPU)."""
    import contextlib
    import torch
    import oracle
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda *a: None)
    wl = W.config3(n_sn=5, n_samples=7)
    W.template_flux(wl.batch, np.random.default_rng(1))
    o = oracle.Oracle(wl.model, wl.bands)
    x2, g = o.chi2(wl.batch, grad=True)
    bf = o.bandflux(wl.batch)
    x2_bad = x2.copy()
    x2_bad[-1] *= 1 + 5e-4   # the last sample of the batch: always among the pairs

    class FakeLib:
        def chi2_grad(self, db):
            return torch.tensor(x2_bad), torch.tensor(g, dtype=torch.float32)

        def bandflux(self, db):
            return torch.tensor(bf, dtype=torch.float32)

    r = bench.sampled_oracle(wl, FakeLib(), None, None, n_picks=12)
    e = r["error_vs_oracle"]
    assert e["samples_compared"] >= 12 and r["kind"] == "oracle"
    np.testing.assert_allclose(e["chi2_max_rel"], 5e-4, rtol=1e-9)
    assert e["bandflux_max_rel"] < 1e-7 and e["grad_max_scaled"] < 1e-6
    # the same through the results of a timed step, with a sample budget
    r2 = bench.sampled_oracle(wl, FakeLib(), None, None, budget_s=0.05,
                              results=(torch.tensor(x2), torch.tensor(g, dtype=torch.float32)))
    assert r2["error_vs_oracle"]["chi2_max_rel"] == 0.0
    assert r2["error_vs_oracle"]["samples_compared"] >= 64 or \
        r2["error_vs_oracle"]["samples_compared"] == wl.batch.n_par
