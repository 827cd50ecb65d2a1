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
