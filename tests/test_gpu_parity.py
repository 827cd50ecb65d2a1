"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs, element by element.

Tolerances: bandflux 1e-5 relative (floor 1e-3 of the supernova's largest
bandflux); chi^2 within the bound that 1e-5 relative bandflux errors
propagate to; gradient 1e-3 of the scaled gradient's inf-norm per sample, or
(a sum with cancellation near a minimum) the bound those bandflux errors
propagate to (tests/_helpers.grad_bound)."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import _helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KERNELS = {"direct": 1, "factorised": 2, "bandwarp": 3, "unit": 4, "auto": 0}


def _salt(wl, **kw):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    return Salt(wl.model, wl.bands, **kw)


@pytest.fixture(scope="module")
def cfg1():
    wl = W.config1()
    o = H.with_oracle_flux(wl)
    return wl, o


@pytest.fixture(scope="module")
def cfg2_sub():
    wl = W.config2(n_sn=160)
    o = H.with_oracle_flux(wl)
    return wl, o


@pytest.fixture(scope="module")
def cfg3_sub():
    wl = W.config3(n_sn=6, n_samples=40)
    o = H.with_oracle_flux(wl)
    return wl, o


@pytest.fixture(scope="module")
def cfg5_sub():
    wl = W.config5(n_sn=60, n_samples=19)
    o = H.with_oracle_flux(wl)
    return wl, o


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_bandflux_single_supernova(cfg1, kernel):
    wl, o = cfg1
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(wl.batch)
    got = s.bandflux(db).cpu().numpy()
    ref = o.bandflux(wl.batch)
    H.assert_bandflux_close(wl.batch, got, ref)
    s.check()


@pytest.mark.parametrize("kernel", ["direct", "factorised", "bandwarp", "unit"])
@pytest.mark.parametrize("tile", [1, 2, 4, 8, 16])
def test_bandflux_and_chi2_batched(cfg2_sub, kernel, tile):
    wl, o = cfg2_sub
    bt = wl.batch
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    s.set_tile(tile)
    db = s.upload(bt)
    bf = s.bandflux(db).cpu().numpy()
    ref_bf = o.bandflux(bt)
    H.assert_bandflux_close(bt, bf, ref_bf)
    x2 = s.chi2(db).cpu().numpy()
    H.assert_chi2_close(bt, x2, o.chi2(bt), ref_bf)
    s.check()


@pytest.mark.parametrize("kernel", ["direct", "factorised", "bandwarp", "unit", "auto"])
@pytest.mark.parametrize("tile", [1, 2, 8])
def test_chi2_grad_many_samples(cfg3_sub, kernel, tile):
    wl, o = cfg3_sub
    bt = wl.batch
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    s.set_tile(tile)
    db = s.upload(bt)
    x2, g = s.chi2_grad(db)
    x2, g = x2.cpu().numpy(), g.cpu().numpy()
    ref_x2, ref_g = o.chi2(bt, grad=True)
    ref_bf = o.bandflux(bt)
    H.assert_chi2_close(bt, x2, ref_x2, ref_bf)
    H.assert_grad_close(bt, g, ref_g, o=o, bf_ref=ref_bf)
    # the chi^2 of the gradient call agrees with the chi^2-only call (separately
    # compiled variants: equal up to FP32 contraction order)
    x2b = s.chi2(db).cpu().numpy()
    H.assert_chi2_close(bt, x2b, ref_x2, ref_bf)
    np.testing.assert_allclose(x2, x2b, rtol=1e-5)
    s.check()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_large_grid_ragged(cfg5_sub, kernel):
    wl, o = cfg5_sub
    bt = wl.batch
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(bt)
    bf = s.bandflux(db).cpu().numpy()
    ref_bf = o.bandflux(bt)
    H.assert_bandflux_close(bt, bf, ref_bf)
    x2, g = s.chi2_grad(db)
    ref_x2, ref_g = o.chi2(bt, grad=True)
    H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
    s.check()


def test_factorised_matches_direct_kernel(cfg3_sub):
    wl, o = cfg3_sub
    s = _salt(wl)
    db = s.upload(wl.batch)
    s.set_kernel(1)
    a = s.bandflux(db).cpu().numpy().astype(np.float64)
    s.set_kernel(2)
    b = s.bandflux(db).cpu().numpy().astype(np.float64)
    H.assert_bandflux_close(wl.batch, b, a, rtol=2e-5)


def test_bitwise_reproducible(cfg3_sub):
    wl, _ = cfg3_sub
    s = _salt(wl)
    db = s.upload(wl.batch)
    x2a, ga = s.chi2_grad(db)
    outs = [s.chi2_grad(db) for _ in range(3)]
    for x2, g in outs:
        assert torch.equal(x2, x2a) and torch.equal(g, ga)
    bfa = s.bandflux(db)
    assert torch.equal(s.bandflux(db), bfa)


@pytest.mark.parametrize("kernel", ["direct", "factorised", "bandwarp", "unit"])
def test_bitwise_reproducible_per_kernel(cfg2_sub, kernel):
    """Every kernel family gives bitwise the same results call after call,
    whatever order its warps or blocks finish in (fixed summation orders; the
    warp-unit kernel combines per-band partials in band order)."""
    wl, _ = cfg2_sub
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(wl.batch)
    x2a, ga = (t.clone() for t in s.chi2_grad(db))
    bfa = s.bandflux(db).clone()
    for _ in range(5):
        x2, g = s.chi2_grad(db)
        assert torch.equal(x2, x2a) and torch.equal(g, ga)
        assert torch.equal(s.bandflux(db), bfa)
    s.check()


# ------------------------------------------------------------------ edge cases

def _edge_workload():
    """Supernovae exercising the degenerate cases: no observations, no samples,
    one observation, a 2-sample band, a band partly outside the grid at the
    sample's z, phases outside the grid, samples at grid nodes and at the
    colour-law boundaries."""
    rng = np.random.default_rng(77)
    model = W.make_model(rng)
    bands = [W.gaussian_band(5500.0, 201), W.Band(wave=np.array([6000.0, 6400.0]),
                                                  trans=np.array([0.7, 1.0])),
             W.tophat_band(2900.0, 3300.0), W.gaussian_band(8600.0, 241),
             W.tophat_band(6900.0, 7100.0, 2.5)]
    n_obs = [0, 5, 1, 12, 7, 30]
    n_par = [3, 0, 1, 4, 5, 9]
    z = [0.05, 0.2, 0.004, 0.3, 0.1, 0.02]
    bt = W.make_batch(rng, model, bands, n_obs, z, n_par, perturb=W.PERTURB)
    # assign bands explicitly (all of them valid ids)
    bt.band[:] = rng.integers(0, len(bands), size=bt.n_obs).astype(np.int32)
    # supernova 3: phases beyond both ends of the grid for some observations
    lo, hi = bt.obs_off[3], bt.obs_off[4]
    bt.mjd[lo:lo + 3] = bt.t0[bt.par_off[3]] + np.array([-40.0, 80.0, 51.0 * 1.3])
    # supernova 4: z = 0 sample, epochs on grid nodes, rest wavelength at the
    # colour-law boundaries and at a grid node
    p4 = bt.par_off[4]
    bt.z[p4] = 0.0
    lo = bt.obs_off[4]
    bt.mjd[lo:lo + 3] = bt.t0[p4] + np.array([0.0, 7.0, -20.0])
    bt.band[lo:lo + 3] = np.array([4, 4, 2], dtype=np.int32)
    wl = W.Workload("edge", model, bands, bt)
    return wl


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_edge_cases(kernel):
    wl = _edge_workload()
    o = H.with_oracle_flux(wl)
    bt = wl.batch
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(bt)
    ref_bf = o.bandflux(bt)
    bf = s.bandflux(db).cpu().numpy()
    H.assert_bandflux_close(bt, bf, ref_bf)
    x2, g = s.chi2_grad(db)
    ref_x2, ref_g = o.chi2(bt, grad=True)
    H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf, max_fallback=0)
    # supernova 0 has no observations: chi^2 = 0 and zero gradient exactly
    p0 = slice(bt.par_off[0], bt.par_off[1])
    assert np.all(x2.cpu().numpy()[p0] == 0.0) and np.all(g.cpu().numpy()[p0] == 0.0)
    s.check()


def _grid_end_workload():
    """Observations whose rest-frame phases fall in the first and last days of
    the phase grid, where the surface tapers steeply, at z up to 2 and epochs
    near 55 000 d: per supernova 8 phases in [-20, -17] d, 8 in [46, 50] d and
    8 anywhere on the grid; samples perturbed by 0.3 d in t0 and 0.002 in z,
    so some of their phases leave the grid."""
    rng = np.random.default_rng(2504)
    model = W.make_model(rng, wave_max=11000.0)
    bands = [W.gaussian_band(c, 201) for c in 3700.0 + 900.0 * np.arange(8)]
    n_sn = 48
    z = rng.uniform(0.01, 2.0, n_sn)
    bt = W.make_batch(rng, model, bands, np.full(n_sn, 24), z, np.full(n_sn, 6),
                      perturb=dict(z=0.002, t0=0.3, logx0=0.02, x1=0.1, c=0.01))
    for s in range(n_sn):
        ph = np.sort(np.concatenate([rng.uniform(-20.0, -17.0, 8), rng.uniform(46.0, 50.0, 8),
                                     rng.uniform(-20.0, 50.0, 8)]))
        zt = float(bt.truth["z"][s])
        bt.mjd[bt.obs_off[s]:bt.obs_off[s + 1]] = bt.truth["t0"][s] + ph * (1.0 + zt)
    return W.Workload("grid_ends", model, bands, bt)


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_phases_at_the_grid_ends(kernel):
    """The phase coordinate is formed to ~1e-10 d (a float pair), so the steep
    ends of the surface see no rounding of epochs ~5e4 d: bandfluxes there
    stay within the tolerance (1.7e-6 measured; an FP32 phase gave 1.3e-4),
    chi^2 and gradients too."""
    wl = _grid_end_workload()
    o = H.with_oracle_flux(wl)
    bt = wl.batch
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(bt)
    ref_bf = o.bandflux(bt)
    H.assert_bandflux_close(bt, s.bandflux(db).cpu().numpy(), ref_bf)
    x2, g = s.chi2_grad(db)
    ref_x2, ref_g = o.chi2(bt, grad=True)
    H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
    s.check()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_many_samples_one_supernova(kernel):
    wl = W.config3(n_sn=1, n_samples=4096)
    o = H.with_oracle_flux(wl)
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(wl.batch)
    x2, g = s.chi2_grad(db)
    idx = np.random.default_rng(3).choice(4096, 64, replace=False)
    sub = W.Batch(obs_off=wl.batch.obs_off, mjd=wl.batch.mjd, band=wl.batch.band,
                  flux=wl.batch.flux, fluxerr=wl.batch.fluxerr, zp=wl.batch.zp,
                  par_off=np.array([0, len(idx)], dtype=np.int64), t0=wl.batch.t0[idx],
                  z=wl.batch.z[idx], x0=wl.batch.x0[idx], x1=wl.batch.x1[idx], c=wl.batch.c[idx])
    ref_x2, ref_g = o.chi2(sub, grad=True)
    H.assert_chi2_close(sub, x2.cpu().numpy()[idx], ref_x2, o.bandflux(sub))
    H.assert_grad_close(sub, g.cpu().numpy()[idx], ref_g, o=o, max_fallback=0)


def test_invalid_data_is_reported():
    from paper_2504_08081_b300 import SaltError
    wl = W.config2(n_sn=5)
    H.with_oracle_flux(wl)
    s = _salt(wl)
    bt = wl.batch
    bt.band = bt.band.copy()
    bt.band[3] = 17  # out of range
    db = s.upload(bt)
    with pytest.raises(SaltError) as ei:
        s.chi2(db, validate=True)
    assert ei.value.code == -1
    x2 = s.chi2(db).cpu().numpy()
    assert np.isnan(x2[0]) and np.all(np.isfinite(x2[1:]))
    with pytest.raises(SaltError) as ei:
        s.check()
    assert ei.value.code == -7
    s.check()  # the sticky flag was cleared


def test_autograd_function(cfg3_sub):
    from paper_2504_08081_b300.torch_api import SaltChi2
    wl, o = cfg3_sub
    s = _salt(wl)
    db = s.upload(wl.batch)
    z = db.t["z"].clone().requires_grad_(True)
    t0 = db.t["t0"].clone().requires_grad_(True)
    x0 = db.t["x0"].clone().requires_grad_(True)
    x1 = db.t["x1"].clone().requires_grad_(True)
    c = db.t["c"].clone().requires_grad_(True)
    x2 = SaltChi2.apply(s, db, z, t0, x0, x1, c)
    w = torch.linspace(0.5, 1.5, x2.numel(), device=x2.device, dtype=x2.dtype)
    (x2 * w).sum().backward()
    _, g = s.chi2_grad(db)
    wf = w.float()[:, None]
    for q, t in enumerate((z, t0, x0, x1, c)):
        torch.testing.assert_close(t.grad.float(), (g * wf)[:, q], rtol=1e-6, atol=0)


def test_gradient_against_central_differences_on_gpu(cfg3_sub):
    # the GPU adjoint against central differences of the GPU chi^2 in all five
    # parameters, with the step the oracle's own check uses:
    # h = 1e-4 max(|theta|, s_theta), s = (0.01, -, |x0|, 1, 0.1), and for t0
    # (an epoch) h = 1e-4 day. The perturbed FP32 parameters are rounded, so
    # the divisor is the difference of the values actually evaluated. FP32
    # photometry makes single differences noisy (the chi^2 resolves ~1e-6
    # relative), hence the median criterion.
    wl, _ = cfg3_sub
    s = _salt(wl)
    db = s.upload(wl.batch)
    _, g = s.chi2_grad(db)
    g = g.cpu().numpy().astype(np.float64)
    for q, name in enumerate(("z", "t0", "x0", "x1", "c")):
        base = db.t[name]
        if name == "t0":
            h = torch.full_like(base, 1e-4)
        else:
            sc = base.abs() if name == "x0" else torch.full_like(base, H.SCALES[q])
            h = 1e-4 * torch.maximum(base.abs(), sc)
        up, dn = base + h, base - h
        xp = s.chi2(db.with_params(**{name: up})).double()
        xm = s.chi2(db.with_params(**{name: dn})).double()
        fd = ((xp - xm) / (up.double() - dn.double())).cpu().numpy()
        scale = np.abs(g[:, q]) + 1e-2 * np.abs(g[:, q]).max() + 1e-300
        rel = np.abs(fd - g[:, q]) / scale
        assert np.median(rel) < 1e-2, (name, float(np.median(rel)))


def _crowded_workload():
    """Supernovae whose observations overflow every kernel's per-pass caches:
    700 observations in one band (several observation passes and chunks),
    130 split over two bands, and a 1-sample supernova with 200 observations
    in one band."""
    rng = np.random.default_rng(91)
    model = W.make_model(rng)
    bands = [W.gaussian_band(5000.0, 181), W.gaussian_band(6500.0, 221)]
    n_obs = [700, 130, 200]
    n_par = [5, 3, 1]
    z = [0.08, 0.3, 0.15]
    bt = W.make_batch(rng, model, bands, n_obs, z, n_par, perturb=W.PERTURB)
    bt.band[:] = 0
    lo, hi = bt.obs_off[1], bt.obs_off[2]
    bt.band[lo:hi] = rng.integers(0, 2, size=hi - lo).astype(np.int32)
    return W.Workload("crowded", model, bands, bt)


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_observation_passes_overflowing_the_caches(kernel):
    wl = _crowded_workload()
    o = H.with_oracle_flux(wl)
    bt = wl.batch
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(bt)
    ref_bf = o.bandflux(bt)
    H.assert_bandflux_close(bt, s.bandflux(db).cpu().numpy(), ref_bf)
    x2, g = s.chi2_grad(db)
    ref_x2, ref_g = o.chi2(bt, grad=True)
    H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
    s.check()


def _empty_like(bt, n_obs_per_sn, n_par_per_sn):
    """A batch with the given per-supernova observation and sample counts,
    arrays filled from bt's first entries (bt must hold enough of them)."""
    oo = np.concatenate([[0], np.cumsum(n_obs_per_sn)]).astype(np.int64)
    po = np.concatenate([[0], np.cumsum(n_par_per_sn)]).astype(np.int64)
    no, npar = int(oo[-1]), int(po[-1])
    return W.Batch(obs_off=oo, mjd=bt.mjd[:no].copy(), band=bt.band[:no].copy(), flux=bt.flux[:no].copy(),
                   fluxerr=bt.fluxerr[:no].copy(), zp=bt.zp[:no].copy(), par_off=po, t0=bt.t0[:npar].copy(),
                   z=bt.z[:npar].copy(), x0=bt.x0[:npar].copy(), x1=bt.x1[:npar].copy(), c=bt.c[:npar].copy())


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_empty_batches(kernel):
    """No supernovae; supernovae without samples; supernovae without
    observations: every call succeeds, with chi^2 = 0 and a zero gradient
    where there are samples but nothing to compare."""
    wl = W.config2(n_sn=4)
    H.with_oracle_flux(wl)
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    for n_obs, n_par in (([], []), ([10, 0, 7], [0, 0, 0]), ([0, 0], [3, 1])):
        bt = _empty_like(wl.batch, n_obs, n_par)
        for plan in (True, False):
            db = s.upload(bt, plan=plan)
            x2, g = s.chi2_grad(db)
            bf = s.bandflux(db)
            x2c = s.chi2(db)
            assert x2.shape == (bt.n_par,) and g.shape == (bt.n_par, 5) and bf.numel() == 0
            assert bool((x2 == 0).all()) and bool((g == 0).all()) and bool((x2c == 0).all())
    s.check()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_maximum_grid(kernel):
    """The largest grid a context takes: 256 phase nodes (0.27 d apart, so an
    observation season touches ~220 rows) by 2001 wavelength nodes (5 A).
    The warp kernels (at most 128 phase nodes) refuse it when forced; the
    autotuner leaves them out."""
    from paper_2504_08081_b300 import SaltError
    rng = np.random.default_rng(5)
    model = W.make_model(rng, wave_max=12000.0, phase=(-20.0, 50.0, 70.0 / 255.0), dwave=5.0)
    assert model.n_phase == 256 and model.n_wave == 2001
    bands = [W.gaussian_band(4500.0, 201), W.gaussian_band(6500.0, 281), W.gaussian_band(9000.0, 301)]
    n_obs = [60, 45, 30, 52]
    n_par = [3, 9, 1, 4]
    bt = W.make_batch(rng, model, bands, n_obs, [0.05, 0.3, 0.6, 0.15], n_par, perturb=W.PERTURB)
    wl = W.Workload("maxgrid", model, bands, bt)
    o = H.with_oracle_flux(wl)
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(bt)
    if kernel in ("unit", "bandwarp"):
        with pytest.raises(SaltError):
            s.chi2_grad(db)
        return
    ref_bf = o.bandflux(bt)
    H.assert_bandflux_close(bt, s.bandflux(db).cpu().numpy(), ref_bf)
    x2, g = s.chi2_grad(db)
    ref_x2, ref_g = o.chi2(bt, grad=True)
    H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
    s.check()


def test_grid_beyond_the_maximum_is_refused():
    from paper_2504_08081_b300 import SaltError
    rng = np.random.default_rng(6)
    model = W.make_model(rng, phase=(-20.0, 50.0, 70.0 / 256.0))
    assert model.n_phase == 257
    with pytest.raises(SaltError):
        _salt(W.Workload("toolarge", model, [W.gaussian_band(5000.0, 201)], None))


def test_fp32_overflow_is_reported():
    """A colour factor beyond the FP32 range (c = 60 at a rest wavelength where
    CL is about -2: 10^(48) and more) gives a non-finite bandflux; salt_check
    reports it as SALT_ERR_DATA and clears the flag, and the other samples are
    unaffected."""
    from paper_2504_08081_b300 import SaltError
    wl = W.config2(n_sn=6)
    o = H.with_oracle_flux(wl)
    bt = wl.batch
    bt.c = bt.c.copy()
    bt.c[2] = np.float32(60.0)
    s = _salt(wl)
    db = s.upload(bt)
    x2, g = s.chi2_grad(db)
    x2 = x2.cpu().numpy()
    assert not np.isfinite(x2[2])
    with pytest.raises(SaltError) as ei:
        s.check()
    assert ei.value.code == -7 and "not finite" in str(ei.value)
    s.check()  # cleared
    others = np.arange(bt.n_par) != 2
    ref_x2 = o.chi2(bt)
    assert np.all(np.isfinite(x2[others]))
    np.testing.assert_allclose(x2[others], ref_x2[others], rtol=1e-4)


@pytest.mark.parametrize("tile", [1, 2])
def test_unit_kernel_on_a_larger_phase_grid_after_a_smaller_one(tile):
    """The warp-unit kernel's shared memory grows with the model's phase
    nodes; in one process it must run on a 71-node context first and a
    128-node context (its maximum) afterwards, every mode matching the
    oracle on both."""
    rng = np.random.default_rng(41)
    small = W.config2(n_sn=24)
    m128 = W.make_model(rng, phase=(-20.0, 50.0, 70.0 / 127.0))
    assert small.model.n_phase == 71 and m128.n_phase == 128
    bt = W.make_batch(rng, m128, small.bands, rng.integers(20, 80, 16),
                      rng.uniform(0.02, 0.5, 16), rng.integers(1, 4, 16), perturb=W.PERTURB)
    big = W.Workload("phase128", m128, small.bands, bt)
    for wl in (small, big):
        o = H.with_oracle_flux(wl)
        s = _salt(wl)
        s.set_kernel(KERNELS["unit"])
        s.set_tile(tile)
        db = s.upload(wl.batch)
        ref_bf = o.bandflux(wl.batch)
        H.assert_bandflux_close(wl.batch, s.bandflux(db).cpu().numpy(), ref_bf)
        ref_x2, ref_g = o.chi2(wl.batch, grad=True)
        H.assert_chi2_close(wl.batch, s.chi2(db).cpu().numpy(), ref_x2, ref_bf)
        x2, g = s.chi2_grad(db)
        H.assert_chi2_close(wl.batch, x2.cpu().numpy(), ref_x2, ref_bf)
        H.assert_grad_close(wl.batch, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
        assert s.last_kernel() == (4, tile)
        s.check()
