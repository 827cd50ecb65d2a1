"""Pins for the FP64 oracle: facts fixed by the paper's definitions and by
mathematics, independent of the oracle's own code.

Each test names the definition it pins: the SALT model form (Eq. 1), the
bandflux integral (Eq. 2) with the trapezoidal rule (Implementation section),
and the readings taken where the paper is silent (Keys a = -1/2 cubic
convolution, SALT2 colour law, AB zero point, diagonal chi^2)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

H = 6.62607015e-27
C_AA = 2.99792458e18
HC = H * C_AA
AB = 3631e-23


def _model(m0, m1=None, phase=(-20.0, 1.0), wave=(2000.0, 10.0), cl=(0.1, -0.2, 0.05, 0.03)):
    m0 = np.asarray(m0, dtype=np.float64)
    m1 = np.zeros_like(m0) if m1 is None else np.asarray(m1, dtype=np.float64)
    return W.Model(phase0=phase[0], dphase=phase[1], n_phase=m0.shape[0], wave0=wave[0],
                   dwave=wave[1], n_wave=m0.shape[1], m0=m0, m1=m1, cl=np.asarray(cl, float))


def _taps(x, x0, dx, n):
    import ctypes as C
    first = C.c_int32()
    w = np.zeros(4)
    dw = np.zeros(4)
    nt = oracle.lib().om_axis_taps(x, x0, dx, n, C.byref(first), w.ctypes.data, dw.ctypes.data)
    return nt, first.value, w[:nt], dw[:nt]


# ---------------------------------------------------------------- interpolation

def test_keys_textbook_midpoint_weights():
    # Keys (1981), a = -1/2: at the midpoint of an interior interval the four
    # weights are (-1, 9, 9, -1) / 16 (the Catmull-Rom midpoint rule).
    nt, first, w, _ = _taps(3.5, 0.0, 1.0, 10)
    assert nt == 4 and first == 2
    np.testing.assert_allclose(w, np.array([-1, 9, 9, -1]) / 16.0, rtol=0, atol=1e-15)


def test_axis_node_reproduction_and_partition_of_unity():
    rng = np.random.default_rng(0)
    n = 12
    for j in range(n):
        nt, first, w, _ = _taps(5.0 + 2.0 * j, 5.0, 2.0, n)
        full = np.zeros(n)
        full[first:first + nt] = w
        expect = np.zeros(n)
        expect[j] = 1.0
        np.testing.assert_allclose(full, expect, atol=1e-15)
    for x in rng.uniform(5.0, 5.0 + 2.0 * (n - 1), 200):
        nt, first, w, dw = _taps(x, 5.0, 2.0, n)
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs(dw.sum()) < 1e-14


def test_axis_quadratic_interior_linear_edges():
    rng = np.random.default_rng(1)
    n, x0, dx = 10, -3.0, 0.5
    nodes = x0 + dx * np.arange(n)
    q = lambda x: 0.3 * x * x - 1.7 * x + 2.0
    dq = lambda x: 0.6 * x - 1.7
    lin = lambda x: -2.5 * x + 0.75
    for x in rng.uniform(nodes[0], nodes[-1], 500):
        nt, first, w, dw = _taps(x, x0, dx, n)
        idx = np.arange(first, first + nt)
        # linear functions are reproduced on every interval (value and slope)
        assert abs(w @ lin(nodes[idx]) - lin(x)) < 1e-12
        assert abs(dw @ lin(nodes[idx]) - (-2.5)) < 1e-12
        if nt == 4:  # interior: Keys a=-1/2 reproduces quadratics exactly
            assert abs(w @ q(nodes[idx]) - q(x)) < 1e-12
            assert abs(dw @ q(nodes[idx]) - dq(x)) < 1e-11
        else:
            assert first in (0, n - 2)


def test_axis_outside_and_last_node():
    assert _taps(-3.0001, -3.0, 0.5, 10)[0] == 0
    assert _taps(1.5001, -3.0, 0.5, 10)[0] == 0
    nt, first, w, _ = _taps(1.5, -3.0, 0.5, 10)  # x == x_max: last interval, t = 1
    assert nt == 2 and first == 8
    np.testing.assert_allclose(w, [0.0, 1.0], atol=1e-15)


def test_surface_nodes_separable_quadratic_and_outside():
    rng = np.random.default_rng(2)
    G = rng.normal(size=(9, 11))
    m = _model(G, phase=(-4.0, 1.5), wave=(3000.0, 20.0))
    o = oracle.Oracle(m, [])
    for r in range(9):
        for j in range(11):
            v, _, _ = o.surface(0, -4.0 + 1.5 * r, 3000.0 + 20.0 * j)
            assert abs(v - G[r, j]) < 1e-13
    # f(p, l) = q1(p) q2(l): reproduced exactly where both axes are interior
    P = -4.0 + 1.5 * np.arange(9)
    L = 3000.0 + 20.0 * np.arange(11)
    q1 = lambda p: 0.2 * p * p + p - 1.0
    q2 = lambda l: 1e-4 * (l - 3100.0) ** 2 - 0.5
    o2 = oracle.Oracle(_model(np.outer(q1(P), q2(L)), phase=(-4.0, 1.5), wave=(3000.0, 20.0)), [])
    for _ in range(200):
        p = rng.uniform(P[1], P[-2])
        lam = rng.uniform(L[1], L[-2])
        v, dp, dl = o2.surface(0, p, lam)
        assert abs(v - q1(p) * q2(lam)) < 1e-11
        assert abs(dp - (0.4 * p + 1.0) * q2(lam)) < 1e-10
        assert abs(dl - q1(p) * 2e-4 * (lam - 3100.0)) < 1e-10
    assert o.surface(0, P[0] - 1e-9, 3100.0)[0] == 0.0
    assert o.surface(0, 0.0, L[-1] + 1e-9)[0] == 0.0


# ---------------------------------------------------------------- colour law

def test_colorlaw_anchors_continuity_and_linear_tails():
    o = oracle.Oracle(_model(np.ones((5, 5))), [])
    # SALT2 normalisation: CL(lambda_B) = 0, CL(lambda_V) = -1
    assert abs(o.colorlaw(4302.57)[0]) < 1e-15
    assert abs(o.colorlaw(5428.55)[0] + 1.0) < 1e-14
    for edge in (2800.0, 7000.0):
        lo, dlo = o.colorlaw(edge - 1e-7)
        hi, dhi = o.colorlaw(edge + 1e-7)
        on, _ = o.colorlaw(edge)
        # value: both sides meet the polynomial at the edge to first order
        assert abs(lo + dlo * 1e-7 - on) < 1e-12 and abs(hi - dhi * 1e-7 - on) < 1e-12
        assert abs(dlo - dhi) < 1e-12
    # outside the range the law is a straight line
    for a, b in ((1500.0, 2500.0), (7500.0, 12000.0)):
        xs = np.linspace(a, b, 7)
        vs = np.array([o.colorlaw(x)[0] for x in xs])
        assert np.max(np.abs(np.diff(vs, 2))) < 1e-12
        slopes = np.array([o.colorlaw(x)[1] for x in xs])
        assert np.ptp(slopes) < 1e-16 + 1e-12 * np.max(np.abs(slopes))
    # slope reported = derivative of the value
    for x in (2500.0, 3500.0, 5000.0, 6900.0, 9000.0):
        fd = (o.colorlaw(x + 1e-3)[0] - o.colorlaw(x - 1e-3)[0]) / 2e-3
        assert abs(fd - o.colorlaw(x)[1]) < 1e-9


# ---------------------------------------------------------------- band integral

def _flat_model(value=1.0, wave=(2000.0, 10.0, 721)):
    return _model(np.full((71, wave[2]), value), phase=(-20.0, 1.0), wave=wave[:2])


def test_tophat_constant_surface_closed_form():
    # M0 = K, x1 = c = 0, T = 1 on [l1, l2]: the integrand x0 a K lam / (hc) is
    # linear, so the trapezoid is exact: B = x0 a K (l2^2 - l1^2) / (2 hc).
    K = 0.25
    band = W.tophat_band(4000.0, 6000.0)
    o = oracle.Oracle(_flat_model(K), [band])
    z, x0 = 0.3, 2e-5
    par = [z, 55000.0, x0, 0.0, 0.0]
    zp = 25.0
    Bzp = o.bandflux_one(0, 55010.0, zp, par)
    B = Bzp * o.band_ab_flux(0) / 10 ** (0.4 * zp)
    expect = x0 / (1 + z) * K * (6000.0 ** 2 - 4000.0 ** 2) / (2 * HC)
    assert abs(B / expect - 1) < 1e-13


def test_ab_flux_within_trapezoid_error_bound():
    # Z_b = AB/h * integral(T / lam) for a top-hat; the trapezoid's error is
    # bounded by (l2 - l1) h^2 max|f''| / 12 with f = 1/lam, f'' = 2/lam^3.
    for lo, hi, step in ((3000.0, 5000.0, 5.0), (6000.0, 9000.0, 10.0)):
        band = W.tophat_band(lo, hi, step)
        o = oracle.Oracle(_flat_model(), [band])
        Z = o.band_ab_flux(0)
        exact = AB / H * math.log(hi / lo)
        bound = AB / H * (hi - lo) * step ** 2 * (2.0 / lo ** 3) / 12.0
        assert 0 < Z - exact <= bound * (1 + 1e-9)  # convex integrand: trapezoid over-estimates


def test_linear_surface_trapezoid_exact_error_term():
    # M0 linear in lam (constant in phase): the integrand g = x0 a (al + be lam/(1+z)) lam/(hc)
    # is quadratic, so trapezoid - integral = (l2 - l1) h^2 g'' / 12 exactly.
    al, be = 0.05, 2e-5
    wave = 2000.0 + 10.0 * np.arange(721)
    m = _model(np.tile(al + be * wave, (71, 1)), phase=(-20.0, 1.0), wave=(2000.0, 10.0))
    band = W.tophat_band(4000.0, 7000.0, 5.0)
    o = oracle.Oracle(m, [band])
    z, x0, zp = 0.2, 1e-5, 20.0
    Bzp = o.bandflux_one(0, 55000.0, zp, [z, 55000.0, x0, 0.0, 0.0])
    B = Bzp * o.band_ab_flux(0) / 10 ** (0.4 * zp)
    a = 1.0 / (1.0 + z)
    c1, c2 = x0 * a * al / HC, x0 * a * be * a / HC  # g = c1 lam + c2 lam^2
    l1, l2, h = 4000.0, 7000.0, 5.0
    integral = c1 * (l2 ** 2 - l1 ** 2) / 2 + c2 * (l2 ** 3 - l1 ** 3) / 3
    expect = integral + (l2 - l1) * h * h * (2 * c2) / 12.0
    assert abs(B / expect - 1) < 1e-12


def test_ab_spectrum_gives_exact_zero_point():
    # A model whose observer-frame flux equals f_AB at every band sample gives
    # bandflux = 10^(0.4 zp) exactly (z = 0, c = 0, band samples on grid nodes).
    wave = 2000.0 + 10.0 * np.arange(721)
    x0 = 1e-5
    fab = AB * C_AA / wave ** 2
    m = _model(np.tile(fab / x0, (71, 1)), phase=(-20.0, 1.0), wave=(2000.0, 10.0))
    band = W.gaussian_band(5500.0, 201, step=10.0)
    o = oracle.Oracle(m, [band])
    for zp in (0.0, 25.0, 27.5):
        v = o.bandflux_one(0, 55000.0, zp, [0.0, 55000.0, x0, 0.0, 0.0])
        assert abs(v / 10 ** (0.4 * zp) - 1) < 1e-13


def test_band_trapezoid_agrees_with_fine_quadrature():
    # The coarse trapezoid on the band's own 5 A samples differs from a fine
    # (0.05 A) quadrature of the same integrand (T linear between samples)
    # by no more than the trapezoid error bound (l2-l1) h^2 max|g''| / 12.
    w = W.config1()
    band = w.bands[1]
    o = oracle.Oracle(w.model, [band])
    par = [0.1, 55000.0, 1e-5, 0.5, 0.05]
    mjd = 55003.0
    coarse = o.bandflux_one(0, mjd, 0.0, par) * o.band_ab_flux(0)
    fine_l = np.arange(band.wave[0], band.wave[-1] + 1e-9, 0.05)
    fine_t = np.interp(fine_l, band.wave, band.trans)
    g = np.array([o.flux_obs(l, mjd, par) for l in fine_l]) * fine_t * fine_l / HC
    fine = np.trapezoid(g, fine_l)
    # g'' estimated from the fine samples (T is piecewise linear, so g'' is
    # taken on the smooth part; bound with a 2x safety factor)
    g_coarse = np.array([o.flux_obs(l, mjd, par) for l in band.wave]) * band.trans * band.wave / HC
    g2 = np.max(np.abs(np.diff(g_coarse, 2))) / 25.0
    bound = 2.0 * (band.wave[-1] - band.wave[0]) * 25.0 * g2 / 12.0
    assert abs(coarse - fine) <= bound
    assert abs(coarse / fine - 1) < 1e-4


# ---------------------------------------------------------------- model form

def test_linear_in_x0_and_x1_and_c_zero():
    w = W.config1()
    o = oracle.Oracle(w.model, w.bands)
    par = np.array([0.1, 55000.0, 1e-5, 0.5, 0.05])
    for b in range(4):
        v1 = o.bandflux_one(b, 55004.0, 27.5, par)
        p2 = par.copy()
        p2[2] *= 2
        assert abs(o.bandflux_one(b, 55004.0, 27.5, p2) / v1 - 2) < 1e-15
        # B is affine in x1: B(x1+1) - B(x1) = x0 a int(M1 ...) = dB/dx1
        p3 = par.copy()
        p3[3] += 1.0
        _, g = o.bandflux_one(b, 55004.0, 27.5, par, grad=True)
        assert abs((o.bandflux_one(b, 55004.0, 27.5, p3) - v1) - g[3]) < 1e-12 * abs(v1)


def test_z0_rest_frame_direct_sum():
    # z = 0, x1 = c = 0, phase on a node, band samples on grid nodes: the
    # bandflux is the trapezoid of x0 G0[r, j] T lam / (hc) straight from the grid.
    w = W.config1()
    band = W.gaussian_band(5000.0, 121, step=10.0)
    o = oracle.Oracle(w.model, [band])
    x0, zp = 1e-5, 27.5
    r = 25  # phase = -20 + 25 = 5 d
    Bzp = o.bandflux_one(0, 55005.0, zp, [0.0, 55000.0, x0, 0.0, 0.0])
    j = ((band.wave - 2000.0) / 10.0).astype(int)
    g = x0 * w.model.m0[r, j].astype(np.float64) * band.trans * band.wave / HC
    B = float(np.sum(0.5 * np.diff(band.wave) * (g[1:] + g[:-1])))
    assert abs(Bzp * o.band_ab_flux(0) / 10 ** (0.4 * zp) / B - 1) < 1e-13


def test_colour_zero_and_epoch_shift():
    w = W.config1()
    o = oracle.Oracle(w.model, w.bands)
    a = o.bandflux_one(2, 55010.0, 27.5, [0.1, 55000.0, 1e-5, 0.5, 0.0])
    b = o.bandflux_one(2, 55010.0 + 123.0, 27.5, [0.1, 55000.0 + 123.0, 1e-5, 0.5, 0.0])
    assert abs(a / b - 1) < 1e-12
    # c = 0: the colour factor is exactly 1, so the flux at any sample is x0 a (M0 + x1 M1)
    lam, mjd = 6000.0, 55007.0
    F = o.flux_obs(lam, mjd, [0.1, 55000.0, 1e-5, 0.5, 0.0])
    M0 = o.surface(0, 7.0 / 1.1, lam / 1.1)[0]
    M1 = o.surface(1, 7.0 / 1.1, lam / 1.1)[0]
    assert abs(F - 1e-5 / 1.1 * (M0 + 0.5 * M1)) < 1e-15 * abs(F) + 1e-300
    # at the V reference wavelength CL = -1, so the colour factor is 10^(0.4 c);
    # at the B reference wavelength CL = 0 and colour has no effect
    for c in (-0.2, 0.07, 0.3):
        for lam_rest, factor in ((5428.55, 10 ** (0.4 * c)), (4302.57, 1.0)):
            lo = lam_rest * 1.1
            Fc = o.flux_obs(lo, mjd, [0.1, 55000.0, 1e-5, 0.5, c])
            F0 = o.flux_obs(lo, mjd, [0.1, 55000.0, 1e-5, 0.5, 0.0])
            assert abs(Fc / F0 / factor - 1) < 1e-12


# ---------------------------------------------------------------- chi^2 and gradient

def _noiseless_config1():
    w = W.config1()
    o = oracle.Oracle(w.model, w.bands)
    m = o.bandflux(w.batch)
    W.add_noise(w.batch, m, np.random.default_rng(0), noiseless=True)
    w.batch.flux = m  # exact FP64 model values (no float32 rounding)
    return w, o


def test_chi2_zero_and_gradient_zero_at_noiseless_truth():
    w, o = _noiseless_config1()
    x2, g = o.chi2(w.batch, grad=True)
    assert x2[0] < 1e-20
    assert np.max(np.abs(g)) < 1e-9


def test_least_squares_x0():
    # For fixed (z, t0, x1, c) chi^2 is quadratic in x0 with minimiser
    # x0* = sum(f mh / s^2) / sum(mh^2 / s^2), mh = bandflux / x0.
    w = W.config1()
    o = oracle.Oracle(w.model, w.bands)
    m = o.bandflux(w.batch)
    W.add_noise(w.batch, m, np.random.default_rng(5))
    bt = w.batch
    mh = m / float(bt.x0[0])
    f = bt.flux.astype(np.float64)
    s = bt.fluxerr.astype(np.float64)
    x0s = np.sum(f * mh / s ** 2) / np.sum(mh ** 2 / s ** 2)
    bt.x0 = np.array([x0s])
    x2, g = o.chi2(bt, grad=True)
    # dchi2/dx0 = 0 relative to its natural scale sum(mh^2/s^2) * x0*
    assert abs(g[0, 2]) < 1e-9 * np.sum(mh ** 2 / s ** 2) * x0s
    expect = np.sum((f - x0s * mh) ** 2 / s ** 2)
    assert abs(x2[0] / expect - 1) < 1e-12


SCALE = np.array([0.01, 1.0, None, 1.0, 0.1], dtype=object)


def test_gradient_matches_central_differences():
    w = W.config2(n_sn=6)
    o = oracle.Oracle(w.model, w.bands)
    m = o.bandflux(w.batch)
    W.add_noise(w.batch, m, np.random.default_rng(3))
    bt = w.batch
    rng = np.random.default_rng(4)
    # move away from the truth so the gradient is not small
    bt.z = bt.z + rng.normal(0, 0.01, bt.n_par)
    bt.t0 = bt.t0 + rng.normal(0, 1.0, bt.n_par)
    bt.x1 = bt.x1 + rng.normal(0, 0.2, bt.n_par)
    bt.c = bt.c + rng.normal(0, 0.02, bt.n_par)
    x2, g = o.chi2(bt, grad=True)
    names = ["z", "t0", "x0", "x1", "c"]
    for q, name in enumerate(names):
        base = np.asarray(getattr(bt, name), dtype=np.float64)
        scale = np.abs(base) if name == "x0" else np.full(base.shape, SCALE[q])
        # t0 is an epoch: its step is relative to the 1-day scale, not to the MJD value
        h = 1e-4 * (scale if name == "t0" else np.maximum(np.abs(base), scale))
        setattr(bt, name, base + h)
        xp = o.chi2(bt)
        setattr(bt, name, base - h)
        xm = o.chi2(bt)
        setattr(bt, name, base)
        fd = (xp - xm) / (2 * h)
        # theta-scaled comparison (g * s) against the inf-norm of the scaled gradient
        gs = g * np.stack([np.full(bt.n_par, 0.01), np.ones(bt.n_par), np.asarray(bt.x0, float),
                           np.ones(bt.n_par), np.full(bt.n_par, 0.1)], 1)
        err = np.abs(fd - g[:, q]) * (scale)
        assert np.all(err <= 1e-6 * np.max(np.abs(gs), axis=1)), (name, err, gs)


def test_tiny_case_against_50_digit_evaluation():
    # 6 x 6 grid, 3-sample band, one observation: the same definitions
    # evaluated in 50-digit arithmetic (mpmath) from scratch.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(7)
    G0 = rng.uniform(0.5, 1.5, (6, 6))
    G1 = rng.uniform(-0.2, 0.2, (6, 6))
    cl = (0.2, -0.1, 0.05, -0.02)
    m = _model(G0, G1, phase=(-2.0, 2.0), wave=(3000.0, 400.0), cl=cl)
    band = W.Band(wave=np.array([4000.0, 4400.0, 4900.0]), trans=np.array([0.3, 1.0, 0.6]))
    o = oracle.Oracle(m, [band])
    par = [0.17, 55000.0, 1.3e-5, 0.4, -0.07]
    mjd, zp = 55003.25, 26.0
    got = o.bandflux_one(0, mjd, zp, par)

    M = mp.mpf
    a = M(-1) / 2

    def W_(s):
        s = abs(s)
        if s <= 1:
            return (a + 2) * s ** 3 - (a + 3) * s ** 2 + 1
        if s < 2:
            return a * s ** 3 - 5 * a * s ** 2 + 8 * a * s - 4 * a
        return M(0)

    def taps(x, x0, dx, n):
        u = (x - x0) / dx
        i = min(max(int(mp.floor(u)), 0), n - 2)
        t = u - i
        if i in (0, n - 2):
            return [(i, 1 - t), (i + 1, t)]
        return [(i - 1 + k, W_(u - (i - 1 + k))) for k in range(4)]

    def surf(Gm, p, lam):
        if not (M(-2) <= p <= M(8) and M(3000) <= lam <= M(5000)):
            return M(0)
        return sum(wp * wl * M(float(Gm[r, j])) for r, wp in taps(p, M(-2), M(2), 6)
                   for j, wl in taps(lam, M(3000), M(400), 6))

    def CL(lam):
        x = (lam - M("4302.57")) / (M("5428.55") - M("4302.57"))
        A = [M(v) for v in cl]
        P = lambda x: (1 - sum(A)) * x + sum(A[m] * x ** (m + 2) for m in range(4))
        dP = lambda x: (1 - sum(A)) + sum((m + 2) * A[m] * x ** (m + 1) for m in range(4))
        for edge, cond in ((M(2800), lam < 2800), (M(7000), lam > 7000)):
            if cond:
                xe = (edge - M("4302.57")) / (M("5428.55") - M("4302.57"))
                return -(P(xe) + dP(xe) * (x - xe))
        return -P(x)

    z, t0, x0, x1, c = [M(v) for v in par]
    hc = M("6.62607015e-27") * M("2.99792458e18")
    g = []
    zab = []
    for lam, T in zip(band.wave, band.trans):
        lam, T = M(float(lam)), M(float(T))
        lr = lam / (1 + z)
        p = (M(mjd) - t0) / (1 + z)
        F = x0 * (surf(G0, p, lr) + x1 * surf(G1, p, lr)) * mp.power(10, -M("0.4") * c * CL(lr)) / (1 + z)
        g.append(F * T * lam / hc)
        zab.append(M("3631e-23") * M("2.99792458e18") / lam ** 2 * T * lam / hc)
    lw = [M(float(v)) for v in band.wave]
    trap = lambda y: sum((lw[k + 1] - lw[k]) * (y[k] + y[k + 1]) / 2 for k in range(2))
    ref = trap(g) * mp.power(10, M("0.4") * M(zp)) / trap(zab)
    assert abs(got / float(ref) - 1) < 1e-14


# ---------------------------------------------------------------- batched CSR drivers

def _ragged_batch():
    """A ragged batch whose supernovae have 0, 1 or several observations and
    0 to 5 parameter samples, with empty supernovae between non-empty ones."""
    w = W.config2(n_sn=4)
    rng = np.random.default_rng(11)
    n_obs = [3, 0, 1, 5, 0, 4, 2, 6, 0]
    n_par = [2, 3, 0, 1, 0, 5, 4, 0, 2]
    z = rng.uniform(0.05, 0.5, len(n_obs)).astype(np.float32)
    bt = W.make_batch(rng, w.model, w.bands, n_obs, z, n_par, perturb=W.PERTURB)
    W.template_flux(bt, rng)
    return w, bt


def test_batched_drivers_follow_the_per_observation_definition():
    # The bandflux of observation i of supernova s for its sample j is Eq. 2
    # evaluated once (om_bandflux_one); the batched drivers only map
    # (s, j, i) to positions in the CSR layout: bandflux at
    # bf_off[s] + j n_s + i, chi^2 of sample j the sum of ((f - B)/sigma)^2
    # over its own supernova's observations and its gradient the sum of
    # -2 r / sigma dB. Evaluated here one pair at a time from the CSR offsets.
    w, bt = _ragged_batch()
    o = oracle.Oracle(w.model, w.bands)
    bf = o.bandflux(bt)
    x2, g = o.chi2(bt, grad=True)
    n_obs = np.diff(bt.obs_off)
    n_par = np.diff(bt.par_off)
    assert len(bf) == int(np.sum(n_obs * n_par)) and len(x2) == bt.n_par
    pos = 0
    seen_par = 0
    for s in range(bt.n_sn):
        for jj in range(int(n_par[s])):
            j = int(bt.par_off[s]) + jj
            par = [float(bt.z[j]), float(bt.t0[j]), float(bt.x0[j]), float(bt.x1[j]), float(bt.c[j])]
            chi, gr = 0.0, np.zeros(5)
            for i in range(int(n_obs[s])):
                ob = int(bt.obs_off[s]) + i
                B, dB = o.bandflux_one(int(bt.band[ob]), float(bt.mjd[ob]), float(bt.zp[ob]), par,
                                       grad=True)
                # the stored bandflux sits at the next position of the layout
                assert bf[pos] == B, (s, jj, i)
                pos += 1
                r = (float(bt.flux[ob]) - B) / float(bt.fluxerr[ob])
                chi += r * r
                gr += -2.0 * r / float(bt.fluxerr[ob]) * dB
            # a sample of a supernova without observations has chi^2 = 0, gradient 0
            assert abs(x2[j] - chi) <= 1e-14 * abs(chi), (s, jj, x2[j], chi)
            assert np.all(np.abs(g[j] - gr) <= 1e-14 * np.max(np.abs(gr))), (s, jj)
            seen_par += 1
    assert pos == len(bf) and seen_par == bt.n_par
    # the layout really is ragged: some chi^2 are zero (no observations), the rest not
    assert np.any(x2 == 0.0) and np.all(x2[np.repeat(n_obs, n_par) > 0] > 0.0)
