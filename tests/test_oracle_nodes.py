"""Pins of the oracle's non-uniform axes (SALT3-NIR-shaped grids): the
reading maps a coordinate to index space u = i + (x - x_i)/(x_{i+1} - x_i) and
applies the Keys kernel there. Checked against: the uniform path (explicit
uniform nodes), node reproduction, exact reproduction of surfaces quadratic in
the node index (the Keys a = -1/2 property, with u from numpy's interpolation
of the index), and finite differences of the analytic derivatives."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def nir():
    return W.make_model_nodes(np.random.default_rng(7), W.NIR_PHASE_NODES, W.NIR_WAVE_NODES)


def test_explicit_uniform_nodes_equal_the_uniform_axes():
    m = W.make_model(np.random.default_rng(3))
    pn = m.phase0 + m.dphase * np.arange(m.n_phase)
    wn = m.wave0 + m.dwave * np.arange(m.n_wave)
    mn = dataclasses.replace(m, phase_nodes=pn, wave_nodes=wn)
    o, on = oracle.Oracle(m, []), oracle.Oracle(mn, [])
    rng = np.random.default_rng(4)
    for _ in range(200):
        p = rng.uniform(m.phase0, m.phase_max)
        lam = rng.uniform(m.wave0, m.wave_max)
        for which in (0, 1):
            a, b = o.surface(which, p, lam), on.surface(which, p, lam)
            np.testing.assert_allclose(b, a, rtol=1e-11, atol=1e-15)


def test_nodes_are_reproduced(nir):
    o = oracle.Oracle(nir, [])
    pn, wn = nir.phase_nodes, nir.wave_nodes
    rng = np.random.default_rng(5)
    for _ in range(100):
        r = int(rng.integers(0, nir.n_phase))
        j = int(rng.integers(0, nir.n_wave))
        v, _, _ = o.surface(0, pn[r], wn[j])
        assert v == pytest.approx(float(nir.m0[r, j]), rel=1e-14, abs=1e-16)


def test_index_quadratic_surfaces_are_reproduced(nir):
    n_p, n_w = nir.n_phase, nir.n_wave
    r = np.arange(n_p)[:, None].astype(np.float64)
    j = np.arange(n_w)[None, :].astype(np.float64)
    q = lambda a, b: 0.3 + 0.02 * a - 0.001 * a * a + 1e-3 * b + 2e-7 * b * b + 1e-5 * a * b
    m = dataclasses.replace(nir, m0=q(r, j), m1=np.zeros_like(q(r, j)))
    o = oracle.Oracle(m, [])
    rng = np.random.default_rng(6)
    pn, wn = nir.phase_nodes, nir.wave_nodes
    for _ in range(300):
        # interior intervals only (edge intervals are linear by the reading)
        p = rng.uniform(pn[1], pn[-2])
        lam = rng.uniform(wn[1], wn[-2])
        up = np.interp(p, pn, np.arange(n_p))
        ul = np.interp(lam, wn, np.arange(n_w))
        v, _, _ = o.surface(0, p, lam)
        assert v == pytest.approx(q(up, ul), rel=1e-12)


def test_derivatives_match_finite_differences(nir):
    o = oracle.Oracle(nir, [])
    rng = np.random.default_rng(8)
    pn, wn = nir.phase_nodes, nir.wave_nodes
    for _ in range(100):
        p = rng.uniform(pn[2], pn[-3])
        lam = rng.uniform(wn[2], wn[-3])
        # keep the stencil inside one interval (the weights have kinks at nodes)
        ip = np.searchsorted(pn, p) - 1
        il = np.searchsorted(wn, lam) - 1
        hp = 1e-4 * (pn[ip + 1] - pn[ip])
        hl = 1e-4 * (wn[il + 1] - wn[il])
        p = np.clip(p, pn[ip] + 2 * hp, pn[ip + 1] - 2 * hp)
        lam = np.clip(lam, wn[il] + 2 * hl, wn[il + 1] - 2 * hl)
        v, dp_, dl_ = o.surface(0, p, lam)
        fdp = (o.surface(0, p + hp, lam)[0] - o.surface(0, p - hp, lam)[0]) / (2 * hp)
        fdl = (o.surface(0, p, lam + hl)[0] - o.surface(0, p, lam - hl)[0]) / (2 * hl)
        scale_p = abs(v) / (pn[ip + 1] - pn[ip]) + 1e-12
        scale_l = abs(v) / (wn[il + 1] - wn[il]) + 1e-12
        assert abs(dp_ - fdp) <= 1e-6 * scale_p
        assert abs(dl_ - fdl) <= 1e-6 * scale_l
