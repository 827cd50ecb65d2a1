"""GPU parity on a non-uniform, SALT3-NIR-shaped grid (66 x 991 nodes, optical
and NIR bands): every kernel family against the FP64 oracle with the same
tolerances as the uniform grids; and a uniform grid given as explicit nodes
agrees with the uniform path."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from tests import _helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KERNELS = {"direct": 1, "factorised": 2, "bandwarp": 3, "unit": 4, "auto": 0}


def _salt(model, bands):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    return Salt(model, bands)


@pytest.fixture(scope="module")
def nir():
    wl = W.config_nir(n_sn=24, n_samples=3)
    o = H.with_oracle_flux(wl)
    bf = o.bandflux(wl.batch)
    x2, g = o.chi2(wl.batch, grad=True)
    return wl, o, bf, x2, g


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_nonuniform_grid_parity(nir, kernel):
    wl, o, ref_bf, ref_x2, ref_g = nir
    bt = wl.batch
    s = _salt(wl.model, wl.bands)
    s.set_kernel(KERNELS[kernel])
    db = s.upload(bt)
    H.assert_bandflux_close(bt, s.bandflux(db).cpu().numpy(), ref_bf)
    x2, g = s.chi2_grad(db)
    s.check()
    H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)


def test_explicit_uniform_nodes_match_the_uniform_axes():
    wl = W.config2(n_sn=40)
    H.with_oracle_flux(wl)
    m = wl.model
    mn = dataclasses.replace(m, phase_nodes=m.phase0 + m.dphase * np.arange(m.n_phase),
                             wave_nodes=m.wave0 + m.dwave * np.arange(m.n_wave))
    a = _salt(m, wl.bands)
    b = _salt(mn, wl.bands)
    bfa = a.bandflux(a.upload(wl.batch)).cpu().numpy()
    bfb = b.bandflux(b.upload(wl.batch)).cpu().numpy()
    H.assert_bandflux_close(wl.batch, bfb, bfa.astype(np.float64))


def test_bad_nodes_are_refused():
    from paper_2504_08081_b300 import _abi
    wl = W.config_nir(n_sn=2)
    m = dataclasses.replace(wl.model, wave_nodes=wl.model.wave_nodes[::-1].copy())
    with pytest.raises(_abi.SaltError):
        _salt(m, wl.bands)
