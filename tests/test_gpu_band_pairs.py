"""GPU parity on bands that exercise the band tables' layout and the paired
band-sample loads of the column-response build.

Every band starts on an even index of the flat band tables: a band of odd
length is followed by a zero-weight pad sample, which no kernel may count.
The CTA kernel's build takes its band samples in pairs from an even index, so
a band whose first in-grid sample has an odd index (a band cut by the blue end
of the grid) starts with a half-empty pair, and one cut by the red end can
end with one. Here bands of odd and even lengths (including 2 and 3 samples)
sit across both ends of the wavelength grid for supernovae at low and high
redshift, with parameter samples spread in z so that the first and last
in-grid sample move from sample to sample; every kernel family and the CTA
kernel's tiles are compared with the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from tests import _helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KERNELS = {"direct": 1, "factorised": 2, "bandwarp": 3, "unit": 4, "auto": 0}


def _salt(wl):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    return Salt(wl.model, wl.bands)


def _edge_band_workload():
    rng = np.random.default_rng(2604)
    model = W.make_model(rng, wave_max=9200.0)
    bands = [W.gaussian_band(3700.0, 151), W.gaussian_band(4400.0, 78), W.gaussian_band(6000.0, 3),
             W.gaussian_band(6500.0, 2), W.gaussian_band(8600.0, 203), W.gaussian_band(9000.0, 150)]
    n_sn = 24
    z = np.concatenate([rng.uniform(0.6, 1.3, n_sn // 2), rng.uniform(0.01, 0.1, n_sn // 2)])
    bt = W.make_batch(rng, model, bands, np.full(n_sn, 18), z, np.full(n_sn, 9),
                      perturb=dict(z=0.02, t0=1.0, logx0=0.05, x1=0.2, c=0.02))
    # every band observed, including those the grid cuts at the true redshift
    for s in range(n_sn):
        lo, hi = bt.obs_off[s], bt.obs_off[s + 1]
        bt.band[lo:hi] = (s + np.arange(hi - lo)) % len(bands)
    return W.Workload("edge_bands", model, bands, bt)


@pytest.fixture(scope="module")
def edge_bands():
    wl = _edge_band_workload()
    o = H.with_oracle_flux(wl)
    # the layout under test does occur: cut bands, first in-grid samples of both parities
    bt, firsts = wl.batch, set()
    for j in range(len(bt.z)):
        a = 1.0 / (1.0 + float(bt.z[j]))
        for band in wl.bands[:2]:
            inside = np.nonzero(band.wave * a >= wl.model.wave0)[0]
            if 0 < len(inside) and inside[0] > 0:
                firsts.add(int(inside[0]) % 2)
    assert firsts == {0, 1}
    return wl, o, o.bandflux(bt), o.chi2(bt, grad=True)


@pytest.mark.parametrize("kernel,tile", [("direct", 1), ("bandwarp", 1), ("bandwarp", 2), ("unit", 1),
                                         ("unit", 2), ("auto", 1)] +
                         [("factorised", t) for t in (1, 2, 4, 8, 16)])
def test_bands_cut_by_the_grid_and_odd_lengths(edge_bands, kernel, tile):
    wl, o, ref_bf, (ref_x2, ref_g) = edge_bands
    bt = wl.batch
    s = _salt(wl)
    s.set_kernel(KERNELS[kernel])
    s.set_tile(tile)
    db = s.upload(bt)
    H.assert_bandflux_close(bt, s.bandflux(db).cpu().numpy(), ref_bf)
    x2, g = s.chi2_grad(db)
    H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
    # the chi^2-only variant agrees as well
    H.assert_chi2_close(bt, s.chi2(db).cpu().numpy(), ref_x2, ref_bf)
    s.check()
    s.close()
