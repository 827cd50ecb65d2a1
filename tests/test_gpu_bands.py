"""Registering a bandpass on a live context (salt_register_band): results equal
those of a context created with the band from the start, including through a
plan made before the registration (its work lists and scratch are rebuilt for
the new band count)."""
import numpy as np
import pytest

import workloads as W
from tests import _helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _salt(model, bands):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    return Salt(model, bands)


def test_registered_band_equals_a_band_given_at_creation():
    from paper_2504_08081_b300 import _abi
    wl = W.config2(n_sn=60)
    H.with_oracle_flux(wl)
    full = _salt(wl.model, wl.bands)
    dbf = full.upload(wl.batch)
    x2_ref, g_ref = (t.cpu().numpy() for t in full.chi2_grad(dbf))
    bf_ref = full.bandflux(dbf).cpu().numpy()

    s = _salt(wl.model, wl.bands[:5])
    db = s.upload(wl.batch)  # plan made while only 5 bands exist
    has5 = np.array([np.any(wl.batch.band[wl.batch.obs_off[k]:wl.batch.obs_off[k + 1]] == 5)
                     for k in range(wl.batch.n_sn)])
    assert has5.any() and (~has5).any()
    x2, _ = s.chi2_grad(db)
    with pytest.raises(_abi.SaltError):
        s.check()  # band 5 does not exist yet
    x2 = x2.cpu().numpy()
    assert np.all(np.isnan(x2[has5])) and np.all(np.isfinite(x2[~has5]))
    np.testing.assert_array_equal(x2[~has5], x2_ref[~has5])

    b5 = wl.bands[5]
    assert s.register_band(b5.wave, b5.trans) == 5
    x2, g = (t.cpu().numpy() for t in s.chi2_grad(db))
    s.check()
    np.testing.assert_array_equal(x2, x2_ref)
    np.testing.assert_array_equal(g, g_ref)
    np.testing.assert_array_equal(s.bandflux(db).cpu().numpy(), bf_ref)


def test_band_from_file_registers(tmp_path):
    from paper_2504_08081_b300 import _abi
    wl = W.config2(n_sn=20)
    H.with_oracle_flux(wl)
    b5 = wl.bands[5]
    p = tmp_path / "b5.dat"
    with open(p, "w") as f:
        for w, t in zip(b5.wave, b5.trans):
            f.write("%.17g %.17g\n" % (w, t))
    w, t = _abi.load_band(p, step=0.0)
    s = _salt(wl.model, wl.bands[:5])
    assert s.register_band(w, t) == 5
    full = _salt(wl.model, wl.bands)
    a = s.chi2(s.upload(wl.batch)).cpu().numpy()
    b = full.chi2(full.upload(wl.batch)).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    with pytest.raises(_abi.SaltError):
        s.register_band(np.array([5000.0]), np.array([1.0]))  # one sample is not a band
