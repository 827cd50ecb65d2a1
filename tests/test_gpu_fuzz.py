"""Randomized parity sweep: seeded workloads of four shapes (the batched
1-sample shape, many samples per supernova, the ragged 71x901 shape, the
non-uniform 66x991 grid) with random sizes, every kernel family against the
FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from tests import _helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KERNELS = {"auto": 0, "direct": 1, "factorised": 2, "bandwarp": 3, "unit": 4}


def _workload(seed):
    rng = np.random.default_rng(seed)
    kind = seed % 4
    if kind == 0:
        return W.config2(seed=5000 + seed, n_sn=int(rng.integers(20, 120)))
    if kind == 1:
        return W.config3(seed=5000 + seed, n_sn=int(rng.integers(2, 6)), n_samples=int(rng.integers(1, 40)))
    if kind == 2:
        return W.config5(seed=5000 + seed, n_sn=int(rng.integers(10, 50)), n_samples=int(rng.integers(1, 12)))
    return W.config_nir(seed=7000 + seed, n_sn=int(rng.integers(5, 40)), n_samples=int(rng.integers(1, 9)))


@pytest.mark.parametrize("seed", range(16))
def test_random_workloads_every_kernel(seed):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    wl = _workload(seed)
    o = H.with_oracle_flux(wl, seed=seed)
    bt = wl.batch
    ref_bf = o.bandflux(bt)
    ref_x2, ref_g = o.chi2(bt, grad=True)
    s = Salt(wl.model, wl.bands)
    db = s.upload(bt)
    for k in KERNELS.values():
        s.set_kernel(k)
        H.assert_bandflux_close(bt, s.bandflux(db).cpu().numpy(), ref_bf)
        x2, g = s.chi2_grad(db)
        H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
        H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
        s.check()
    s.close()
