"""No-allocation chi^2 + gradient entry point (salt_chi2_grad_noalloc).

Two calls in a row must give what salt_chi2_grad gives on the same batch:
identical values against the same kernel configuration (warp-unit kernel,
one sample per unit) and agreement within the parity tolerances against the
autotuned default. A batch beyond the fixed scratch is rejected with a clear
message and untouched outputs. The file name sorts last so that the module
also runs after every other GPU test of a session."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from tests import _helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _salt(wl):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    return Salt(wl.model, wl.bands)


def _grad_close(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-30)
    worst = float((np.abs(got - ref) / scale).max()) if ref.size else 0.0
    assert worst <= H.GRAD_RTOL, f"gradient differs by {worst:.3e} of its inf-norm"


@pytest.mark.parametrize("which", ["one_sample_per_sn", "many_samples_per_sn"])
def test_noalloc_matches_chi2_grad_on_two_calls(which):
    wl = W.config2(n_sn=300) if which == "one_sample_per_sn" else W.config3(n_sn=7, n_samples=45)
    o = H.with_oracle_flux(wl)
    s = _salt(wl)
    db = s.upload(wl.batch)
    n = db.n_par
    x2_auto, g_auto = s.chi2_grad(db)
    s.set_kernel(4)
    s.set_tile(1)
    x2_unit, g_unit = s.chi2_grad(db)
    s.set_kernel(0)
    s.set_tile(0)
    outs = []
    for call in range(2):
        x2 = torch.full((n,), -1.0, dtype=torch.float64, device=s.device)
        g = torch.full((n, 5), -1.0, dtype=torch.float32, device=s.device)
        s.chi2_grad_noalloc(db, x2, g, validate=(call == 1))
        s.check()
        outs.append((x2.cpu().numpy(), g.cpu().numpy()))
    xa, ga = x2_auto.cpu().numpy(), g_auto.cpu().numpy()
    xu, gu = x2_unit.cpu().numpy(), g_unit.cpu().numpy()
    for x2, g in outs:
        assert np.all(np.isfinite(x2)) and np.all(np.isfinite(g))
        np.testing.assert_array_equal(x2, xu)
        np.testing.assert_array_equal(g, gu)
        np.testing.assert_allclose(x2, xa, rtol=1e-4, atol=0)
        _grad_close(g, ga)
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    # and directly against the FP64 oracle, within the parity tolerances
    ref_x2, ref_g = o.chi2(wl.batch, grad=True)
    ref_bf = o.bandflux(wl.batch)
    H.assert_chi2_close(wl.batch, outs[1][0], ref_x2, ref_bf)
    H.assert_grad_close(wl.batch, outs[1][1], ref_g, o=o, bf_ref=ref_bf)


def test_noalloc_call_allocates_no_device_memory():
    """After a first call (which looks the scratch array's address up), a
    further call leaves the device's free memory unchanged: the scratch is the
    library's fixed array, nothing is allocated for the call."""
    wl = W.config2(n_sn=200)
    H.with_oracle_flux(wl)
    s = _salt(wl)
    db = s.upload(wl.batch, plan=False)
    n = db.n_par
    x2 = torch.empty(n, dtype=torch.float64, device=s.device)
    g = torch.empty((n, 5), dtype=torch.float32, device=s.device)
    s.chi2_grad_noalloc(db, x2, g)
    torch.cuda.synchronize()
    free = []
    for _ in range(3):
        before = torch.cuda.mem_get_info(s.device)[0]
        s.chi2_grad_noalloc(db, x2, g)
        torch.cuda.synchronize()
        free.append((before, torch.cuda.mem_get_info(s.device)[0]))
    s.check()
    assert all(b == a for b, a in free), free


def test_noalloc_rejects_a_batch_beyond_its_scratch():
    from paper_2504_08081_b300 import _abi
    wl = W.config3(n_sn=1, n_samples=50000)  # 6 bands: ~21 MB of scratch needed
    s = _salt(wl)
    db = s.upload(wl.batch, plan=False)
    x2 = torch.full((db.n_par,), -1.0, dtype=torch.float64, device=s.device)
    g = torch.full((db.n_par, 5), -1.0, dtype=torch.float32, device=s.device)
    with pytest.raises(_abi.SaltError) as ei:
        s.chi2_grad_noalloc(db, x2, g)
    assert ei.value.code == -1
    assert "SALT_NOALLOC_SCRATCH_BYTES" in str(ei.value)
    torch.cuda.synchronize()
    assert bool((x2 == -1.0).all()) and bool((g == -1.0).all())
    # a batch that fits still runs on the same context afterwards
    b = wl.batch
    small = dataclasses.replace(b, par_off=np.array([0, 5], np.int64),
                                **{k: getattr(b, k)[:5] for k in ("t0", "z", "x0", "x1", "c")})
    sdb = s.upload(small, plan=False)
    y2 = torch.empty(5, dtype=torch.float64, device=s.device)
    gy = torch.empty((5, 5), dtype=torch.float32, device=s.device)
    s.chi2_grad_noalloc(sdb, y2, gy)
    s.check()
    ref2, refg = s.chi2_grad(sdb)
    np.testing.assert_allclose(y2.cpu().numpy(), ref2.cpu().numpy(), rtol=1e-4, atol=0)
    _grad_close(gy.cpu().numpy(), refg.cpu().numpy())
