"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times (autotuned kernel choice, graph replay of repeated calls):

- batched_chi2_1000sn (1000 supernovae, one sample each): every chi^2,
  gradient and bandflux against the FP64 oracle;
- diff_256sn_x1024 and large_ragged_100000sn_x64: the whole batch on the GPU,
  then sampled (supernova, sample) pairs that the oracle evaluates one by one.

Inputs are the benchmark's own (same seeds, model-free template fluxes), so the
residuals are large and the chi^2 bound (the change 1e-5 relative bandflux
errors can make) is correspondingly wide; tolerances as in the other parity
tests."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import _helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bench_workload(config):
    """The benchmark's inputs for a configuration (seed 1000 + config)."""
    seed = 1000 + config
    wl = W.make(config, seed=seed)
    W.template_flux(wl.batch, np.random.default_rng(seed + 1))
    return wl


def _salt(wl):
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    return Salt(wl.model, wl.bands)


def _run(s, db, calls=3):
    """Repeated calls on the same buffers, as the benchmark makes them: the
    first tunes and launches directly, the next capture and replay a graph."""
    x2 = torch.empty(db.n_par, dtype=torch.float64, device=s.device)
    g = torch.empty((db.n_par, 5), dtype=torch.float32, device=s.device)
    for _ in range(calls):
        x2.fill_(float("nan"))
        s.chi2_grad(db, x2, g)
    torch.cuda.synchronize()
    s.check()
    return x2, g


def _picks_batch(bt, picks):
    """One supernova per picked global sample index: that sample's supernova's
    observations and the sample alone."""
    sn_of = np.searchsorted(bt.par_off, picks, side="right") - 1
    sub = W.subset(bt, sn_of)
    sub.par_off = np.arange(len(picks) + 1, dtype=np.int64)
    for k in ("t0", "z", "x0", "x1", "c"):
        setattr(sub, k, getattr(bt, k)[picks].copy())
    return sub, sn_of


def test_batched_1000sn_every_output():
    wl = _bench_workload(2)
    bt = wl.batch
    assert bt.n_sn == 1000
    o = oracle.Oracle(wl.model, wl.bands)
    s = _salt(wl)
    db = s.upload(bt)
    x2, g = _run(s, db)
    fam, tile = s.last_kernel()
    assert fam in (2, 3, 4) and tile >= 1
    ref_bf = o.bandflux(bt)
    ref_x2, ref_g = o.chi2(bt, grad=True)
    H.assert_chi2_close(bt, x2.cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(bt, g.cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
    bf = s.bandflux(db).cpu().numpy()
    H.assert_bandflux_close(bt, bf, ref_bf)
    s.check()


@pytest.mark.parametrize("config,n_picks", [(3, 96), (5, 192)])
def test_full_batch_sampled_pairs(config, n_picks):
    wl = _bench_workload(config)
    bt = wl.batch
    o = oracle.Oracle(wl.model, wl.bands)
    s = _salt(wl)
    db = s.upload(bt)
    x2, g = _run(s, db)
    assert bool(torch.isfinite(x2).all()) and bool(torch.isfinite(g).all())
    rng = np.random.default_rng(4242 + config)
    # the first and last samples of the batch, plus random ones
    picks = np.unique(np.concatenate([[0, bt.n_par - 1], rng.choice(bt.n_par, n_picks, replace=False)]))
    sub, sn_of = _picks_batch(bt, picks)
    ref_bf = o.bandflux(sub)
    ref_x2, ref_g = o.chi2(sub, grad=True)
    pk = torch.as_tensor(picks, device=s.device)
    H.assert_chi2_close(sub, x2[pk].cpu().numpy(), ref_x2, ref_bf)
    H.assert_grad_close(sub, g[pk].cpu().numpy(), ref_g, o=o, bf_ref=ref_bf)
    # bandfluxes of the same pairs from a full-batch bandflux call
    bf = s.bandflux(db)
    off = oracle.Oracle.bandflux_offsets(bt)
    idx = []
    for p, sn in zip(picks, sn_of):
        n = int(bt.obs_off[sn + 1] - bt.obs_off[sn])
        j = int(p - bt.par_off[sn])
        idx.append(np.arange(off[sn] + j * n, off[sn] + (j + 1) * n))
    got = bf[torch.as_tensor(np.concatenate(idx), device=s.device)].cpu().numpy()
    del bf
    H.assert_bandflux_close(sub, got, ref_bf)
    s.check()
