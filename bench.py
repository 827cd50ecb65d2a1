"""Benchmark: batched SALT chi^2 + gradient on one B300 (per rank).

One step = one salt_chi2_grad call over the whole batch (phase/wavelength,
bicubic M0/M1, colour law, band integral, zero point, FP64 chi^2 and the
adjoint gradient) through the fused persistent factorised kernel. The primary
workload is the large ragged batch: 100 000 supernovae x 64 parameter samples,
observation counts log-uniform in [8, 400] over 8 bands, the 71 x 901 grid,
z ~ U(0.01, 2) (6.4e8 bandfluxes per step, 0.39 GB of inputs, larger than L2);
inputs are resident in HBM and L2 is flushed between timed steps as well.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own seeded batch of the same shape (weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

KERNEL_NAMES = {1: "salt::k_direct<MODE_GRAD>", 2: "salt::fk::k_fact<{},MODE_GRAD>",
                3: "salt::bw::k_bandwarp<{},MODE_GRAD>", 4: "salt::uk::k_unit<{},MODE_GRAD>"}
METRIC = "bandfluxes/s and chi2+grad evals/s on 1 B300 vs oracle; serving p50/p99 ms"
UNIT = "bandfluxes/s"

# Algorithmic FP32 work of the factorised method (FLOP per unit; each FMA = 2).
# The gradient is counted in its cheapest form (no value computed twice): the
# column responses E, E_c = dE/dc and E_z (the lambda' part of dE/dz) built in
# one pass, forward row dots of E, the adjoint rows back-projected once
# (Q = Y^T H), and dchi2/dc, dchi2/dz as the dots Q.E_c, Q.E_z.
FLOP_K_FWD = 33      # per (sample, band, in-grid band sample), forward: lambda', Keys weights,
                     # colour law, exp2, weight, 4 weighted taps and their column sums
FLOP_K_GRAD = 74     # ... with Keys derivatives, colour-law slope, 12 weighted taps (E, E_c,
                     # E_z) and their column sums
FLOP_RC_GRAD = 8     # per (sample, band, touched row, window column): forward + reverse FMA pair
FLOP_RC_FWD = 4
FLOP_C_GRAD = 4      # per (sample, band, window column): Q.E_c and Q.E_z
FLOP_OBS_GRAD = 60   # per (sample, observation): phase taps, 4-row combine, residual, gradient
FLOP_OBS_FWD = 24
WORK_SAMPLES = 20000  # samples the FLOP count visits (larger batches: a seeded subsample, scaled)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", type=int, default=5, choices=[2, 3, 5])
    ap.add_argument("--n-sn", type=int, default=0,
                    help="supernovae of the workload (0: its configured size); smaller sizes of the "
                         "same generator are for profiling captures")
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle CPU-baseline budget")
    ap.add_argument("--profile", action="store_true",
                    help="timed steps only (no e2e, CPU baseline or secondary workloads): for ncu")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def make_workload(config: int, rank: int, n_sn: int = 0):
    seed = 1000 + config + 7919 * rank
    wl = W.make(config, seed=seed, **({"n_sn": n_sn} if n_sn else {}))
    W.template_flux(wl.batch, np.random.default_rng(seed + 1))
    return wl


def algorithmic_flops(wl, grad=True, max_par=2_000_000):
    """Exact count of the factorised method's necessary FP32 work for one
    pass over the batch: per (sample, band) the in-grid band samples, the
    window columns and the distinct phase rows its own observations touch."""
    return algorithmic_work(wl, grad, max_par)[0]


def interval(x, x0, dx, nodes):
    """Interval index of x on a model axis: uniform (x0, dx) or, with nodes, the
    last node at or below x."""
    if nodes is None:
        return np.floor((np.asarray(x) - x0) / dx).astype(np.int64)
    return np.searchsorted(np.asarray(nodes), np.asarray(x), side="right").astype(np.int64) - 1


def algorithmic_work(wl, grad=True, max_par=2_000_000):
    """(FLOP, grid bytes) of one pass: the FP32 work above, and the grid
    values the row dots read, touched rows x window columns x 8 bytes (M0 and
    M1 as one float2) per (sample, band)."""
    m, bt = wl.model, wl.batch
    nb = len(wl.bands)
    lam_lo = np.array([b.wave[0] for b in wl.bands])
    lam_hi = np.array([b.wave[-1] for b in wl.bands])
    waves = [np.asarray(b.wave, dtype=np.float64) for b in wl.bands]
    n_obs = np.diff(bt.obs_off)
    n_par = np.diff(bt.par_off)
    total = 0.0
    grid_bytes = 0.0
    rng = np.random.default_rng(0)
    # subsample very large batches and scale (the count is a sum over samples)
    idx_all = np.arange(bt.n_par)
    scale = 1.0
    if bt.n_par > max_par:
        idx_all = np.sort(rng.choice(bt.n_par, max_par, replace=False))
        scale = bt.n_par / max_par
    sn_of = np.repeat(np.arange(bt.n_sn), n_par)
    for chunk in np.array_split(idx_all, max(1, len(idx_all) // 20000)):
        for j in chunk:
            s = sn_of[j]
            lo, hi = bt.obs_off[s], bt.obs_off[s + 1]
            if hi == lo:
                continue
            a = 1.0 / (1.0 + float(bt.z[j]))
            p = (bt.mjd[lo:hi] - bt.t0[j]) * a
            bands = bt.band[lo:hi]
            ok = (p >= m.phase0) & (p <= m.phase_max)
            iv = np.clip(interval(p, m.phase0, m.dphase, m.phase_nodes), 0, m.n_phase - 2)
            first = np.where(iv == 0, 0, np.where(iv == m.n_phase - 2, m.n_phase - 4, iv - 1))
            for b in np.unique(bands):
                sel = (bands == b)
                nb_obs = int(sel.sum())
                fr = first[sel & ok]
                rows = np.unique((fr[:, None] + np.arange(4)[None, :]).ravel()).size if fr.size else 0
                lr = waves[b] * a
                kin = int(((lr >= m.wave0) & (lr <= m.wave_max)).sum())
                if kin:
                    lri = lr[(lr >= m.wave0) & (lr <= m.wave_max)]
                    c0 = np.clip(interval(lri[[0, -1]], m.wave0, m.dwave, m.wave_nodes), 0, m.n_wave - 2)
                    f0 = [0 if c == 0 else (m.n_wave - 4 if c == m.n_wave - 2 else c - 1) for c in c0]
                    cols = f0[1] + 3 - f0[0] + 1
                else:
                    cols = 0
                grid_bytes += 8.0 * rows * cols
                if grad:
                    total += (FLOP_K_GRAD * kin + FLOP_RC_GRAD * rows * cols + FLOP_C_GRAD * cols
                              + FLOP_OBS_GRAD * nb_obs)
                else:
                    total += FLOP_K_FWD * kin + FLOP_RC_FWD * rows * cols + FLOP_OBS_FWD * nb_obs
    del lam_lo, lam_hi, nb
    return total * scale, grid_bytes * scale


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason sampling during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        # nvidia-smi's start-up (driver queries before its first sample) disturbs
        # the first milliseconds of GPU work: begin timing after its first sample
        t_end = time.perf_counter() + 5.0
        while self.proc is not None and not self.lines and time.perf_counter() < t_end:
            time.sleep(0.01)
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        time.sleep(0.25)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    the same workload per step."""
    if rank != 0:
        return
    import oracle
    wl = make_workload(args.workload, 0, args.n_sn)
    bt = wl.batch
    o = oracle.Oracle(wl.model, wl.bands)
    # per step: the first supernovae of the batch up to ~1/4 s of CPU work
    n_sn = min(bt.n_sn, 250 if args.workload == 2 else 8)
    sub = W.subset(bt, np.arange(n_sn))
    for _ in range(args.warmup):
        o.chi2(sub, grad=True)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.chi2(sub, grad=True)
        t.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(t)
    nbf = sub.n_bandflux()
    value = nbf / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W.CONFIG_NAMES[args.workload], "sample_supernovae": n_sn},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.threads, "kind": "oracle",
                         "sample": f"first {n_sn} supernovae ({nbf} bandfluxes) per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm

def reduce_over_ranks(ms, n_bandflux, n_par, device):
    """Whole-job figures over the ranks of the default process group (if any):
    the slowest rank's time per step and the summed work of all ranks. Each
    rank owns its own supernovae; nothing else is exchanged."""
    import torch
    import torch.distributed as dist
    ms_t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    cnt = torch.tensor([float(n_bandflux), float(n_par)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    return float(ms_t.item()), float(cnt[0].item()), float(cnt[1].item())


def time_steps_graph(fn, steps, warmup, stream, flush=None):
    """Device time of each step with no host work inside the timed region:
    the K steps (L2 flush, event, step, event) are captured once into one CUDA
    graph, whose event nodes record on the stream, and the graph is launched
    once; one synchronize on each side. Returns None when the capture cannot be
    made (the caller then falls back to time_steps)."""
    import torch
    try:
        from cuda.bindings import runtime as rt
    except ImportError:
        return None
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    st = rt.cudaStream_t(stream.cuda_stream)
    evs = []
    for _ in range(2 * steps):
        err, ev = rt.cudaEventCreate()
        if err != rt.cudaError_t.cudaSuccess:
            return None
        evs.append(ev)
    graph = exec_ = None
    try:
        if rt.cudaStreamBeginCapture(st, rt.cudaStreamCaptureMode.cudaStreamCaptureModeThreadLocal)[0] != \
                rt.cudaError_t.cudaSuccess:
            return None
        ok = True
        with torch.cuda.stream(stream):
            for i in range(steps):
                if flush is not None:
                    flush()
                ok &= rt.cudaEventRecordWithFlags(evs[2 * i], st, rt.cudaEventRecordExternal)[0] == \
                    rt.cudaError_t.cudaSuccess
                fn()
                ok &= rt.cudaEventRecordWithFlags(evs[2 * i + 1], st, rt.cudaEventRecordExternal)[0] == \
                    rt.cudaError_t.cudaSuccess
        err, graph = rt.cudaStreamEndCapture(st)
        if err != rt.cudaError_t.cudaSuccess or not ok:
            return None
        err, exec_ = rt.cudaGraphInstantiate(graph, 0)
        if err != rt.cudaError_t.cudaSuccess:
            return None
        # one untimed replay (first launch of a graph uploads it), then the timed one
        for rep in range(2):
            torch.cuda.synchronize()
            if rt.cudaGraphLaunch(exec_, st)[0] != rt.cudaError_t.cudaSuccess:
                return None
            torch.cuda.synchronize()
        durs = []
        for i in range(steps):
            err, ms = rt.cudaEventElapsedTime(evs[2 * i], evs[2 * i + 1])
            if err != rt.cudaError_t.cudaSuccess:
                return None
            durs.append(ms)
        return durs
    finally:
        if exec_ is not None:
            rt.cudaGraphExecDestroy(exec_)
        if graph is not None:
            rt.cudaGraphDestroy(graph)
        for ev in evs:
            rt.cudaEventDestroy(ev)


def time_steps(fn, steps, warmup, stream, flush=None, queue_ahead=True):
    """Device time of each step: a pair of CUDA events on `stream` around it,
    the L2 flush (if any) enqueued before the first event. With queue_ahead
    the stream first spins for a few ms on the device, so the host has
    enqueued every step before the first one starts and the device never waits
    for the host inside a timed bracket; one synchronize on each side. Without
    it every step is synchronised (host-inclusive per-call latency)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if queue_ahead:
        with torch.cuda.stream(stream):
            torch.cuda._sleep(int(4e6) * max(1, steps // 5))  # ~2 ms per 5 steps at 2 GHz
        # untimed steps queued behind the spin bring the clocks back up before
        # the first timed step (the one-thread spin and the idle host let them drop)
        for _ in range(10):
            if flush is not None:
                flush()
            fn()
    evs = []
    for _ in range(steps):
        if flush is not None:
            flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        evs.append((e0, e1))
        if not queue_ahead:
            e1.synchronize()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def sampled_oracle(wl, s, db, stream, n_picks=None, budget_s=None, results=None):
    """The oracle on seeded (supernova, sample) pairs of a batch too large for
    it: its chi^2 + gradient rate on those pairs, and the error of this
    library's full-batch results at those pairs against it (chi^2 and
    gradient: `results` = (chi2, grad) device tensors of a timed step, else a
    new salt_chi2_grad call; bandfluxes: a full-batch salt_bandflux call).
    The number of pairs is n_picks, or, with budget_s, what fills about that
    many seconds of oracle time at the rate measured on a first 512 pairs. The
    first and last sample of the batch are always among them."""
    import torch
    import oracle
    bt = wl.batch
    o = oracle.Oracle(wl.model, wl.bands)
    rng = np.random.default_rng(77)

    def pairs(n):
        p = rng.choice(bt.n_par, min(n, bt.n_par), replace=False)
        p = np.unique(np.concatenate([p, [0, bt.n_par - 1]])) if bt.n_par else p
        sn = np.searchsorted(bt.par_off, p, side="right") - 1
        sub = W.subset(bt, sn)
        sub.par_off = np.arange(len(p) + 1, dtype=np.int64)
        for k in ("t0", "z", "x0", "x1", "c"):
            setattr(sub, k, getattr(bt, k)[p].copy())
        return p, sn, sub

    if budget_s is not None:
        # calibration on enough pairs to keep every host thread busy
        _, _, cal = pairs(512)
        t0 = time.perf_counter()
        o.chi2(cal, grad=True)
        rate = cal.n_bandflux() / max(time.perf_counter() - t0, 1e-6)
        per_pair = bt.n_bandflux() / max(bt.n_par, 1)
        n_picks = int(np.clip(budget_s * rate / per_pair, 64, 32768))
    picks, sn_of, sub = pairs(n_picks)
    with torch.cuda.stream(stream):
        x2, g = results if results is not None else s.chi2_grad(db)
        bf = s.bandflux(db)
    torch.cuda.synchronize()
    off = oracle.Oracle.bandflux_offsets(bt)
    idx = np.concatenate([np.arange(off[sn] + (p - bt.par_off[sn]) * (bt.obs_off[sn + 1] - bt.obs_off[sn]),
                                    off[sn] + (p - bt.par_off[sn] + 1) * (bt.obs_off[sn + 1] - bt.obs_off[sn]))
                          for p, sn in zip(picks, sn_of)])
    pk = torch.as_tensor(picks, device=x2.device)
    gpu = (x2[pk].cpu().numpy(), g[pk].cpu().numpy(), bf[torch.as_tensor(idx, device=bf.device)].cpu().numpy())
    del bf
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    rx2, rg = o.chi2(sub, grad=True)
    t = time.perf_counter() - t0
    share = sub.n_bandflux() / max(bt.n_bandflux(), 1)
    return {"value": sub.n_bandflux() / t, "unit": UNIT, "cores": o.threads, "kind": "oracle",
            "sample": f"{len(picks)} seeded (supernova, sample) pairs of the batch (the first and last "
                      f"sample among them; {sub.n_bandflux()} bandfluxes, {share:.2e} of the step), "
                      f"chi2+grad, FP64 C with OpenMP ({t:.2f} s); the rate is per bandflux, so the "
                      f"whole step would take the oracle ~{t / share:.0f} s",
            "cpu_model": cpu_model(),
            "error_vs_oracle": error_vs_oracle(sub, gpu, (rx2, rg, o.bandflux(sub)))}


def secondary(args, salt_mod, torch, dev, stream, fp32_peak):
    """Shorter measurements of the other workloads (not the bench line), each
    guarded so that one failing record does not drop the others."""
    from paper_2504_08081_b300.torch_api import Salt
    out = {}
    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def timed_workload(wl, steps, sampled_pairs, max_par=2_000_000, full_oracle=False):
        """chi^2 + gradient steps of a workload (graph-timed, L2 flushed), its
        counted FLOP rate against the FP32 peak and, optionally, errors against
        the oracle on sampled pairs or on every output."""
        s = Salt(wl.model, wl.bands, device=dev.index or 0)
        try:
            with torch.cuda.stream(stream):
                db = s.upload(wl.batch)
                torch.cuda.synchronize()
                durs = time_steps_graph(lambda: s.chi2_grad(db), steps, 2, stream, flush=flush_buf.zero_) or \
                    time_steps(lambda: s.chi2_grad(db), steps, 2, stream, flush=flush_buf.zero_)
            ms = statistics.median(durs)
            fam, tile = s.last_kernel()
            nbf = wl.batch.n_bandflux()
            flops = algorithmic_flops(wl, grad=True, max_par=max_par)
            res = {"ms_per_step": ms, "bandfluxes_per_s": nbf / (ms / 1e3),
                   "chi2_grad_evals_per_s": wl.batch.n_par / (ms / 1e3), "bandfluxes": nbf,
                   "samples": wl.batch.n_par, "kernel": KERNEL_NAMES[fam].format(tile),
                   "grid": [wl.model.n_phase, wl.model.n_wave],
                   "achieved_tflops": flops / (ms / 1e3) / 1e12,
                   "frac_fp32": flops / (ms / 1e3) / 1e12 / fp32_peak}
            if sampled_pairs:
                res["cpu_baseline"] = sampled_oracle(wl, s, db, stream, n_picks=sampled_pairs)
            if full_oracle:
                with torch.cuda.stream(stream):
                    x2, g = s.chi2_grad(db)
                    bf = s.bandflux(db)
                torch.cuda.synchronize()
                res["cpu_baseline"] = cpu_baseline(wl, 2.0, gpu=(x2.cpu().numpy(), g.cpu().numpy(),
                                                                 bf.cpu().numpy()))
            return res
        finally:
            s.close()

    def guarded(name, fn):
        try:
            out[name] = fn()
        except Exception as ex:  # one record's failure must not sink the others
            out[name] = {"error": repr(ex)}

    # the 1000-supernova batched configuration (one sample each; every output
    # against the oracle) and the 256 x 1024 differentiation batch
    guarded(W.CONFIG_NAMES[2], lambda: timed_workload(make_workload(2, 0), 20, 0, full_oracle=True))
    guarded(W.CONFIG_NAMES[3], lambda: timed_workload(make_workload(3, 0), 5, 128, max_par=20000))

    def scaled_bench_workload():
        # the bench workload's shape at 10x the supernovae: how the one-sample
        # kernel's throughput grows once each warp has many units to run
        wl = W.config2(seed=1002, n_sn=10000)
        W.template_flux(wl.batch, np.random.default_rng(1003))
        return timed_workload(wl, 10, 0)
    guarded("batched_chi2_10000sn", scaled_bench_workload)

    def nonuniform_grid():
        # non-uniform (SALT3-NIR-shaped) grid: 66 x 991 nodes, binary-search indexing
        wl = W.config_nir(n_sn=4000, n_samples=4)
        W.template_flux(wl.batch, np.random.default_rng(1007))
        return timed_workload(wl, 10, 128)
    guarded("nir_nonuniform_4000sn_x4", nonuniform_grid)

    guarded("band_files", lambda: band_file_secondary(dev))

    def serving():
        from paper_2504_08081_b300 import serving as SV
        return SV.run_serving_bench(dev.index or 0)
    guarded(W.CONFIG_NAMES[4], serving)
    guarded("fit_" + W.CONFIG_NAMES[2], lambda: fit_secondary(dev, args.cpu_seconds))
    guarded("nested_" + W.CONFIG_NAMES[3], lambda: nested_secondary(dev, args.cpu_seconds))
    return out


def nested_secondary(dev, cpu_seconds, n_live=1024, n_batch=256, n_steps=10):
    """Nested sampling (salt_nested) of the 256-supernova differentiation
    batch with 1024 live points each (its 1024 samples per supernova as live
    points): observed fluxes are this library's bandfluxes at the truth plus
    5 % noise, prior box t0 +- 5 d, x0 x [0.5, 1.5], x1 in [-3, 3], c in
    [-0.3, 0.3]; beside it, the reference sampler on the FP64 oracle for one
    supernova with the same settings."""
    import torch
    import oracle
    import oracle.nested as NS
    from paper_2504_08081_b300.torch_api import Salt
    wl = make_workload(3, 0)
    s = Salt(wl.model, wl.bands, device=dev.index or 0)
    tb = W.truth_batch(wl.batch)
    m_true = s.bandflux(s.upload(tb, plan=False)).cpu().numpy()
    W.add_noise(tb, m_true, np.random.default_rng(2026))
    n = tb.n_sn
    ref = np.stack([tb.z, tb.t0, tb.x0, tb.x1, tb.c], axis=1).astype(np.float64)
    lo, hi = ref.copy(), ref.copy()
    lo[:, 1], hi[:, 1] = ref[:, 1] - 5.0, ref[:, 1] + 5.0
    lo[:, 2], hi[:, 2] = 0.5 * ref[:, 2], 1.5 * ref[:, 2]
    lo[:, 3], hi[:, 3] = -3.0, 3.0
    lo[:, 4], hi[:, 4] = -0.3, 0.3
    db = s.upload(tb)
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev).contiguous()  # noqa: E731
    kw = dict(n_live=n_live, n_batch=n_batch, n_steps=n_steps, seed=1)
    s.nested(db, T(lo), T(hi), **kw)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    logz, err, mean, std, st = s.nested(db, T(lo), T(hi), **kw)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = st.cpu().numpy()
    iters = int(st.max())
    # evaluations made: every supernova's live points, then its chains' steps
    # for the iterations it ran (a stopped supernova's chains are skipped)
    per_sn_iters = np.where(st >= 0, st, iters)
    evals = int(n * n_live + per_sn_iters.sum() * n_batch * n_steps)
    out = {"supernovae": n, "n_live": n_live, "n_batch": n_batch, "n_steps": n_steps,
           "wall_s": wall, "iterations_max": iters, "likelihood_evals": evals,
           "likelihood_evals_per_s": evals / wall, "posteriors_per_s": n / wall,
           "logz_err_median": float(np.median(err.cpu().numpy())),
           "timing": "wall clock around salt_nested (it synchronises)"}
    # counted chi^2-only FLOP per likelihood evaluation (the supernovae at their
    # truth), times the evaluation rate: the sampler's whole-run FP32 rate
    per_eval = algorithmic_flops(SimpleNamespace(model=wl.model, bands=wl.bands, batch=tb), grad=False) / n
    out["achieved_tflops"] = per_eval * evals / wall / 1e12
    s.close()
    o = oracle.Oracle(wl.model, wl.bands)
    t0 = time.perf_counter()
    r = NS.run_one(o, tb, 0, lo[0], hi[0], n_live=n_live, n_batch=n_batch, n_steps=n_steps, seed=1,
                   max_iter=max(1, int(cpu_seconds)))
    t_cpu = time.perf_counter() - t0
    ev_cpu = n_live + r["iterations"] * n_batch * n_steps
    out["cpu_baseline"] = {"value": ev_cpu / t_cpu, "unit": "likelihood evals/s", "cores": o.threads,
                           "kind": "oracle",
                           "sample": f"supernova 0, {r['iterations']} iterations of the reference sampler "
                                     f"(FP64 oracle chi^2, OpenMP over proposals, {t_cpu:.1f} s)"}
    return out


def band_file_secondary(dev):
    """Bandpass files (salt_band_load) and registration (salt_register_band):
    a 2001-sample transmission curve in nm, comma separated with a comment
    header, read and resampled onto 5 A, then added to a live context; wall
    time of each (host work plus the band-table upload)."""
    import tempfile
    from paper_2504_08081_b300 import _abi
    from paper_2504_08081_b300.torch_api import Salt
    wl = make_workload(2, 0)
    s = Salt(wl.model, wl.bands, device=dev.index or 0)
    lam_nm = np.linspace(400.0, 600.0, 2001)
    trans = np.exp(-0.5 * ((lam_nm - 500.0) / 30.0) ** 2)
    with tempfile.NamedTemporaryFile("w", suffix=".dat", delete=False) as f:
        f.write("# wavelength_nm, transmission\n")
        for a, t in zip(lam_nm, trans):
            f.write(f"{a:.4f}, {t:.8f}\n")
        path = f.name
    try:
        t0 = time.perf_counter()
        for _ in range(20):
            wave, tr = _abi.load_band(path, wave_scale=10.0, step=5.0)
        t_load = (time.perf_counter() - t0) / 20
        t0 = time.perf_counter()
        idx = s.register_band(wave, tr)
        t_reg = time.perf_counter() - t0
    finally:
        os.unlink(path)
    s.close()
    return {"file_samples": len(lam_nm), "resampled_samples": len(wave), "load_ms": 1e3 * t_load,
            "register_ms": 1e3 * t_reg, "band_index": idx}


def fit_secondary(dev, cpu_seconds):
    """Batched per-supernova fitting (salt_fit) of the 1000-supernova batch:
    observed fluxes are this library's bandfluxes at the truth plus 5 % noise,
    starts are perturbed from the truth; beside it, the reference minimiser
    (scipy L-BFGS-B on the FP64 oracle chi^2) on the first supernovae for a
    bounded time."""
    import torch
    from paper_2504_08081_b300.torch_api import Salt
    wl = make_workload(2, 0)
    s = Salt(wl.model, wl.bands, device=dev.index or 0)
    tb = W.truth_batch(wl.batch)
    m_true = s.bandflux(s.upload(tb, plan=False)).cpu().numpy()
    W.add_noise(wl.batch, m_true, np.random.default_rng(2024))
    start = W.fit_start(wl.batch, np.random.default_rng(2025))
    db = s.upload(start)
    s.fit(db)  # warm: tunes the chi^2 kernel for this layout
    walls, res = [], None
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = s.fit(db)
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
    th, f, st = (r.cpu().numpy() for r in res)
    ms = statistics.median(walls) * 1e3
    out = {"supernovae": start.n_sn, "ms_per_batch_fit": ms, "fits_per_s": start.n_sn / (ms / 1e3),
           "iterations_mean": float(st[st >= 0].mean()) if (st >= 0).any() else None,
           "iterations_max": int(st.max()), "converged": int((st >= 0).sum()),
           "timing": "wall clock around salt_fit (it synchronises), median of 3"}
    s.close()
    # reference minimiser on the host cores, bounded sample
    import oracle
    import oracle.fit as OF
    o = oracle.Oracle(wl.model, wl.bands)
    n_done, t = 0, 0.0
    while n_done < start.n_sn and t < cpu_seconds:
        t0 = time.perf_counter()
        OF.fit_one(o, start, n_done, gtol=1e-5, ftol=2.2e-9)
        t += time.perf_counter() - t0
        n_done += 1
    out["cpu_baseline"] = {"value": n_done / t, "unit": "fits/s", "cores": 1, "kind": "oracle",
                           "sample": f"first {n_done} supernovae, scipy L-BFGS-B (default-like "
                                     f"tolerances) on the FP64 oracle chi^2, one thread ({t:.1f} s)"}
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2504_08081_b300 import build as B
    B.build()
    from paper_2504_08081_b300.torch_api import Salt

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    wl = make_workload(args.workload, rank, args.n_sn)
    bt = wl.batch
    stream = torch.cuda.Stream(dev)
    salt = Salt(wl.model, wl.bands, device=local_rank)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    with torch.cuda.stream(stream):
        db = salt.upload(bt)
        chi2 = torch.empty(bt.n_par, dtype=torch.float64, device=dev)
        grad = torch.empty((bt.n_par, 5), dtype=torch.float32, device=dev)
        step = lambda: salt.chi2_grad(db, chi2, grad)  # noqa: E731
        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_rank) as clk:
            t_wall = time.perf_counter()
            durs = time_steps_graph(step, args.steps, 0, stream, flush=flush_buf.zero_)
            timing = "one CUDA graph of the K steps (flush, event, step, event), launched once"
            if durs is None:
                durs = time_steps(step, args.steps, 0, stream, flush=flush_buf.zero_)
                timing = "per-step events, steps queued behind a device-side spin"
            torch.cuda.synchronize()
            t_wall = time.perf_counter() - t_wall
        barrier()
        # host-inclusive latency of one synchronous call (not the bench value)
        sync_ms = statistics.median(time_steps(step, 10, 0, stream, flush=flush_buf.zero_, queue_ahead=False))
        salt.check()
    ms = statistics.mean(durs)
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": W.CONFIG_NAMES[args.workload], "ms_per_step": ms,
                              "bandfluxes": bt.n_bandflux()}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    ms_max, n_bf_all, n_par_all = reduce_over_ranks(ms, bt.n_bandflux(), bt.n_par, dev)
    value = n_bf_all / (ms_max / 1e3)

    # ---- end to end through the public API: pinned host inputs -> device -> host results.
    # The ten input arrays live in one pinned host buffer (each 256-byte aligned)
    # and go up in one transfer per step; the results come back in one transfer
    # per output. Two device input/output sets alternate, so that a step's
    # upload (copy stream) and download (output stream) overlap the neighbouring
    # steps' kernels (compute stream), as a user streaming batches would run it.
    obs_names = ["mjd", "band", "flux", "fluxerr", "zp"]
    par_names = ["t0", "z", "x0", "x1", "c"]
    src = {k: db.t[k].cpu() for k in obs_names + par_names}
    offs, total = {}, 0
    for k, v in src.items():
        offs[k] = total
        total += (v.numel() * v.element_size() + 255) // 256 * 256
    host_buf = torch.empty(total, dtype=torch.uint8).pin_memory()

    def view(buf, k):
        v = src[k]
        return buf[offs[k]:offs[k] + v.numel() * v.element_size()].view(v.dtype)

    for k in src:
        view(host_buf, k).copy_(src[k])
    from paper_2504_08081_b300.torch_api import DeviceBatch
    sets = []
    for _ in range(2):
        dbuf = torch.empty(total, dtype=torch.uint8, device=dev)
        sets.append(SimpleNamespace(
            buf=dbuf, db=DeviceBatch(db.obs_off, db.par_off, {k: view(dbuf, k) for k in src}, db.plan),
            chi2=torch.empty(bt.n_par, dtype=torch.float64, device=dev),
            grad=torch.empty((bt.n_par, 5), dtype=torch.float32, device=dev),
            chi2_h=torch.empty(bt.n_par, dtype=torch.float64).pin_memory(),
            grad_h=torch.empty((bt.n_par, 5), dtype=torch.float32).pin_memory(),
            ev_in=torch.cuda.Event(), ev_done=torch.cuda.Event(), ev_out=torch.cuda.Event()))
    h2d = total
    d2h = sets[0].chi2_h.numel() * 8 + sets[0].grad_h.numel() * 4
    copy_st = torch.cuda.Stream(device=dev)
    out_st = torch.cuda.Stream(device=dev)

    def e2e_step(i, flush=None):
        S = sets[i & 1]
        copy_st.wait_event(S.ev_done)          # step i-2's kernel has read this input set
        with torch.cuda.stream(copy_st):
            S.buf.copy_(host_buf, non_blocking=True)
        S.ev_in.record(copy_st)
        with torch.cuda.stream(stream):
            if flush is not None:
                flush()
            stream.wait_event(S.ev_in)
            stream.wait_event(S.ev_out)        # step i-2's results have left this output set
            salt.chi2_grad(S.db, S.chi2, S.grad)
            S.ev_done.record(stream)
        out_st.wait_event(S.ev_done)
        with torch.cuda.stream(out_st):
            S.chi2_h.copy_(S.chi2, non_blocking=True)
            S.grad_h.copy_(S.grad, non_blocking=True)
        S.ev_out.record(out_st)

    def e2e_span(steps, flush=None, queue_ahead=True):
        """Device time from the first upload to the last download of `steps`
        back-to-back steps (L2 flush, when given, inside the span before each
        kernel); the streams are held behind a spin until all are enqueued."""
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            if queue_ahead:
                torch.cuda._sleep(int(4e6) * max(1, steps // 4))
            e0.record(stream)
        copy_st.wait_event(e0)
        out_st.wait_event(e0)
        for i in range(steps):
            e2e_step(i, flush)
        stream.wait_stream(copy_st)
        stream.wait_stream(out_st)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    for i in range(max(args.warmup, 3)):
        e2e_step(i)
    torch.cuda.synchronize()
    # one step alone (upload, kernel, download in series), then the pipelined stream
    e2e_serial_ms = statistics.median(e2e_span(1, flush_buf.zero_) for _ in range(5))
    e2e_ms = e2e_span(args.steps, flush_buf.zero_)
    e2e_max, _, _ = reduce_over_ranks(e2e_ms, 0, 0, dev)
    e2e_value = n_bf_all / (e2e_max / 1e3)
    for S in sets:
        np.testing.assert_array_equal(S.chi2_h.numpy(), chi2.cpu().numpy())
        np.testing.assert_array_equal(S.grad_h.numpy(), grad.cpu().numpy())

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (the one the plan launched)
    fam, tile = salt.last_kernel()
    flops, grid_bytes = algorithmic_work(wl, grad=True, max_par=WORK_SAMPLES)
    work_how = ("exact count over every sample" if bt.n_par <= WORK_SAMPLES else
                f"counted over {WORK_SAMPLES} seeded samples of {bt.n_par}, scaled by their share")
    clocks = clk.summary()
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    max_mhz = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2032.0
    fp32_peak = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12  # TFLOP/s at the max SM clock
    achieved = flops / (ms / 1e3) / 1e12
    kname = KERNEL_NAMES[fam].format(tile)
    # the derived FP32 peak checked by the library's FMA microbenchmark (and the
    # L2 / shared-memory read bandwidths), measured after the timed region
    try:
        pk = salt.measure_peaks()
        peak_check = {"fp32_tflops_measured": pk["fp32_tflops"], "fp32_tflops_derived": sm_count * 128 * 2 *
                      max_mhz * 1e6 / 1e12, "l2_read_gbs": pk["l2_read_gbs"],
                      "smem_read_gbs": pk["smem_read_gbs"], "source": "salt_measure_peaks"}
    except Exception as ex:  # a diagnostic must not sink the bench line
        peak_check = {"error": repr(ex)}
    traffic, traffic_src = measured_traffic(kname, W.CONFIG_NAMES[args.workload])
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic, "traffic_source": traffic_src,
                "kernel": KERNEL_NAMES[fam].format(tile),
                "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                "flop_per_launch": flops, "flop_count": work_how,
                "ncu_counters": measured_counters(kname, W.CONFIG_NAMES[args.workload]),
                "peak_check": peak_check}
    # the same launch against the measured L2 read bandwidth: the grid values
    # the row dots must read (the kernel's on-chip gather)
    l2_peak = peak_check.get("l2_read_gbs")
    l2_achieved = grid_bytes / (ms / 1e3) / 1e9
    roofline_l2 = {"bound": "l2", "achieved": l2_achieved, "peak": l2_peak, "unit": "GB/s",
                   "frac": l2_achieved / l2_peak if l2_peak else None, "bytes_per_launch": grid_bytes,
                   "bytes": "grid values read by the row dots: touched rows x window columns x 8 B "
                            "per (sample, band)", "peak_source": "salt_measure_peaks (measured)"}

    # ---- CPU baseline: the oracle as it stands, on the host cores, and the
    # error of this step's results (and of a bandflux call) against its results:
    # whole passes of a batch it finishes in seconds, else seeded sampled pairs
    if bt.n_bandflux() <= 2_000_000:
        with torch.cuda.stream(stream):
            bf_gpu = salt.bandflux(db)
        torch.cuda.synchronize()
        cpu = cpu_baseline(wl, args.cpu_seconds,
                           gpu=(chi2.cpu().numpy(), grad.cpu().numpy(), bf_gpu.cpu().numpy()))
        del bf_gpu
    else:
        cpu = sampled_oracle(wl, salt, db, stream, budget_s=args.cpu_seconds, results=(chi2, grad))

    extras = {}
    if world == 1 and not args.no_extras:
        try:
            extras = secondary(args, None, torch, dev, stream, fp32_peak)
        except Exception as ex:  # secondary numbers must not sink the bench line
            extras = {"error": repr(ex)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 epoch difference and chi2 sum)",
        "data": "synthetic (seeded; model-free template fluxes)",
        "config": {"workload": W.CONFIG_NAMES[args.workload], "supernovae": bt.n_sn * world,
                   "bandfluxes_per_step": int(n_bf_all), "samples_per_step": int(n_par_all),
                   "bands": len(wl.bands), "grid": [wl.model.n_phase, wl.model.n_wave],
                   "step": "salt_chi2_grad (chi2 + adjoint gradient)",
                   "input_bytes": int(h2d),
                   "l2": "flushed between steps (256 MB write outside the timed events)" +
                         (f"; the inputs ({h2d / 1e9:.2f} GB) are larger than L2 as well"
                          if h2d > 126e6 else ""),
                   "timing": timing,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "chi2_grad_evals_per_s": n_par_all / (ms_max / 1e3),
        "ms_per_step_median": statistics.median(durs), "ms_per_step_min": min(durs),
        "ms_per_step_all": [round(d, 4) for d in durs],
        "sync_call_ms": sync_ms,
        "gpu_launches": args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_max,
                "method": "K back-to-back steps from pinned host memory: upload, L2 flush, "
                          "salt_chi2_grad, download of chi2 and grad; two device buffer sets, so "
                          "uploads and downloads overlap the neighbouring steps' kernels; span "
                          "from the first upload to the last download / K",
                "serial_ms_per_step": e2e_serial_ms,
                "serial_value": bt.n_bandflux() / (e2e_serial_ms / 1e3)},
        "roofline": roofline,
        "roofline_l2": roofline_l2,
        "cpu_baseline": cpu,
        "clocks": clocks,
        # host wall time of the timing call: capturing the K steps into a graph,
        # instantiating it and launching it twice (untimed, timed), with syncs
        "wall_s_timing_call": t_wall,
        "secondary": extras,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measured_traffic(kernel, workload):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    committed ncu capture summary, or None when there is none or the kernel's
    sources have changed since it was taken."""
    import hashlib
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(f"{kernel} @ {workload}")
    except (OSError, ValueError):
        return None, "no capture"
    if not rec:
        return None, "no capture of this kernel on this workload"
    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for f in rec["sources"]:
        h.update(open(os.path.join(root, f), "rb").read())
    if h.hexdigest() != rec["sources_sha256"]:
        return None, "kernel changed since the ncu capture"
    return rec["dram_read_bytes"] + rec["dram_write_bytes"], rec["summary"]


def measured_counters(kernel, workload):
    """The ncu counters (issue, FMA pipe, L2/L1 throughput, ...) of the same
    committed capture, under the same source check as measured_traffic."""
    traffic, src = measured_traffic(kernel, workload)
    if traffic is None:
        return None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "traffic.json")
    return json.load(open(path)).get(f"{kernel} @ {workload}", {}).get("counters")


def cpu_baseline(wl, budget_s, gpu=None):
    """The oracle timed on the host cores over whole passes of the batch; with
    `gpu` = (chi2, grad, bandflux) of this library on the same batch (numpy),
    also the error of those results against the oracle's."""
    import oracle
    o = oracle.Oracle(wl.model, wl.bands)
    bt = wl.batch
    done, n_bf, t = 0, 0, 0.0
    # whole batch passes until the budget is spent (at least one)
    while True:
        t0 = time.perf_counter()
        ref_x2, ref_g = o.chi2(bt, grad=True)
        t += time.perf_counter() - t0
        done += 1
        n_bf += bt.n_bandflux()
        if t >= budget_s or done >= 50:
            break
    out = {"value": n_bf / t, "unit": UNIT, "cores": o.threads, "kind": "oracle",
           "sample": f"{done} full pass(es) of the {bt.n_sn}-supernova batch, chi2+grad, "
                     f"FP64 C with OpenMP ({t:.1f} s)", "cpu_model": cpu_model()}
    # the same oracle on one thread, over the first supernovae (about 2 s)
    o1 = oracle.Oracle(wl.model, wl.bands, threads=1)
    n1 = min(bt.n_sn, 100)
    sub = W.subset(bt, np.arange(n1))
    t0 = time.perf_counter()
    o1.chi2(sub, grad=True)
    t1 = time.perf_counter() - t0
    out["single_thread"] = {"value": sub.n_bandflux() / t1, "unit": UNIT,
                            "sample": f"first {n1} supernovae, chi2+grad, one thread ({t1:.1f} s)"}
    if gpu is not None:
        out["error_vs_oracle"] = error_vs_oracle(bt, gpu, (ref_x2, ref_g, o.bandflux(bt)))
    return out


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo) and thread count."""
    name = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    name = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{name} ({os.cpu_count()} threads)"


def error_vs_oracle(bt, gpu, ref):
    """Worst errors of (chi2, grad, bandflux) against the FP64 oracle's, in the
    parity tests' measures: bandflux |dB| / max(|B|, 1e-3 max |B| of its
    supernova) (limit 1e-5); chi2 |dchi2| / chi2; gradient per sample
    |d(g s)|_inf / |g s|_inf with s = (0.01, 1 d, |x0|, 1, 0.1) (limit 1e-3)."""
    import oracle
    x2, g, bf = gpu
    rx2, rg, rbf = ref
    off = oracle.Oracle.bandflux_offsets(bt)
    scale = np.abs(rbf)
    for sn in range(bt.n_sn):
        lo, hi = off[sn], off[sn + 1]
        if hi > lo:
            scale[lo:hi] = np.maximum(scale[lo:hi], 1e-3 * np.abs(rbf[lo:hi]).max())
    bf_err = np.abs(bf.astype(np.float64) - rbf) / np.maximum(scale, 1e-300)
    x2_err = np.abs(x2 - rx2) / np.maximum(np.abs(rx2), 1e-300)
    sc = np.stack([np.full(bt.n_par, 0.01), np.ones(bt.n_par), np.abs(bt.x0.astype(np.float64)),
                   np.ones(bt.n_par), np.full(bt.n_par, 0.1)], 1)
    gs, rgs = g.astype(np.float64) * sc, rg * sc
    g_err = np.abs(gs - rgs).max(1) / np.maximum(np.abs(rgs).max(1), 1e-300)
    return {"bandflux_max_rel": float(bf_err.max()), "chi2_max_rel": float(x2_err.max()),
            "chi2_median_rel": float(np.median(x2_err)), "grad_max_scaled": float(g_err.max()),
            "bandfluxes_compared": int(bf.size), "samples_compared": int(x2.size),
            "limits": {"bandflux": 1e-5, "grad": 1e-3}}


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
