"""Serving client: replay a stream of chi^2 / chi^2+gradient requests against
the library's continuous-batching engine (salt_serve_submit / poll), and the
same stream as plain per-request launches for comparison.

Latency is the engine's own submit -> results-on-host time (steady clock in
the library); throughput is completed requests over the replay's wall time.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import _abi
from .torch_api import Salt


def _req_arrays(rq):
    b = rq.batch
    return dict(n_obs=b.n_obs, mjd=b.mjd, band=b.band, flux=b.flux, fluxerr=b.fluxerr, zp=b.zp,
                t0=b.t0, z=b.z, x0=b.x0, x1=b.x1, c=b.c, want_grad=rq.want_grad)


def _prepared(requests):
    """ctypes request descriptors and result buffers built ahead of the replay,
    so the timed loops only call into the library."""
    import ctypes as C
    out = []
    for rq in requests:
        b = rq.batch
        arrs = [np.ascontiguousarray(b.mjd, np.float64), np.ascontiguousarray(b.band, np.int32),
                np.ascontiguousarray(b.flux, np.float32), np.ascontiguousarray(b.fluxerr, np.float32),
                np.ascontiguousarray(b.zp, np.float32), np.ascontiguousarray(b.t0, np.float64),
                np.ascontiguousarray(b.z, np.float32), np.ascontiguousarray(b.x0, np.float32),
                np.ascontiguousarray(b.x1, np.float32), np.ascontiguousarray(b.c, np.float32)]
        req = _abi.Request(int(b.n_obs), len(arrs[5]), 1 if rq.want_grad else 0, *[a.ctypes.data for a in arrs])
        chi2 = np.empty(b.n_par, np.float64)
        grad = np.empty((b.n_par, 5), np.float32) if rq.want_grad else None
        out.append((req, arrs, chi2, grad, C.c_uint64()))
    return out


def replay(salt: Salt, requests, arrivals_s=None, collect=True):
    """Submit requests (at their arrival times when given, else all at once),
    wait for every result. Request descriptors and result buffers are built
    before the clock starts; the submitting and the polling thread then only
    call into the library (ctypes releases the interpreter lock meanwhile).
    Returns (wall seconds, results list, stats dict)."""
    import ctypes as C
    n = len(requests)
    prep = _prepared(requests)
    L = _abi.lib()
    h = salt.ctx.h
    tickets = [None] * n
    errors = []
    abort = [False]

    def poller():
        try:
            for i in range(n):
                while tickets[i] is None:
                    if abort[0]:
                        return
                    time.sleep(0)
                _, _, chi2, grad, _ = prep[i]
                rc = L.salt_serve_poll(h, tickets[i], -1, chi2.ctypes.data,
                                       grad.ctypes.data if grad is not None else None)
                if rc != _abi.SALT_OK:
                    errors.append((i, rc))
        except Exception as ex:  # pragma: no cover - surfaced below
            errors.append(("poller", repr(ex)))

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for i in range(n):
        if arrivals_s is not None:
            target = t0 + arrivals_s[i]
            while True:
                dt = target - time.perf_counter()
                if dt <= 0:
                    break
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
        req, _, _, _, tk = prep[i]
        rc = L.salt_serve_submit(h, C.byref(req), C.byref(tk))
        if rc != _abi.SALT_OK:
            errors.append((i, rc))
            abort[0] = True
            break
        tickets[i] = tk.value
    th.join()
    wall = time.perf_counter() - t0
    if errors:
        raise RuntimeError(f"serving errors: {errors[:5]}")
    results = [(p[2], p[3]) for p in prep] if collect else [None] * n
    return wall, results, salt.serve_stats()


def _request_array(prep):
    """ctypes array of salt_request descriptors (the prepared entries keep the
    host arrays alive)."""
    arr = (_abi.Request * max(1, len(prep)))()
    for i, p in enumerate(prep):
        arr[i] = p[0]
    return arr


def replay_native(salt: Salt, requests, arrivals_s=None, collect=False):
    """The replay of `replay` from the native client (salt_client_replay): a
    submitting and a polling thread in C++, no interpreter in the loop.
    Returns (wall seconds, results list or None, engine stats dict, client
    stats dict)."""
    import ctypes as C
    n = len(requests)
    prep = _prepared(requests)
    reqs = _request_array(prep)
    arr = None if arrivals_s is None else np.ascontiguousarray(arrivals_s, np.float64)
    c_out = g_out = None
    if collect:
        c_out = (C.c_void_p * n)(*[p[2].ctypes.data for p in prep])
        g_out = (C.c_void_p * n)(*[p[3].ctypes.data if p[3] is not None else None for p in prep])
    lat = np.zeros(n)
    st = _abi.ReplayStats()
    rc = _abi.client().salt_client_replay(salt.ctx.h, C.addressof(reqs), n,
                                          None if arr is None else arr.ctypes.data,
                                          None if c_out is None else C.addressof(c_out),
                                          None if g_out is None else C.addressof(g_out), lat.ctypes.data,
                                          C.byref(st))
    if rc != _abi.SALT_OK:
        raise _abi.SaltError(rc, "replay")
    results = [(p[2], p[3]) for p in prep] if collect else None
    cs = {"wall_s": st.wall_s, "submit_s": st.submit_s, "completed": int(st.completed),
          "client_p50_ms": st.p50_ms, "client_p99_ms": st.p99_ms}
    return st.wall_s, results, salt.serve_stats(), cs


def plain_native(salt: Salt, requests, limit_s: float = 8.0, pack_bytes: int = 1 << 30):
    """The same requests as plain per-request batch calls from the native
    client (salt_client_plain): inputs pre-packed in pinned memory, per request
    one upload into preallocated device buffers, one plan-less salt_chi2 /
    salt_chi2_grad, one download, a synchronisation. Returns (requests done,
    wall seconds, p50 ms, p99 ms)."""
    import ctypes as C
    prep = _prepared(requests)
    reqs = _request_array(prep)
    st = _abi.PlainStats()
    rc = _abi.client().salt_client_plain(salt.ctx.h, C.addressof(reqs), len(prep), limit_s, pack_bytes, None,
                                         C.byref(st))
    if rc != _abi.SALT_OK:
        raise _abi.SaltError(rc, "plain")
    return int(st.completed), st.wall_s, st.p50_ms, st.p99_ms


def plain_per_request(salt: Salt, requests, limit_s: float = 20.0):
    """Each request alone: its own upload, one launch, result download, sync.
    Returns (requests done, wall seconds, per-request latency ms)."""
    import torch
    lat = []
    t0 = time.perf_counter()
    k = 0
    for rq in requests:
        s0 = time.perf_counter()
        db = salt.upload(rq.batch, plan=False)
        if rq.want_grad:
            x2, g = salt.chi2_grad(db)
            x2.cpu(), g.cpu()
        else:
            salt.chi2(db).cpu()
        torch.cuda.current_stream().synchronize()
        lat.append(1e3 * (time.perf_counter() - s0))
        k += 1
        if time.perf_counter() - t0 > limit_s:
            break
    return k, time.perf_counter() - t0, lat


def run_serving_bench(device: int = 0, n_req: int = 20000, seed: int = 1004,
                      rates=(0.5, 0.8, 0.95), serve_mem: int = 512 << 20, max_replay_s: float = 8.0):
    """Saturated throughput, Poisson replays at fractions of it, and the plain
    per-request baseline on the same request stream, all driven by the native
    client (salt_client.h); beside them the device time of the same requests
    as two batch calls."""
    import workloads as W
    wl = W.config4(seed=seed, n_req=n_req)
    reqs = wl.requests
    out = {"requests": len(reqs),
           "samples_total": int(sum(r.batch.n_par for r in reqs)),
           "bandfluxes_total": int(sum(r.batch.n_par * r.batch.n_obs for r in reqs)),
           "client": "native (salt_client_replay / salt_client_plain: C++ threads over the C ABI)"}
    # saturated: everything submitted at once
    s = Salt(wl.model, wl.bands, device=device, serve_mem_bytes=serve_mem)
    replay_native(s, reqs[:500])  # warm the engine (first launches, allocator)
    s.close()
    s = Salt(wl.model, wl.bands, device=device, serve_mem_bytes=serve_mem)
    wall, _, st, cs = replay_native(s, reqs)
    sat = len(reqs) / wall
    out["saturated"] = {"req_per_s": sat, "bandfluxes_per_s": out["bandfluxes_total"] / wall,
                        "wall_s": wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                        "launches": st["launches"], **cs}
    s.close()
    rng = np.random.default_rng(seed + 1)
    for fr in rates:
        rate = fr * sat
        n = int(min(len(reqs), max(200, rate * max_replay_s)))
        arr = np.cumsum(rng.exponential(1.0 / rate, size=n))
        s = Salt(wl.model, wl.bands, device=device, serve_mem_bytes=serve_mem)
        wall, _, st, cs = replay_native(s, reqs[:n], arr)
        out[f"poisson_{fr:.2f}"] = {"offered_req_per_s": rate, "served_req_per_s": n / wall,
                                     "requests": n, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                                     "launches": st["launches"], **cs}
        s.close()
    # the same requests as two batch calls (the chi^2-only ones, the gradient
    # ones): the device time the stream needs without any serving machinery
    import torch
    s = Salt(wl.model, wl.bands, device=device)
    g_idx = [i for i, r in enumerate(reqs) if r.want_grad]
    c_idx = [i for i, r in enumerate(reqs) if not r.want_grad]
    dbg = s.upload(W.subset(wl.batch, g_idx))
    dbc = s.upload(W.subset(wl.batch, c_idx))
    for _ in range(2):  # tune and warm
        s.chi2_grad(dbg)
        s.chi2(dbc)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.chi2_grad(dbg)
    s.chi2(dbc)
    e1.record()
    e1.synchronize()
    gpu_s = e0.elapsed_time(e1) / 1e3
    out["batch_equivalent"] = {"device_s": gpu_s, "req_per_s": len(reqs) / gpu_s,
                               "bandfluxes_per_s": out["bandfluxes_total"] / gpu_s,
                               "how": "the whole stream as two batch calls (chi^2 only, chi^2 + gradient)"}
    out["saturated_vs_batch"] = sat / (len(reqs) / gpu_s)
    del dbg, dbc
    s.close()
    # plain per-request launches on the same stream (closed loop, bounded time)
    s = Salt(wl.model, wl.bands, device=device)
    plain_native(s, reqs[:50], limit_s=1.0)  # warm
    k, wall, p50, p99 = plain_native(s, reqs, limit_s=max_replay_s)
    out["plain_per_request"] = {"req_per_s": k / wall, "requests": k, "p50_ms": p50, "p99_ms": p99,
                                "how": "native loop over the C ABI: per request one upload from pinned "
                                       "memory into preallocated device buffers, a plan-less salt_chi2 / "
                                       "salt_chi2_grad, one download, a synchronisation"}
    out["batched_vs_plain_throughput"] = sat / (k / wall)
    s.close()
    return out
