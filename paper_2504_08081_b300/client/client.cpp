// Native load generator over the public C ABI (salt_client.h): a replay of a
// request stream against the serving engine, and the same requests as plain
// per-request batch calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "salt_client.h"

namespace {

using Clock = std::chrono::steady_clock;

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t lo = (size_t)pos, hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// Byte layout of one request's inputs, the same in the pinned pack and in the
// device buffer: the two float64 arrays first, then the 32-bit ones.
struct Layout {
    size_t mjd, t0, band, flux, fluxerr, zp, z, x0, x1, c, total;
    explicit Layout(const salt_request &r) {
        const size_t n = (size_t)r.n_obs, s = (size_t)r.n_par;
        size_t o = 0;
        auto take = [&](size_t bytes) { const size_t at = o; o = al16(o + bytes); return at; };
        mjd = take(8 * n);
        t0 = take(8 * s);
        band = take(4 * n);
        flux = take(4 * n);
        fluxerr = take(4 * n);
        zp = take(4 * n);
        z = take(4 * s);
        x0 = take(4 * s);
        x1 = take(4 * s);
        c = take(4 * s);
        total = o;
    }
};

}  // namespace

extern "C" int salt_client_replay(salt_ctx *ctx, const salt_request *reqs, int32_t n, const double *arrival_s,
                                  double *const *chi2_out, float *const *grad_out, double *lat_ms,
                                  salt_replay_stats *out) {
    if (!ctx || !out || n < 0 || (n > 0 && !reqs)) return SALT_ERR_INVALID;
    std::memset(out, 0, sizeof(*out));
    if (n == 0) return SALT_OK;
    int max_par = 1;
    for (int i = 0; i < n; ++i) max_par = std::max(max_par, reqs[i].n_par);
    std::vector<uint64_t> tickets((size_t)n, 0);
    std::vector<std::atomic<int>> state((size_t)n);  // 0 waiting, 1 submitted, 2 refused
    for (auto &s : state) s.store(0, std::memory_order_relaxed);
    std::vector<Clock::time_point> t_arr((size_t)n), t_done((size_t)n);
    std::atomic<int> first_err{SALT_OK};
    Clock::time_point t_sub_end;
    const Clock::time_point t0 = Clock::now();

    std::thread submitter([&] {
        for (int i = 0; i < n; ++i) {
            Clock::time_point due = t0;
            if (arrival_s) {
                due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
                for (;;) {
                    const double left = secs(Clock::now(), due);
                    if (left <= 0.0) break;
                    if (left > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(left - 1e-4));
                }
            }
            t_arr[(size_t)i] = arrival_s ? due : Clock::now();
            const int rc = salt_serve_submit(ctx, &reqs[i], &tickets[(size_t)i]);
            if (rc != SALT_OK) {
                int expect = SALT_OK;
                first_err.compare_exchange_strong(expect, rc);
                state[(size_t)i].store(2, std::memory_order_release);
            } else {
                state[(size_t)i].store(1, std::memory_order_release);
            }
        }
        t_sub_end = Clock::now();
    });

    // The poller sweeps, without waiting, the oldest outstanding requests (a
    // window of kWin), so a request's completion time is taken when its own
    // results are ready (within the back-off below), not after the slower
    // requests submitted before it.
    constexpr int kWin = 32;
    std::vector<double> chi2_tmp((size_t)max_par);
    std::vector<float> grad_tmp(5 * (size_t)max_par);
    std::vector<char> fin((size_t)n, 0);
    int64_t done = 0;
    int head = 0;  // every request before head is finished
    while (head < n) {
        bool progress = false;
        const int end = std::min(n, head + kWin);
        for (int i = head; i < end; ++i) {
            if (fin[(size_t)i]) continue;
            const int st = state[(size_t)i].load(std::memory_order_acquire);
            if (st == 0) break;  // not submitted yet: neither are the later ones
            if (st == 2) { fin[(size_t)i] = 1; progress = true; continue; }
            double *c2 = (chi2_out && chi2_out[i]) ? chi2_out[i] : chi2_tmp.data();
            float *g = (grad_out && grad_out[i]) ? grad_out[i] : grad_tmp.data();
            const int rc = salt_serve_poll(ctx, tickets[(size_t)i], 0, c2, reqs[i].want_grad ? g : nullptr);
            if (rc == SALT_PENDING) continue;
            t_done[(size_t)i] = Clock::now();
            fin[(size_t)i] = 1;
            progress = true;
            if (rc == SALT_OK) {
                ++done;
            } else {
                int expect = SALT_OK;
                first_err.compare_exchange_strong(expect, rc);
            }
        }
        while (head < n && fin[(size_t)head]) ++head;
        // nothing ready: back off briefly, so the polls do not keep the engine
        // lock from the submitting thread and the scheduler
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    submitter.join();
    const Clock::time_point t_end = Clock::now();
    std::vector<double> lat;
    lat.reserve((size_t)n);
    for (int i = 0; i < n; ++i) {
        if (state[(size_t)i].load() != 1) continue;
        const double ms = 1e3 * secs(t_arr[(size_t)i], t_done[(size_t)i]);
        lat.push_back(ms);
        if (lat_ms) lat_ms[i] = ms;
    }
    out->wall_s = secs(t0, t_end);
    out->submit_s = secs(t0, t_sub_end);
    out->completed = done;
    out->p50_ms = percentile(lat, 0.50);
    out->p99_ms = percentile(lat, 0.99);
    return first_err.load();
}

extern "C" int salt_client_plain(salt_ctx *ctx, const salt_request *reqs, int32_t n, double time_limit_s,
                                 size_t pack_bytes, double *lat_ms, salt_plain_stats *out) {
    if (!ctx || !out || n < 0 || (n > 0 && !reqs)) return SALT_ERR_INVALID;
    std::memset(out, 0, sizeof(*out));
    if (n == 0) return SALT_OK;
    // requests that fit the pack, their offsets in it, and the largest one
    std::vector<size_t> at;
    size_t total = 0, max_in = 0;
    int max_par = 1, m = 0;
    for (; m < n; ++m) {
        const Layout L(reqs[m]);
        if (total + L.total > pack_bytes) break;
        at.push_back(total);
        total += L.total;
        max_in = std::max(max_in, L.total);
        max_par = std::max(max_par, reqs[m].n_par);
    }
    if (m == 0) return SALT_ERR_INVALID;
    unsigned char *pack = nullptr, *din = nullptr;
    double *dchi2 = nullptr, *hchi2 = nullptr;
    float *dgrad = nullptr, *hgrad = nullptr;
    cudaStream_t st = nullptr;
    int rc = SALT_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == SALT_OK) rc = e == cudaErrorMemoryAllocation ? SALT_ERR_OOM : SALT_ERR_CUDA;
        return rc == SALT_OK;
    };
    if (ck(cudaHostAlloc((void **)&pack, total, cudaHostAllocDefault)) && ck(cudaMalloc((void **)&din, max_in)) &&
        ck(cudaMalloc((void **)&dchi2, 8 * (size_t)max_par)) && ck(cudaMalloc((void **)&dgrad, 20 * (size_t)max_par)) &&
        ck(cudaHostAlloc((void **)&hchi2, 8 * (size_t)max_par, cudaHostAllocDefault)) &&
        ck(cudaHostAlloc((void **)&hgrad, 20 * (size_t)max_par, cudaHostAllocDefault)) &&
        ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) {
        for (int i = 0; i < m; ++i) {
            const salt_request &r = reqs[i];
            const Layout L(r);
            unsigned char *p = pack + at[(size_t)i];
            const size_t nn = (size_t)r.n_obs, s = (size_t)r.n_par;
            if (nn) {
                std::memcpy(p + L.mjd, r.mjd, 8 * nn);
                std::memcpy(p + L.band, r.band, 4 * nn);
                std::memcpy(p + L.flux, r.flux, 4 * nn);
                std::memcpy(p + L.fluxerr, r.fluxerr, 4 * nn);
                std::memcpy(p + L.zp, r.zp, 4 * nn);
            }
            std::memcpy(p + L.t0, r.t0, 8 * s);
            std::memcpy(p + L.z, r.z, 4 * s);
            std::memcpy(p + L.x0, r.x0, 4 * s);
            std::memcpy(p + L.x1, r.x1, 4 * s);
            std::memcpy(p + L.c, r.c, 4 * s);
        }
        std::vector<double> lat;
        const Clock::time_point t0 = Clock::now();
        for (int k = 0; k < m && rc == SALT_OK; ++k) {
            const salt_request &r = reqs[k];
            const Layout L(r);
            const Clock::time_point s0 = Clock::now();
            if (!ck(cudaMemcpyAsync(din, pack + at[(size_t)k], L.total, cudaMemcpyHostToDevice, st))) break;
            const int64_t oo[2] = {0, r.n_obs}, po[2] = {0, r.n_par};
            salt_batch b{};
            b.n_sn = 1;
            b.obs_off = oo;
            b.par_off = po;
            b.mjd = (const double *)(din + L.mjd);
            b.band = (const int32_t *)(din + L.band);
            b.flux = (const float *)(din + L.flux);
            b.fluxerr = (const float *)(din + L.fluxerr);
            b.zp = (const float *)(din + L.zp);
            b.t0 = (const double *)(din + L.t0);
            b.z = (const float *)(din + L.z);
            b.x0 = (const float *)(din + L.x0);
            b.x1 = (const float *)(din + L.x1);
            b.c = (const float *)(din + L.c);
            const int crc = r.want_grad ? salt_chi2_grad(ctx, &b, dchi2, dgrad, st) : salt_chi2(ctx, &b, dchi2, st);
            if (crc != SALT_OK) { rc = crc; break; }
            if (!ck(cudaMemcpyAsync(hchi2, dchi2, 8 * (size_t)r.n_par, cudaMemcpyDeviceToHost, st))) break;
            if (r.want_grad && !ck(cudaMemcpyAsync(hgrad, dgrad, 20 * (size_t)r.n_par, cudaMemcpyDeviceToHost, st)))
                break;
            if (!ck(cudaStreamSynchronize(st))) break;
            const double ms = 1e3 * secs(s0, Clock::now());
            lat.push_back(ms);
            if (lat_ms) lat_ms[k] = ms;
            if (secs(t0, Clock::now()) > time_limit_s) break;
        }
        out->wall_s = secs(t0, Clock::now());
        out->completed = (int64_t)lat.size();
        out->p50_ms = percentile(lat, 0.50);
        out->p99_ms = percentile(lat, 0.99);
    }
    if (st) cudaStreamDestroy(st);
    if (hgrad) cudaFreeHost(hgrad);
    if (hchi2) cudaFreeHost(hchi2);
    if (dgrad) cudaFree(dgrad);
    if (dchi2) cudaFree(dchi2);
    if (din) cudaFree(din);
    if (pack) cudaFreeHost(pack);
    (void)cudaGetLastError();
    return rc;
}
