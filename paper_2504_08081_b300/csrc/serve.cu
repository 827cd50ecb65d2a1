// Serving engine: continuous batching of chi^2 / chi^2+gradient requests.
//
// Requests (one supernova each, any number of samples) are copied at submit,
// queued, and admitted while their observations and samples fit the device
// arenas (memory admission). The arenas are structure-of-arrays: every
// observation array (mjd, band, flux, fluxerr, zp) shares one element index
// space and every sample array (t0, z, x0, x1, c, chi2, grad) another, so one
// work item addresses a request's data with a single element offset. A
// scheduler thread turns the admitted requests' fixed-size sample chunks
// (8 samples: one tile, so a request's items spread over many CTAs and finish
// fast) into one ragged work list per (mode, tile) and launches the fused
// factorised kernel over it; requests that arrive while earlier launches run
// on the GPU join the next one, and with 8 launch groups in flight new
// requests wait to be grouped into larger ones. A tick's admitted requests are
// packed into a pinned staging buffer and uploaded with one copy per array and
// one scatter kernel. Uploads, kernels and downloads run on three streams
// ordered by events, so copies overlap other requests' kernels; a launch
// group's results are downloaded right behind its kernel, with one copy per
// result array over the arena range its requests occupy (per request when
// that range is mostly other requests' space). A submission
// wakes the scheduler only when it is idle; while work is queued or in
// flight the scheduler comes back every ~20 us by itself, so a burst of
// submissions neither waits on a scheduler pass per request nor splits into
// one launch per request. A request's
// chunks go through exactly the same per-item code whatever else shares the
// launch, so its results are bitwise identical alone and in a mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <list>

#include "salt_internal.cuh"

namespace salt {

namespace {

using Clock = std::chrono::steady_clock;

double now_ms() {
    return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}

// First-fit allocator over element range [0, size) with a coalescing free list.
class RangeAlloc {
  public:
    explicit RangeAlloc(size_t size) : size_(size) {
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t &off) {
        n = std::max<size_t>(n, 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n, noff = it->first + n;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = std::max<size_t>(n, 1);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

  private:
    size_t size_, used_ = 0;
    std::map<size_t, size_t> free_;
};

// ADMITTING: arena ranges taken, inputs being packed and uploaded by the scheduler
// outside the engine lock (poll and cancel only flag it)
enum class St { QUEUED, ADMITTING, ACTIVE, DONE, CANCELLED, FAILED };

struct Req {
    uint64_t ticket = 0;
    int n_obs = 0, n_par = 0;
    bool grad = false;
    int tile = 1;
    size_t oo = SIZE_MAX, po = SIZE_MAX;  // element offsets in the observation / sample arenas
    St st = St::QUEUED;
    bool cancel = false;
    bool launched = false;
    int inflight = 0;  // launches referencing this request that have not completed
    double t_submit = 0, t_done = 0;
    // inputs until admitted, in one buffer: mjd [n_obs], t0 [n_par] (float64),
    // band, flux, fluxerr, zp [n_obs], z, x0, x1, c [n_par] (32-bit)
    std::unique_ptr<unsigned char[]> in;
    std::vector<double> chi2;  // results
    std::vector<float> gout;
    const double *mjd() const { return (const double *)in.get(); }
    const double *t0() const { return mjd() + n_obs; }
    const int32_t *band() const { return (const int32_t *)(t0() + n_par); }
    const float *f32(int k) const { return (const float *)(band() + n_obs) + (size_t)k * n_obs; }  // flux, fluxerr, zp
    const float *par32(int k) const { return f32(3) + (size_t)k * n_par; }                         // z, x0, x1, c
    static size_t in_bytes(int n, int S) { return 8 * ((size_t)n + S) + 4 * (4 * (size_t)n + 4 * (size_t)S); }
};

struct Launch {
    cudaEvent_t ev = nullptr;  // the group's results are in the host mirrors
    std::vector<uint64_t> reqs;
    int slot = -1;
};

constexpr int kSlots = 16;          // item-list buffers (launch groups in flight)
constexpr int kMaxItems = 1 << 15;  // items per launch group

// bytes one observation / one sample occupies across all arrays
constexpr size_t kObsBytes = 8 + 4 * 4;        // mjd, band, flux, fluxerr, zp
constexpr size_t kParBytes = 8 + 4 * 4 + 8 + 20;  // t0, z, x0, x1, c, chi2, grad[5]

// Upload staging: the requests admitted in one tick are packed into a pinned
// buffer, copied with one transfer per array and scattered into the arenas by
// one kernel (instead of ten small pageable copies per request). Two buffers
// alternate so the host fills one while the other is in flight.
constexpr size_t kStageObs = size_t(1) << 19;  // observations per staging buffer
constexpr size_t kStagePar = size_t(1) << 19;  // samples per staging buffer
constexpr int kStageReq = 8192;                // requests per staging buffer

struct UpDesc {  // one request: where its rows sit in the staging buffer and in the arenas
    int64_t src_obs, dst_obs, n_obs, src_par, dst_par, n_par;
};

struct StageLayout {  // byte offsets inside a staging buffer (host and device alike)
    size_t mjd, t0, band, flux, fluxerr, zp, z, x0, x1, c, desc, total;
    StageLayout() {
        size_t o = 0;
        auto take = [&](size_t bytes) { const size_t at = o; o += (bytes + 255) & ~size_t(255); return at; };
        mjd = take(8 * kStageObs);
        t0 = take(8 * kStagePar);
        band = take(4 * kStageObs);
        flux = take(4 * kStageObs);
        fluxerr = take(4 * kStageObs);
        zp = take(4 * kStageObs);
        z = take(4 * kStagePar);
        x0 = take(4 * kStagePar);
        x1 = take(4 * kStagePar);
        c = take(4 * kStagePar);
        desc = take(sizeof(UpDesc) * kStageReq);
        total = o;
    }
};

struct Stage {
    unsigned char *h = nullptr, *d = nullptr;
    cudaEvent_t ev = nullptr;  // the last upload from this buffer has finished
    bool busy = false;
};

}  // namespace

struct ServeEngine {
    salt_ctx *ctx = nullptr;
    RangeAlloc obs_a, par_a;
    // device arrays (SoA) and their pinned host mirrors
    double *d_mjd = nullptr, *d_t0 = nullptr, *d_chi2 = nullptr;
    int32_t *d_band = nullptr;
    float *d_flux = nullptr, *d_fluxerr = nullptr, *d_zp = nullptr, *d_z = nullptr, *d_x0 = nullptr,
          *d_x1 = nullptr, *d_c = nullptr, *d_grad = nullptr;
    double *h_chi2 = nullptr;
    float *h_grad = nullptr;
    cudaStream_t s_up = nullptr, s_comp = nullptr, s_down = nullptr;
    cudaEvent_t ev_up = nullptr;
    WorkItem *items_d[kSlots] = {};
    WorkItem *items_h[kSlots] = {};
    int *counters_d = nullptr;
    bool slot_busy[kSlots] = {};
    Stage stage[2];
    int stage_cur = 0;
    StageLayout SL;
    int max_inflight = 8;  // launch groups in flight before new requests wait to be grouped
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    // requests by state, so a tick touches only what can change
    std::vector<uint64_t> pending[2][4];  // admitted, not launched: [chi2 / grad][tile 1, 2, 4, 8]
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::list<Launch> inflight;
    std::vector<double> lat_ms;
    std::vector<cudaEvent_t> ev_pool;  // recycled launch events
    uint64_t next_ticket = 1;
    uint64_t n_submitted = 0, n_completed = 0, n_cancelled = 0, n_rejected = 0, n_launches = 0;
    bool stop = false;
    bool idle = false;  // the engine thread waits for work with nothing queued or in flight
    std::string fatal;
    std::thread th;

    ServeEngine(size_t obs_cap, size_t par_cap) : obs_a(obs_cap), par_a(par_cap) {}
};

namespace {

void fail_all(ServeEngine *e, const std::string &why) {
    e->fatal = why;
    for (auto &kv : e->reqs)
        if (kv.second->st != St::DONE && kv.second->st != St::CANCELLED) kv.second->st = St::FAILED;
    e->cv_done.notify_all();
}

void release_req(ServeEngine *e, Req &r) {
    if (r.oo != SIZE_MAX) e->obs_a.release(r.oo, (size_t)r.n_obs);
    if (r.po != SIZE_MAX) e->par_a.release(r.po, (size_t)r.n_par);
    r.oo = r.po = SIZE_MAX;
}

cudaError_t pool_event(ServeEngine *e, cudaEvent_t *ev) {
    if (!e->ev_pool.empty()) {
        *ev = e->ev_pool.back();
        e->ev_pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
}

// Scatter one tick's staged requests into the arenas: thread per row.
__global__ void k_stage_scatter(const unsigned char *stg, StageLayout L, int n_desc, int64_t n_obs, int64_t n_par,
                                double *mjd, int32_t *band, float *flux, float *fluxerr, float *zp, double *t0,
                                float *z, float *x0, float *x1, float *c) {
    const UpDesc *d = (const UpDesc *)(stg + L.desc);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_obs; i += stride) {
        int lo = 0, hi = n_desc;  // the last request whose rows start at or before i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (d[mid].src_obs <= i) lo = mid; else hi = mid;
        }
        const int64_t o = d[lo].dst_obs + (i - d[lo].src_obs);
        mjd[o] = ((const double *)(stg + L.mjd))[i];
        band[o] = ((const int32_t *)(stg + L.band))[i];
        flux[o] = ((const float *)(stg + L.flux))[i];
        fluxerr[o] = ((const float *)(stg + L.fluxerr))[i];
        zp[o] = ((const float *)(stg + L.zp))[i];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_par; i += stride) {
        int lo = 0, hi = n_desc;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (d[mid].src_par <= i) lo = mid; else hi = mid;
        }
        const int64_t q = d[lo].dst_par + (i - d[lo].src_par);
        t0[q] = ((const double *)(stg + L.t0))[i];
        z[q] = ((const float *)(stg + L.z))[i];
        x0[q] = ((const float *)(stg + L.x0))[i];
        x1[q] = ((const float *)(stg + L.x1))[i];
        c[q] = ((const float *)(stg + L.c))[i];
    }
}

int tile_for(int n_par) {
    if (n_par >= 8) return 8;
    if (n_par >= 4) return 4;
    if (n_par >= 2) return 2;
    return 1;
}

template <class T>
cudaError_t up(T *dst, const T *src, size_t n, size_t off, cudaStream_t st) {
    if (!n) return cudaSuccess;
    return cudaMemcpyAsync(dst + off, src, n * sizeof(T), cudaMemcpyHostToDevice, st);
}

// Enqueue, on the download stream, the copies of a launch group's results
// into the host mirrors: one copy per result array over the arena range the
// group's requests span when that range is at most twice their samples (plus
// a margin), else one copy per request. Copying other requests' space as well
// is harmless: a request's results are read from the mirror only after its
// own group's download, and only its own kernel writes them on the device.
cudaError_t download_results(ServeEngine *e, const std::vector<Req *> &members, bool grad) {
    size_t lo = SIZE_MAX, hi = 0, need = 0;
    for (const Req *rp : members) {
        const Req &r = *rp;
        lo = std::min(lo, r.po);
        hi = std::max(hi, r.po + (size_t)r.n_par);
        need += (size_t)r.n_par;
    }
    cudaError_t err = cudaSuccess;
    if (hi > lo && hi - lo <= 2 * need + 4096) {
        err = cudaMemcpyAsync(e->h_chi2 + lo, e->d_chi2 + lo, 8 * (hi - lo), cudaMemcpyDeviceToHost, e->s_down);
        if (err == cudaSuccess && grad)
            err = cudaMemcpyAsync(e->h_grad + 5 * lo, e->d_grad + 5 * lo, 20 * (hi - lo), cudaMemcpyDeviceToHost,
                                  e->s_down);
        return err;
    }
    for (const Req *rp : members) {
        const Req &r = *rp;
        err = cudaMemcpyAsync(e->h_chi2 + r.po, e->d_chi2 + r.po, 8 * (size_t)r.n_par, cudaMemcpyDeviceToHost,
                              e->s_down);
        if (err == cudaSuccess && grad)
            err = cudaMemcpyAsync(e->h_grad + 5 * r.po, e->d_grad + 5 * r.po, 20 * (size_t)r.n_par,
                                  cudaMemcpyDeviceToHost, e->s_down);
        if (err != cudaSuccess) return err;
    }
    return err;
}

// One scheduler pass, entered and left with the engine lock held. Under the
// lock it retires finished launch groups, takes arena ranges for the queued
// requests that fit (FIFO; they become ADMITTING) and picks the launch groups;
// it then releases the lock while it packs and uploads the admitted requests
// and builds and launches the groups (submit, poll and cancel go on meanwhile:
// the requests it works on are ADMITTING or already marked launched, which
// poll and cancel only flag, and it reaches them through their own pointers,
// never through the request map), and commits under the lock again. Returns
// false after a CUDA error.
bool tick(ServeEngine *e, std::unique_lock<std::mutex> &lk) {
    cudaError_t err;
    // 1. retire launch groups whose results have reached the host mirrors
    bool finished = false;
    for (auto it = e->inflight.begin(); it != e->inflight.end();) {
        err = cudaEventQuery(it->ev);
        if (err == cudaErrorNotReady) { ++it; continue; }
        if (err != cudaSuccess) { fail_all(e, cudaGetErrorString(err)); return false; }
        const double t = now_ms();
        for (uint64_t tk : it->reqs) {
            auto rq = e->reqs.find(tk);
            if (rq == e->reqs.end()) continue;
            Req &r = *rq->second;
            if (--r.inflight > 0) continue;
            if (!r.cancel) {
                r.t_done = t;
                r.chi2.assign(e->h_chi2 + r.po, e->h_chi2 + r.po + r.n_par);
                if (r.grad) r.gout.assign(e->h_grad + 5 * r.po, e->h_grad + 5 * (r.po + r.n_par));
            }
            release_req(e, r);
            r.st = r.cancel ? St::CANCELLED : St::DONE;
            if (r.st == St::DONE) {
                e->lat_ms.push_back(r.t_done - r.t_submit);
                e->n_completed++;
            }
            finished = true;
        }
        e->ev_pool.push_back(it->ev);
        e->slot_busy[it->slot] = false;
        it = e->inflight.erase(it);
    }
    if (finished) e->cv_done.notify_all();

    // 2. admission: arena ranges for the queued requests while both arenas (and
    // the staging buffer) have room, FIFO
    Stage *sg = nullptr;
    for (int t = 0; t < 2 && !sg; ++t) {
        Stage &c = e->stage[(e->stage_cur + t) & 1];
        if (c.busy) {
            err = cudaEventQuery(c.ev);
            if (err == cudaErrorNotReady) continue;
            if (err != cudaSuccess) { fail_all(e, cudaGetErrorString(err)); return false; }
            c.busy = false;
        }
        sg = &c;
        e->stage_cur = (e->stage_cur + t) & 1;
    }
    struct Adm {
        Req *r;
        size_t so, sp;  // rows in the staging buffer (not used for direct uploads)
        bool direct;
    };
    std::vector<Adm> adm;
    size_t so = 0, sp = 0;  // staged observations / samples this pass
    int nd = 0;
    while (!e->queue.empty()) {
        auto rq = e->reqs.find(e->queue.front());
        if (rq == e->reqs.end() || rq->second->st != St::QUEUED) { e->queue.pop_front(); continue; }
        Req &r = *rq->second;
        // requests larger than a staging buffer go straight to the arenas
        const bool direct = (size_t)r.n_obs > kStageObs || (size_t)r.n_par > kStagePar;
        if (!direct && (!sg || so + r.n_obs > kStageObs || sp + r.n_par > kStagePar || nd >= kStageReq)) break;
        size_t oo = SIZE_MAX, po = SIZE_MAX;
        if (!e->par_a.alloc((size_t)r.n_par, po)) break;
        if (!e->obs_a.alloc((size_t)r.n_obs, oo)) { e->par_a.release(po, (size_t)r.n_par); break; }
        r.oo = oo;
        r.po = po;
        adm.push_back(Adm{&r, so, sp, direct});
        if (!direct) {
            so += r.n_obs;
            sp += r.n_par;
            ++nd;
        }
        r.st = St::ADMITTING;
        e->pending[r.grad ? 1 : 0][r.tile == 1 ? 0 : r.tile == 2 ? 1 : r.tile == 4 ? 2 : 3].push_back(r.ticket);
        e->queue.pop_front();
    }

    // 3. launch groups: one per (mode, tile) over the requests admitted and not
    // yet launched (this pass's included: their uploads come first in stream
    // order); while enough launches keep the GPU busy, requests gather into
    // larger groups
    const int chunk = std::max(1, e->ctx->serve_chunk);
    struct Grp {
        int mode, tile, slot;
        std::vector<Req *> members;
        std::vector<uint64_t> tickets;
        cudaEvent_t ev;
    };
    std::vector<Grp> grps;
    for (int mode = MODE_CHI2; mode <= MODE_GRAD; ++mode) {
        for (int ti = 0; ti < 4; ++ti) {
            std::vector<uint64_t> &bucket = e->pending[mode == MODE_GRAD ? 1 : 0][ti];
            if (bucket.empty()) continue;
            if ((int)(e->inflight.size() + grps.size()) >= e->max_inflight) break;
            int slot = -1;
            for (int q = 0; q < kSlots; ++q)
                if (!e->slot_busy[q]) { slot = q; break; }
            if (slot < 0) break;  // all item buffers in flight: next pass
            Grp G{mode, 1 << ti, slot, {}, {}, nullptr};
            std::vector<uint64_t> later;
            int n_items = 0;
            for (uint64_t t : bucket) {
                auto rq = e->reqs.find(t);
                if (rq == e->reqs.end()) continue;
                Req &r = *rq->second;
                if ((r.st != St::ACTIVE && r.st != St::ADMITTING) || r.launched || r.cancel) continue;
                // a request too large for one item list takes larger chunks
                const int cr = std::max(chunk, (r.n_par + kMaxItems - 1) / kMaxItems);
                const int need = (r.n_par + cr - 1) / cr;
                if (n_items + need > kMaxItems) { later.push_back(t); continue; }
                n_items += need;
                r.launched = true;
                r.inflight = 1;
                G.members.push_back(&r);
                G.tickets.push_back(t);
            }
            bucket.swap(later);
            if (G.members.empty()) continue;
            err = pool_event(e, &G.ev);
            if (err != cudaSuccess) { fail_all(e, cudaGetErrorString(err)); return false; }
            e->slot_busy[slot] = true;
            grps.push_back(std::move(G));
        }
    }
    if (adm.empty() && grps.empty()) return true;

    // 4. outside the lock: pack and upload the admitted requests, build and
    // launch the groups, and queue their result downloads
    Stage *sgu = nd > 0 ? sg : nullptr;
    lk.unlock();
    err = cudaSuccess;
    const StageLayout &SL = e->SL;
    for (const Adm &ad : adm) {
        if (err != cudaSuccess) break;
        const Req &r = *ad.r;
        const size_t n = (size_t)r.n_obs, S = (size_t)r.n_par, oo = r.oo, po = r.po;
        if (ad.direct) {
            // pageable sources: each copy is staged by the driver before the call returns
            err = up(e->d_mjd, r.mjd(), n, oo, e->s_up);
            if (err == cudaSuccess) err = up(e->d_band, r.band(), n, oo, e->s_up);
            if (err == cudaSuccess) err = up(e->d_flux, r.f32(0), n, oo, e->s_up);
            if (err == cudaSuccess) err = up(e->d_fluxerr, r.f32(1), n, oo, e->s_up);
            if (err == cudaSuccess) err = up(e->d_zp, r.f32(2), n, oo, e->s_up);
            if (err == cudaSuccess) err = up(e->d_t0, r.t0(), S, po, e->s_up);
            if (err == cudaSuccess) err = up(e->d_z, r.par32(0), S, po, e->s_up);
            if (err == cudaSuccess) err = up(e->d_x0, r.par32(1), S, po, e->s_up);
            if (err == cudaSuccess) err = up(e->d_x1, r.par32(2), S, po, e->s_up);
            if (err == cudaSuccess) err = up(e->d_c, r.par32(3), S, po, e->s_up);
        } else {
            unsigned char *h = sgu->h;
            auto put = [&](size_t base, size_t at, const void *src, size_t bytes) {
                if (bytes) std::memcpy(h + base + at, src, bytes);
            };
            put(SL.mjd, 8 * ad.so, r.mjd(), 8 * n);
            put(SL.band, 4 * ad.so, r.band(), 4 * n);
            put(SL.flux, 4 * ad.so, r.f32(0), 4 * n);
            put(SL.fluxerr, 4 * ad.so, r.f32(1), 4 * n);
            put(SL.zp, 4 * ad.so, r.f32(2), 4 * n);
            put(SL.t0, 8 * ad.sp, r.t0(), 8 * S);
            put(SL.z, 4 * ad.sp, r.par32(0), 4 * S);
            put(SL.x0, 4 * ad.sp, r.par32(1), 4 * S);
            put(SL.x1, 4 * ad.sp, r.par32(2), 4 * S);
            put(SL.c, 4 * ad.sp, r.par32(3), 4 * S);
        }
    }
    if (err == cudaSuccess && sgu) {
        UpDesc *dsc = (UpDesc *)(sgu->h + SL.desc);
        int q = 0;
        for (const Adm &ad : adm)
            if (!ad.direct)
                dsc[q++] = UpDesc{(int64_t)ad.so, (int64_t)ad.r->oo, ad.r->n_obs, (int64_t)ad.sp, (int64_t)ad.r->po,
                                  ad.r->n_par};
        // one transfer per array (used prefix) and one scatter kernel for the whole pass
        const size_t parts[][2] = {{SL.mjd, 8 * so}, {SL.band, 4 * so}, {SL.flux, 4 * so},
                                   {SL.fluxerr, 4 * so}, {SL.zp, 4 * so}, {SL.t0, 8 * sp},
                                   {SL.z, 4 * sp}, {SL.x0, 4 * sp}, {SL.x1, 4 * sp},
                                   {SL.c, 4 * sp}, {SL.desc, sizeof(UpDesc) * (size_t)nd}};
        for (const auto &pt : parts)
            if (err == cudaSuccess && pt[1])
                err = cudaMemcpyAsync(sgu->d + pt[0], sgu->h + pt[0], pt[1], cudaMemcpyHostToDevice, e->s_up);
        if (err == cudaSuccess) {
            const int64_t rows = (int64_t)std::max(so, sp);
            const int blocks = (int)std::min<int64_t>((rows + 255) / 256, 4 * (int64_t)e->ctx->num_sms);
            k_stage_scatter<<<std::max(blocks, 1), 256, 0, e->s_up>>>(
                sgu->d, SL, nd, (int64_t)so, (int64_t)sp, e->d_mjd, e->d_band, e->d_flux, e->d_fluxerr, e->d_zp,
                e->d_t0, e->d_z, e->d_x0, e->d_x1, e->d_c);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess) err = cudaEventRecord(sgu->ev, e->s_up);
    }
    if (err == cudaSuccess && !adm.empty()) {
        err = cudaEventRecord(e->ev_up, e->s_up);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(e->s_comp, e->ev_up, 0);
    }
    BatchDev b{};
    b.mjd = e->d_mjd; b.band = e->d_band; b.flux = e->d_flux; b.fluxerr = e->d_fluxerr; b.zp = e->d_zp;
    b.t0 = e->d_t0; b.z = e->d_z; b.x0 = e->d_x0; b.x1 = e->d_x1; b.c = e->d_c;
    OutDev o{nullptr, nullptr, e->d_chi2, e->d_grad, e->ctx->err_d};
    for (size_t gi = 0; gi < grps.size() && err == cudaSuccess; ++gi) {
        const Grp &G = grps[gi];
        int n_items = 0;
        for (const Req *rp : G.members) {
            const Req &r = *rp;
            const int cr = std::max(chunk, (r.n_par + kMaxItems - 1) / kMaxItems);
            for (int j0 = 0; j0 < r.n_par; j0 += cr) {
                WorkItem w{};
                w.obs0 = (int64_t)r.oo;
                w.par0 = (int64_t)r.po + j0;
                w.bf0 = 0;
                w.nobs = r.n_obs;
                w.nj = std::min(cr, r.n_par - j0);
                w.jloc0 = j0;
                e->items_h[G.slot][n_items++] = w;
            }
        }
        err = cudaMemcpyAsync(e->items_d[G.slot], e->items_h[G.slot], (size_t)n_items * sizeof(WorkItem),
                              cudaMemcpyHostToDevice, e->s_comp);
        if (err == cudaSuccess)
            err = launch_factorised_items(e->ctx, G.tile, e->items_d[G.slot], n_items, e->counters_d + 4 * G.slot, b,
                                          o, G.mode, e->s_comp);
        if (err == cudaSuccess) err = cudaEventRecord(G.ev, e->s_comp);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(e->s_down, G.ev, 0);
        if (err == cudaSuccess) err = download_results(e, G.members, G.mode == MODE_GRAD);
        if (err == cudaSuccess) err = cudaEventRecord(G.ev, e->s_down);
    }
    lk.lock();

    // 5. commit
    if (sgu && err == cudaSuccess) {
        sgu->busy = true;
        e->stage_cur ^= 1;
    }
    for (const Adm &ad : adm) {
        Req &r = *ad.r;
        r.in.reset();
        if (r.st == St::ADMITTING) r.st = St::ACTIVE;
        if (r.cancel && !r.launched && r.st == St::ACTIVE) {
            // cancelled while being admitted and not in any launch: its upload is
            // queued before anything that could reuse its ranges
            release_req(e, r);
            r.st = St::CANCELLED;
            e->cv_done.notify_all();
        }
    }
    for (size_t gi = 0; gi < grps.size(); ++gi) {
        Launch L;
        L.slot = grps[gi].slot;
        L.reqs = std::move(grps[gi].tickets);
        L.ev = grps[gi].ev;
        e->inflight.push_back(std::move(L));
        e->n_launches++;
    }
    if (err != cudaSuccess) { fail_all(e, cudaGetErrorString(err)); return false; }
    return true;
}

bool has_work(ServeEngine *e) {
    if (!e->inflight.empty() || !e->queue.empty()) return true;
    for (auto &mode : e->pending)
        for (auto &bucket : mode)
            if (!bucket.empty()) return true;
    return false;
}

void run(ServeEngine *e) {
    cudaSetDevice(e->ctx->device);
    std::unique_lock<std::mutex> lk(e->mu);
    while (!e->stop) {
        if (!e->fatal.empty()) {
            e->cv_work.wait(lk, [&] { return e->stop; });
            break;
        }
        if (!has_work(e)) {
            e->idle = true;
            e->cv_work.wait(lk);
            e->idle = false;
            continue;
        }
        tick(e, lk);
        // with work queued or in flight the engine comes back on its own after a
        // short wait; submissions meanwhile only queue (they wake an idle engine)
        if (has_work(e)) e->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
}

}  // namespace

ServeEngine *serve_create(salt_ctx *ctx, size_t mem_limit) {
    // split the budget: half observations, half samples
    const size_t obs_cap = std::max<size_t>(mem_limit / 2 / kObsBytes, 1024);
    const size_t par_cap = std::max<size_t>(mem_limit / 2 / kParBytes, 1024);
    auto *e = new (std::nothrow) ServeEngine(obs_cap, par_cap);
    if (!e) return nullptr;
    e->ctx = ctx;
    bool ok = true;
    auto dm = [&](void **p, size_t bytes) { if (ok) ok = cudaMalloc(p, bytes) == cudaSuccess; };
    dm((void **)&e->d_mjd, 8 * obs_cap);
    dm((void **)&e->d_band, 4 * obs_cap);
    dm((void **)&e->d_flux, 4 * obs_cap);
    dm((void **)&e->d_fluxerr, 4 * obs_cap);
    dm((void **)&e->d_zp, 4 * obs_cap);
    dm((void **)&e->d_t0, 8 * par_cap);
    dm((void **)&e->d_z, 4 * par_cap);
    dm((void **)&e->d_x0, 4 * par_cap);
    dm((void **)&e->d_x1, 4 * par_cap);
    dm((void **)&e->d_c, 4 * par_cap);
    dm((void **)&e->d_chi2, 8 * par_cap);
    dm((void **)&e->d_grad, 20 * par_cap);
    dm((void **)&e->counters_d, 4 * sizeof(int) * kSlots);
    if (ok) ok = cudaHostAlloc(&e->h_chi2, 8 * par_cap, cudaHostAllocDefault) == cudaSuccess;
    if (ok) ok = cudaHostAlloc(&e->h_grad, 20 * par_cap, cudaHostAllocDefault) == cudaSuccess;
    if (ok) ok = cudaStreamCreateWithFlags(&e->s_up, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaStreamCreateWithFlags(&e->s_comp, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaStreamCreateWithFlags(&e->s_down, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaEventCreateWithFlags(&e->ev_up, cudaEventDisableTiming) == cudaSuccess;
    for (int q = 0; ok && q < 2; ++q) {
        dm((void **)&e->stage[q].d, e->SL.total);
        if (ok) ok = cudaHostAlloc(&e->stage[q].h, e->SL.total, cudaHostAllocDefault) == cudaSuccess;
        if (ok) ok = cudaEventCreateWithFlags(&e->stage[q].ev, cudaEventDisableTiming) == cudaSuccess;
    }
    for (int q = 0; ok && q < kSlots; ++q) {
        dm((void **)&e->items_d[q], kMaxItems * sizeof(WorkItem));
        if (ok) ok = cudaHostAlloc(&e->items_h[q], kMaxItems * sizeof(WorkItem), cudaHostAllocDefault) == cudaSuccess;
    }
    if (!ok) {
        serve_destroy(e);
        return nullptr;
    }
    e->th = std::thread(run, e);
    return e;
}

void serve_destroy(ServeEngine *e) {
    if (!e) return;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stop = true;
    }
    e->cv_work.notify_all();
    e->cv_done.notify_all();
    if (e->th.joinable()) e->th.join();
    for (cudaStream_t s : {e->s_up, e->s_comp, e->s_down})
        if (s) cudaStreamSynchronize(s);
    for (auto &L : e->inflight)
        if (L.ev) cudaEventDestroy(L.ev);
    for (cudaEvent_t ev : e->ev_pool) cudaEventDestroy(ev);
    for (int q = 0; q < kSlots; ++q) {
        if (e->items_d[q]) cudaFree(e->items_d[q]);
        if (e->items_h[q]) cudaFreeHost(e->items_h[q]);
    }
    for (auto &sg : e->stage) {
        if (sg.d) cudaFree(sg.d);
        if (sg.h) cudaFreeHost(sg.h);
        if (sg.ev) cudaEventDestroy(sg.ev);
    }
    void *dptrs[] = {e->d_mjd, e->d_band, e->d_flux, e->d_fluxerr, e->d_zp, e->d_t0, e->d_z, e->d_x0,
                     e->d_x1, e->d_c, e->d_chi2, e->d_grad, e->counters_d};
    for (void *p : dptrs)
        if (p) cudaFree(p);
    if (e->h_chi2) cudaFreeHost(e->h_chi2);
    if (e->h_grad) cudaFreeHost(e->h_grad);
    if (e->ev_up) cudaEventDestroy(e->ev_up);
    for (cudaStream_t s : {e->s_up, e->s_comp, e->s_down})
        if (s) cudaStreamDestroy(s);
    delete e;
}

int serve_submit(ServeEngine *e, const salt_request *q, uint64_t *ticket) {
    if (!q || !ticket || q->n_obs < 0 || q->n_par < 1) return SALT_ERR_INVALID;
    const int n = q->n_obs, S = q->n_par;
    if (n > 0 && (!q->mjd || !q->band || !q->flux || !q->fluxerr || !q->zp)) return SALT_ERR_INVALID;
    if (!q->t0 || !q->z || !q->x0 || !q->x1 || !q->c) return SALT_ERR_INVALID;
    const int nb = e->ctx->mp.bands.n_bands;
    for (int i = 0; i < n; ++i)
        if (q->band[i] < 0 || q->band[i] >= nb || !(q->fluxerr[i] > 0.f) || !std::isfinite(q->fluxerr[i]) ||
            !std::isfinite(q->mjd[i]) || !std::isfinite(q->flux[i]) || !std::isfinite(q->zp[i]))
            return SALT_ERR_INVALID;
    for (int j = 0; j < S; ++j)
        if (!std::isfinite(q->t0[j]) || !std::isfinite(q->z[j]) || !(q->z[j] > -1.f) || !std::isfinite(q->x0[j]) ||
            !std::isfinite(q->x1[j]) || !std::isfinite(q->c[j]))
            return SALT_ERR_INVALID;
    if ((size_t)n > e->obs_a.size() || (size_t)S > e->par_a.size()) {
        std::lock_guard<std::mutex> lk(e->mu);
        e->n_rejected++;
        return SALT_ERR_OOM;
    }
    auto r = std::make_unique<Req>();
    r->n_obs = n;
    r->n_par = S;
    r->grad = q->want_grad != 0;
    r->tile = tile_for(S);
    r->in.reset(new (std::nothrow) unsigned char[Req::in_bytes(n, S)]);
    if (!r->in) return SALT_ERR_OOM;
    {
        unsigned char *p = r->in.get();
        auto put = [&p](const void *src, size_t bytes) {
            if (bytes) std::memcpy(p, src, bytes);
            p += bytes;
        };
        put(q->mjd, 8 * (size_t)n);
        put(q->t0, 8 * (size_t)S);
        put(q->band, 4 * (size_t)n);
        put(q->flux, 4 * (size_t)n);
        put(q->fluxerr, 4 * (size_t)n);
        put(q->zp, 4 * (size_t)n);
        put(q->z, 4 * (size_t)S);
        put(q->x0, 4 * (size_t)S);
        put(q->x1, 4 * (size_t)S);
        put(q->c, 4 * (size_t)S);
    }
    r->t_submit = now_ms();
    bool wake = false;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        if (!e->fatal.empty()) return SALT_ERR_CUDA;
        if (e->stop) return SALT_ERR_CANCELLED;
        r->ticket = e->next_ticket++;
        *ticket = r->ticket;
        e->queue.push_back(r->ticket);
        e->reqs.emplace(r->ticket, std::move(r));
        e->n_submitted++;
        wake = e->idle;
    }
    if (wake) e->cv_work.notify_one();
    return SALT_OK;
}

int serve_poll(ServeEngine *e, uint64_t ticket, int32_t wait_ms, double *chi2, float *grad) {
    std::unique_lock<std::mutex> lk(e->mu);
    auto it = e->reqs.find(ticket);
    if (it == e->reqs.end()) return SALT_ERR_NOT_FOUND;
    Req *rp = it->second.get();
    auto ready = [rp] { return rp->st == St::DONE || rp->st == St::CANCELLED || rp->st == St::FAILED; };
    if (!ready()) {
        if (wait_ms == 0) return SALT_PENDING;
        if (wait_ms < 0)
            e->cv_done.wait(lk, ready);
        else if (!e->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready))
            return SALT_ERR_TIMEOUT;
    }
    int rc = SALT_OK;
    if (rp->st == St::CANCELLED) rc = SALT_ERR_CANCELLED;
    else if (rp->st == St::FAILED) rc = SALT_ERR_CUDA;
    else {
        if (chi2) std::memcpy(chi2, rp->chi2.data(), 8 * (size_t)rp->n_par);
        if (grad && rp->grad) std::memcpy(grad, rp->gout.data(), 20 * (size_t)rp->n_par);
    }
    e->reqs.erase(ticket);
    return rc;
}

int serve_cancel(ServeEngine *e, uint64_t ticket) {
    std::lock_guard<std::mutex> lk(e->mu);
    auto it = e->reqs.find(ticket);
    if (it == e->reqs.end()) return SALT_ERR_NOT_FOUND;
    Req &r = *it->second;
    if (r.st == St::DONE || r.st == St::FAILED || r.st == St::CANCELLED) return SALT_OK;
    if (!r.cancel) e->n_cancelled++;
    r.cancel = true;
    if (r.st == St::QUEUED) {
        r.st = St::CANCELLED;
        e->cv_done.notify_all();
    } else if (r.st == St::ACTIVE && !r.launched) {
        // its upload may still be in flight: drain the upload stream first
        cudaStreamSynchronize(e->s_up);
        release_req(e, r);
        r.st = St::CANCELLED;
        e->cv_done.notify_all();
    }
    // launched: released when its launch retires (tick)
    return SALT_OK;
}

int serve_stats(ServeEngine *e, salt_serve_stats *out) {
    std::lock_guard<std::mutex> lk(e->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = e->n_submitted;
    out->completed = e->n_completed;
    out->cancelled = e->n_cancelled;
    out->rejected = e->n_rejected;
    out->launches = e->n_launches;
    out->queued = e->queue.size();
    uint64_t act = 0;
    for (auto &kv : e->reqs)
        if (kv.second->st == St::ACTIVE || kv.second->st == St::ADMITTING) act++;
    out->active = act;
    out->mem_in_use = e->obs_a.used() * kObsBytes + e->par_a.used() * kParBytes;
    out->mem_limit = e->obs_a.size() * kObsBytes + e->par_a.size() * kParBytes;
    if (!e->lat_ms.empty()) {
        std::vector<double> v = e->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const double pos = q * (double)(v.size() - 1);
            const size_t lo = (size_t)pos;
            const size_t hi = std::min(lo + 1, v.size() - 1);
            return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    return SALT_OK;
}

}  // namespace salt
