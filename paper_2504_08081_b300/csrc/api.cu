// C ABI entry points: model upload, planning, batch calls, options, errors.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>

#include "salt_internal.cuh"

using namespace salt;

namespace {

// CGS constants for the bandpass weights: Planck (exact SI), c in A/s (exact),
// the AB reference flux density 3631 Jy.
constexpr double kPlanck = 6.62607015e-27;
constexpr double kLightAA = 2.99792458e18;
constexpr double kAB = 3631e-23;
// SALT2 colour-law reference wavelengths.
constexpr double kLamB = 4302.57, kLamV = 5428.55;

int set_err(salt_ctx *ctx, int code, const std::string &msg) {
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->last_error = msg;
    }
    return code;
}

int cuda_err(salt_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();  // the status code reports it: do not leave it for the caller's runtime
    return set_err(ctx, e == cudaErrorMemoryAllocation ? SALT_ERR_OOM : SALT_ERR_CUDA, m);
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, what); \
    } while (0)

double cl_poly(const double a[4], double x) {
    const double lin = 1.0 - a[0] - a[1] - a[2] - a[3];
    double xp = x, P = lin * x;
    for (int q = 0; q < 4; ++q) { xp *= x; P += a[q] * xp; }
    return P;
}

double cl_dpoly(const double a[4], double x) {
    const double lin = 1.0 - a[0] - a[1] - a[2] - a[3];
    double xp = 1.0, dP = lin;
    for (int q = 0; q < 4; ++q) { xp *= x; dP += (q + 2) * a[q] * xp; }
    return dP;
}

bool finite_all(const float *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Check one band and append its samples and trapezoid weights
// lambda T Delta / (h c Z_b) (FP64, rounded to float32) to lam / w.
bool band_tables(const salt_band_desc &bd, std::vector<float> &lam, std::vector<float> &w) {
    if (bd.n < 2 || !bd.wave || !bd.trans) return false;
    for (int k = 0; k < bd.n; ++k) {
        if (!std::isfinite(bd.wave[k]) || !std::isfinite(bd.trans[k]) || !(bd.wave[k] > 0)) return false;
        if (k > 0 && !(bd.wave[k] > bd.wave[k - 1])) return false;
    }
    const double hc = kPlanck * kLightAA;
    const int K = bd.n;
    std::vector<double> wk(K);
    double Z = 0.0;
    for (int k = 0; k < K; ++k) {
        const double lo = (k > 0) ? bd.wave[k - 1] : bd.wave[k];
        const double hi = (k + 1 < K) ? bd.wave[k + 1] : bd.wave[k];
        const double delta = 0.5 * (hi - lo);
        wk[k] = bd.wave[k] * bd.trans[k] * delta / hc;
        Z += wk[k] * kAB * kLightAA / (bd.wave[k] * bd.wave[k]);
    }
    if (!(Z > 0) || !std::isfinite(Z)) return false;
    for (int k = 0; k < K; ++k) {
        lam.push_back((float)bd.wave[k]);
        w.push_back((float)(wk[k] / Z));
    }
    // every band starts on an even index (8-byte aligned), so kernels can read
    // two consecutive samples with one load; the pad sample has zero weight
    if (lam.size() & 1) {
        lam.push_back(lam.back());
        w.push_back(0.f);
    }
    return true;
}

}  // namespace

// ------------------------------------------------------------------ model

extern "C" int salt_init_model(const salt_model_desc *md, const salt_band_desc *bands, int32_t n_bands,
                               int32_t device, size_t serve_mem_bytes, salt_ctx **out) {
    if (!out) return SALT_ERR_INVALID;
    *out = nullptr;
    salt_ctx *ctx = nullptr;
    if (!md || (!bands && n_bands > 0) || n_bands < 0 || n_bands > SALT_MAX_BANDS) return SALT_ERR_INVALID;
    auto axis_ok = [](const double *nodes, int n, double x0, double dx) {
        if (!nodes) return dx > 0 && std::isfinite(x0) && std::isfinite(dx);
        for (int i = 0; i < n; ++i) {
            if (!std::isfinite(nodes[i])) return false;
            if (i > 0 && !(nodes[i] > nodes[i - 1])) return false;
        }
        return true;
    };
    if (md->n_phase < 4 || md->n_wave < 4 || md->n_phase > 256 || !md->m0 || !md->m1 || md->n_cl != 4 ||
        !md->cl || !(md->cl_lo < md->cl_hi) || !axis_ok(md->phase_nodes, md->n_phase, md->phase0, md->dphase) ||
        !axis_ok(md->wave_nodes, md->n_wave, md->wave0, md->dwave))
        return SALT_ERR_INVALID;
    const size_t ng = (size_t)md->n_phase * md->n_wave;
    if (!finite_all(md->m0, ng) || !finite_all(md->m1, ng)) return SALT_ERR_INVALID;
    for (int q = 0; q < 4; ++q)
        if (!std::isfinite(md->cl[q])) return SALT_ERR_INVALID;
    ctx = new (std::nothrow) salt_ctx();
    if (!ctx) return SALT_ERR_OOM;
    ctx->device = device;
    ctx->host_cl.assign(md->cl, md->cl + 4);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete ctx; return SALT_ERR_CUDA; }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    ctx->num_sms = sms > 0 ? sms : 1;

    ModelParams &mp = ctx->mp;
    mp.n_phase = md->n_phase;
    mp.n_wave = md->n_wave;
    // axis ends (and, on uniform axes, the inverse step); non-uniform axes keep
    // their nodes and inverse interval widths on the device
    const double p0 = md->phase_nodes ? md->phase_nodes[0] : md->phase0;
    const double p1 = md->phase_nodes ? md->phase_nodes[md->n_phase - 1] : md->phase0 + (md->n_phase - 1) * md->dphase;
    const double w0 = md->wave_nodes ? md->wave_nodes[0] : md->wave0;
    const double w1 = md->wave_nodes ? md->wave_nodes[md->n_wave - 1] : md->wave0 + (md->n_wave - 1) * md->dwave;
    mp.phase0 = (float)p0;
    mp.inv_dphase = (float)(md->phase_nodes ? (md->n_phase - 1) / (p1 - p0) : 1.0 / md->dphase);
    mp.phase_max = (float)p1;
    mp.dphase = (float)(md->phase_nodes ? 1.0 : md->dphase);
    mp.phase0_d = p0;
    mp.inv_dphase_d = md->phase_nodes ? (md->n_phase - 1) / (p1 - p0) : 1.0 / md->dphase;
    mp.wave0 = (float)w0;
    mp.inv_dwave = (float)(md->wave_nodes ? (md->n_wave - 1) / (w1 - w0) : 1.0 / md->dwave);
    mp.wave_max = (float)w1;
    mp.dwave = (float)(md->wave_nodes ? (w1 - w0) / (md->n_wave - 1) : md->dwave);
    const double a[4] = {md->cl[0], md->cl[1], md->cl[2], md->cl[3]};
    mp.cl_p[0] = (float)(1.0 - a[0] - a[1] - a[2] - a[3]);
    for (int q = 0; q < 4; ++q) mp.cl_p[q + 1] = (float)a[q];
    const double span = kLamV - kLamB;
    mp.cl_lamB = (float)kLamB;
    mp.cl_inv_span = (float)(1.0 / span);
    mp.cl_lo = (float)md->cl_lo;
    mp.cl_hi = (float)md->cl_hi;
    const double xlo = (md->cl_lo - kLamB) / span, xhi = (md->cl_hi - kLamB) / span;
    mp.cl_xlo = (float)xlo;
    mp.cl_Plo = (float)cl_poly(a, xlo);
    mp.cl_dPlo = (float)cl_dpoly(a, xlo);
    mp.cl_xhi = (float)xhi;
    mp.cl_Phi = (float)cl_poly(a, xhi);
    mp.cl_dPhi = (float)cl_dpoly(a, xhi);

    // bandpass weights: trapezoid Delta_k, lambda T Delta / (h c), divided by
    // the AB photon integral Z_b (FP64 on the host, then float32)
    std::vector<float> lam_h, w_h;
    mp.bands.n_bands = n_bands;
    for (int b = 0; b < n_bands; ++b) {
        const salt_band_desc &bd = bands[b];
        const int off = (int)lam_h.size();
        if (!band_tables(bd, lam_h, w_h)) { delete ctx; return SALT_ERR_INVALID; }
        mp.bands.off[b] = off;
        mp.bands.n[b] = bd.n;
        mp.bands.lam_lo[b] = (float)bd.wave[0];
        mp.bands.lam_hi[b] = (float)bd.wave[bd.n - 1];
    }
    mp.bands.k_total = (int)lam_h.size();
    // interleaved (M0, M1) rows with an even pitch so every row starts on 16 bytes
    const int nwp = md->n_wave + (md->n_wave & 1);
    mp.nw_pitch = nwp;
    const size_t ngp = (size_t)md->n_phase * nwp;
    std::vector<float2> g(ngp, make_float2(0.f, 0.f));
    for (int r = 0; r < md->n_phase; ++r)
        for (int j = 0; j < md->n_wave; ++j) {
            const size_t q = (size_t)r * md->n_wave + j;
            g[(size_t)r * nwp + j] = make_float2(md->m0[q], md->m1[q]);
        }

    auto fail = [&](cudaError_t err, const char *what) {
        int code = cuda_err(nullptr, err, what);
        salt_destroy(ctx);
        return code;
    };
    if ((e = cudaMalloc(&ctx->g01_d, ngp * sizeof(float2))) != cudaSuccess) return fail(e, "cudaMalloc grid");
    if ((e = cudaMemcpy(ctx->g01_d, g.data(), ngp * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "upload grid");
    const size_t nk = std::max<size_t>(lam_h.size(), 1);
    if ((e = cudaMalloc(&ctx->band_lam_d, nk * sizeof(float))) != cudaSuccess) return fail(e, "cudaMalloc bands");
    if ((e = cudaMalloc(&ctx->band_w_d, nk * sizeof(float))) != cudaSuccess) return fail(e, "cudaMalloc bands");
    if (!lam_h.empty()) {
        if ((e = cudaMemcpy(ctx->band_lam_d, lam_h.data(), lam_h.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e, "upload bands");
        if ((e = cudaMemcpy(ctx->band_w_d, w_h.data(), w_h.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e, "upload bands");
    }
    if (md->phase_nodes || md->wave_nodes) {
        // [phase nodes | phase inverse widths | wave nodes | wave inverse widths | phase node
        // remainders], each n long
        const int np = md->n_phase, nw = md->n_wave;
        std::vector<float> nodes(3 * (size_t)np + 2 * (size_t)nw, 0.f);
        auto fill = [&](const double *x, int n, float *node, float *inv) {
            for (int i = 0; i < n; ++i) node[i] = (float)x[i];
            for (int i = 0; i + 1 < n; ++i) inv[i] = (float)(1.0 / (x[i + 1] - x[i]));
        };
        if (md->phase_nodes) fill(md->phase_nodes, np, nodes.data(), nodes.data() + np);
        if (md->wave_nodes) fill(md->wave_nodes, nw, nodes.data() + 2 * np, nodes.data() + 2 * np + nw);
        if (md->phase_nodes) {
            float *rem = nodes.data() + 2 * np + 2 * nw;
            for (int i = 0; i < np; ++i) rem[i] = (float)(md->phase_nodes[i] - (double)nodes[i]);
        }
        if ((e = cudaMalloc(&ctx->nodes_d, nodes.size() * sizeof(float))) != cudaSuccess)
            return fail(e, "cudaMalloc nodes");
        if ((e = cudaMemcpy(ctx->nodes_d, nodes.data(), nodes.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return fail(e, "upload nodes");
        if (md->phase_nodes) {
            mp.pnode = ctx->nodes_d; mp.pinv = ctx->nodes_d + np; mp.pnode_lo = ctx->nodes_d + 2 * np + 2 * nw;
        }
        if (md->wave_nodes) { mp.wnode = ctx->nodes_d + 2 * np; mp.winv = ctx->nodes_d + 2 * np + nw; }
    }
    if ((e = cudaMalloc(&ctx->err_d, 2 * sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc err");
    if ((e = cudaMemset(ctx->err_d, 0, 2 * sizeof(int))) != cudaSuccess) return fail(e, "memset err");
    mp.g01 = ctx->g01_d;
    mp.band_lam = ctx->band_lam_d;
    mp.band_w = ctx->band_w_d;
    ctx->host_lam = std::move(lam_h);
    ctx->host_w = std::move(w_h);
    ctx->serve_mem = serve_mem_bytes;
    if (serve_mem_bytes > 0) {
        ctx->serve = serve_create(ctx, serve_mem_bytes);
        if (!ctx->serve) { salt_destroy(ctx); return SALT_ERR_OOM; }
    }
    *out = ctx;
    return SALT_OK;
}

extern "C" void salt_destroy(salt_ctx *ctx) {
    if (!ctx) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    if (ctx->serve) {
        serve_destroy(ctx->serve);
        ctx->serve = nullptr;
    }
    if (ctx->g01_d) cudaFree(ctx->g01_d);
    if (ctx->band_lam_d) cudaFree(ctx->band_lam_d);
    if (ctx->band_w_d) cudaFree(ctx->band_w_d);
    if (ctx->err_d) cudaFree(ctx->err_d);
    if (ctx->nodes_d) cudaFree(ctx->nodes_d);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    delete ctx;
    cudaSetDevice(prev);
    (void)cudaGetLastError();
}

extern "C" int salt_register_band(salt_ctx *ctx, const salt_band_desc *band, int32_t *band_id) {
    if (!ctx || !band || !band_id) return SALT_ERR_INVALID;
    if (ctx->mp.bands.n_bands >= SALT_MAX_BANDS)
        return set_err(ctx, SALT_ERR_INVALID, "band registry full (SALT_MAX_BANDS)");
    std::vector<float> lam = ctx->host_lam, w = ctx->host_w;
    if (!band_tables(*band, lam, w))
        return set_err(ctx, SALT_ERR_INVALID, "band needs >= 2 finite samples, ascending positive wavelengths "
                                              "and a positive AB integral");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    float *lam_d = nullptr, *w_d = nullptr;
    cudaError_t e = cudaMalloc(&lam_d, lam.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&w_d, w.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(lam_d, lam.data(), lam.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w_d, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (lam_d) cudaFree(lam_d);
        if (w_d) cudaFree(w_d);
        return cuda_err(ctx, e, "register band");
    }
    // cudaFree waits for work in flight that may still read the old tables
    cudaFree(ctx->band_lam_d);
    cudaFree(ctx->band_w_d);
    ctx->band_lam_d = lam_d;
    ctx->band_w_d = w_d;
    BandTable &bt = ctx->mp.bands;
    const int b = bt.n_bands;
    bt.off[b] = bt.k_total;  // (even: every band is padded to an even length)
    bt.n[b] = band->n;
    bt.lam_lo[b] = (float)band->wave[0];
    bt.lam_hi[b] = (float)band->wave[band->n - 1];
    bt.k_total = (int)lam.size();
    bt.n_bands = b + 1;
    ctx->mp.band_lam = lam_d;
    ctx->mp.band_w = w_d;
    ctx->host_lam = std::move(lam);
    ctx->host_w = std::move(w);
    ++ctx->band_gen;  // plans drop their work lists, scratch and graphs on next use
    *band_id = b;
    return SALT_OK;
}

// ------------------------------------------------------------------ planning

namespace salt {

static bool offsets_ok(int64_t n_sn, const int64_t *off) {
    if (!off || off[0] != 0) return false;
    for (int64_t s = 0; s < n_sn; ++s)
        if (off[s + 1] < off[s]) return false;
    return true;
}

int plan_build(salt_ctx *ctx, int64_t n_sn, const int64_t *obs_off, const int64_t *par_off, int /*tile*/,
               salt_plan *p, cudaStream_t st, bool async_alloc) {
    if (n_sn < 0 || !offsets_ok(n_sn, obs_off) || !offsets_ok(n_sn, par_off))
        return set_err(ctx, SALT_ERR_INVALID, "offsets must start at 0 and be nondecreasing");
    for (int64_t s = 0; s < n_sn; ++s) {
        if (par_off[s + 1] - par_off[s] > INT32_MAX / 2)
            return set_err(ctx, SALT_ERR_INVALID, "too many samples for one supernova");
        if (obs_off[s + 1] - obs_off[s] > INT32_MAX / 2)
            return set_err(ctx, SALT_ERR_INVALID, "too many observations for one supernova");
    }
    p->ctx = ctx;
    p->device = ctx->device;
    p->band_gen = ctx->band_gen;
    p->n_sn = n_sn;
    p->n_obs = obs_off[n_sn];
    p->n_par = par_off[n_sn];
    p->obs_off_h.assign(obs_off, obs_off + n_sn + 1);
    p->par_off_h.assign(par_off, par_off + n_sn + 1);
    p->bf_off_h.assign(n_sn + 1, 0);
    for (int64_t s = 0; s < n_sn; ++s)
        p->bf_off_h[s + 1] = p->bf_off_h[s] + (obs_off[s + 1] - obs_off[s]) * (par_off[s + 1] - par_off[s]);
    p->n_bandflux = p->bf_off_h[n_sn];
    auto alloc = [&](void **ptr, size_t bytes) -> cudaError_t {
        bytes = std::max<size_t>(bytes, 16);
        return async_alloc ? cudaMallocAsync(ptr, bytes, st) : cudaMalloc(ptr, bytes);
    };
    CK(alloc((void **)&p->obs_off_d, (n_sn + 1) * 8), "alloc offsets");
    CK(alloc((void **)&p->par_off_d, (n_sn + 1) * 8), "alloc offsets");
    CK(alloc((void **)&p->bf_off_d, (n_sn + 1) * 8), "alloc offsets");
    CK(alloc((void **)&p->counter_d, 16), "alloc counter");
    CK(cudaMemcpyAsync(p->obs_off_d, obs_off, (n_sn + 1) * 8, cudaMemcpyHostToDevice, st), "upload offsets");
    CK(cudaMemcpyAsync(p->par_off_d, par_off, (n_sn + 1) * 8, cudaMemcpyHostToDevice, st), "upload offsets");
    CK(cudaMemcpyAsync(p->bf_off_d, p->bf_off_h.data(), (n_sn + 1) * 8, cudaMemcpyHostToDevice, st),
       "upload offsets");
    if (async_alloc) CK(cudaStreamSynchronize(st), "plan upload");
    return SALT_OK;
}

// Work list for one launch configuration: (supernova, sample-range) items,
// longest first (cost ~ tiles x (observations + per-band setup)).
static int build_items(salt_ctx *ctx, salt_plan *p, int key, cudaStream_t st) {
    if (p->lists.count(key)) return SALT_OK;
    const int family = cfg_family(key), tile = cfg_tile(key);
    const int64_t n_sn = p->n_sn;
    const int64_t *po = p->par_off_h.data(), *oo = p->obs_off_h.data();
    int span;
    if (family == FAM_WARP) {
        span = bandwarp_item_samples();
    } else if (family == FAM_UNIT) {
        span = tile;
    } else {
        int64_t total_tiles = 0;
        for (int64_t s = 0; s < n_sn; ++s) total_tiles += (po[s + 1] - po[s] + tile - 1) / tile;
        const int64_t target = (int64_t)ctx->num_sms * 16;
        const int tpi = (int)std::min<int64_t>(8, std::max<int64_t>(1, total_tiles / std::max<int64_t>(target, 1)));
        span = tile * tpi;
    }
    struct Cost { double c; WorkItem w; };
    std::vector<Cost> items;
    for (int64_t s = 0; s < n_sn; ++s) {
        const int64_t S = po[s + 1] - po[s];
        const int64_t n = oo[s + 1] - oo[s];
        for (int64_t j0 = 0; j0 < S; j0 += span) {
            const int nj = (int)std::min<int64_t>(span, S - j0);
            const double cost = (double)((nj + tile - 1) / tile) * (64.0 + (double)n) * tile;
            items.push_back({cost, WorkItem{oo[s], po[s] + j0, p->bf_off_h[s], (int32_t)n, nj, (int32_t)j0, 0}});
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const Cost &x, const Cost &y) { return x.c > y.c; });
    std::vector<WorkItem> wl(items.size());
    for (size_t q = 0; q < items.size(); ++q) wl[q] = items[q].w;
    salt_plan::ItemList L;
    L.n = (int)wl.size();
    const size_t bytes = std::max<size_t>(wl.size() * sizeof(WorkItem), 16);
    CK(p->temporary ? cudaMallocAsync((void **)&L.d, bytes, st) : cudaMalloc((void **)&L.d, bytes),
       "alloc work list");
    if (family == FAM_UNIT) {
        const size_t sb = unit_scratch_bytes(L.n, tile, ctx->mp.bands.n_bands);
        CK(p->temporary ? cudaMallocAsync(&L.scratch, sb, st) : cudaMalloc(&L.scratch, sb), "alloc scratch");
        CK(cudaMemsetAsync(L.scratch, 0, sb, st), "clear scratch");
    }
    p->lists[key] = L;
    if (!wl.empty()) {
        CK(cudaMemcpyAsync(L.d, wl.data(), wl.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, st),
           "upload work list");
        // pageable source: staged before return, but keep the host copy alive until then
        CK(cudaStreamSynchronize(st), "upload work list");
    }
    return SALT_OK;
}

void plan_free(salt_plan *p, cudaStream_t st) {
    for (auto &kv : p->graphs)
        for (auto &G : kv.second.e)
            if (G.exec) cudaGraphExecDestroy(G.exec);
    p->graphs.clear();
    std::vector<void *> ptrs = {p->obs_off_d, p->par_off_d, p->bf_off_d, p->counter_d};
    for (auto &kv : p->lists) {
        ptrs.push_back(kv.second.d);
        ptrs.push_back(kv.second.scratch);
    }
    for (void *q : ptrs)
        if (q) {
            if (p->temporary) cudaFreeAsync(q, st); else cudaFree(q);
        }
    p->lists.clear();
    p->obs_off_d = p->par_off_d = p->bf_off_d = nullptr;
    p->counter_d = nullptr;
}

static cudaError_t launch_key(salt_ctx *ctx, salt_plan *p, int key, const BatchDev &b, const OutDev &o, int mode,
                              cudaStream_t st) {
    const salt_plan::ItemList &L = p->lists[key];
    if (cfg_family(key) == FAM_WARP)
        return launch_bandwarp_items(ctx, cfg_tile(key), L.d, L.n, p->counter_d, b, o, mode, st);
    if (cfg_family(key) == FAM_UNIT)
        return launch_unit_items(ctx, cfg_tile(key), L.d, L.n, p->counter_d, L.scratch, b, o, mode, st);
    return launch_factorised_items(ctx, cfg_tile(key), L.d, L.n, p->counter_d, b, o, mode, st);
}

// Heuristic configuration (used for one-off plans and while capturing).
static bool unit_ok(const salt_ctx *ctx, const salt_plan *p, int ts) {
    if (ctx->mp.n_phase > unit_max_phase() || ctx->mp.bands.n_bands < 1) return false;
    const int64_t items = p->n_par / ts + p->n_sn;
    return unit_scratch_bytes((int)std::min<int64_t>(items, INT32_MAX), ts, ctx->mp.bands.n_bands) <= ((size_t)256 << 20);
}

static int default_config(const salt_ctx *ctx, const salt_plan *p) {
    const double mean = p->n_sn > 0 ? (double)p->n_par / (double)p->n_sn : 1.0;
    if (mean < 4 && unit_ok(ctx, p, mean >= 2 ? 2 : 1)) return cfg_key(FAM_UNIT, mean >= 2 ? 2 : 1);
    const bool warp_ok = ctx->mp.n_phase <= bandwarp_max_phase();
    if (warp_ok && mean < 4) return cfg_key(FAM_WARP, mean >= 2 ? 2 : 1);
    if (mean >= 8) return cfg_key(FAM_CTA, 8);
    if (mean >= 4) return cfg_key(FAM_CTA, 4);
    return cfg_key(FAM_CTA, mean >= 2 ? 2 : 1);
}

// Autotuner: process-wide cache of tuned configurations keyed by the batch
// layout signature, optionally persisted as JSON lines (SALT_TUNE_CACHE).
struct TuneCache {
    std::mutex mu;
    std::map<std::string, int> best;
    bool loaded = false;
    void load() {
        if (loaded) return;
        loaded = true;
        const char *path = getenv("SALT_TUNE_CACHE");
        if (!path) return;
        FILE *f = fopen(path, "r");
        if (!f) return;
        char line[512];
        while (fgets(line, sizeof line, f)) {
            char sig[400];
            int key;
            if (sscanf(line, "{\"sig\": \"%399[^\"]\", \"key\": %d}", sig, &key) == 2) best[sig] = key;
        }
        fclose(f);
    }
    void store(const std::string &sig, int key) {
        best[sig] = key;
        const char *path = getenv("SALT_TUNE_CACHE");
        if (!path) return;
        FILE *f = fopen(path, "a");
        if (!f) return;
        fprintf(f, "{\"sig\": \"%s\", \"key\": %d}\n", sig.c_str(), key);
        fclose(f);
    }
};
static TuneCache g_tune;

static std::string plan_signature(const salt_ctx *ctx, const salt_plan *p, int mode) {
    char buf[256];
    snprintf(buf, sizeof buf, "sm%d np%d nw%d nb%d m%d sn%lld obs%lld par%lld", ctx->num_sms, ctx->mp.n_phase,
             ctx->mp.n_wave, ctx->mp.bands.n_bands, mode, (long long)p->n_sn, (long long)p->n_obs,
             (long long)p->n_par);
    return buf;
}

static int tune(salt_ctx *ctx, salt_plan *p, const BatchDev &b, const OutDev &o, int mode, cudaStream_t st,
                int *best_key) {
    std::vector<int> cands;
    const double mean = p->n_sn > 0 ? (double)p->n_par / (double)p->n_sn : 1.0;
    for (int t : {1, 2, 4, 8})  // 16-sample tiles measured slower than 8 on every workload
        if (t == 1 || mean >= 0.75 * t) cands.push_back(cfg_key(FAM_CTA, t));
    if (ctx->mp.n_phase <= bandwarp_max_phase()) {
        cands.push_back(cfg_key(FAM_WARP, 1));
        if (mean >= 1.5) cands.push_back(cfg_key(FAM_WARP, 2));
    }
    if (unit_ok(ctx, p, 1)) cands.push_back(cfg_key(FAM_UNIT, 1));
    if (mean >= 1.5 && unit_ok(ctx, p, 2)) cands.push_back(cfg_key(FAM_UNIT, 2));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "tune");
    CK(cudaEventCreate(&e1), "tune");
    float best_ms = 1e30f;
    int best = -1;
    int rc = SALT_OK;
    for (int key : cands) {
        if ((rc = build_items(ctx, p, key, st)) != SALT_OK) break;
        cudaError_t e = launch_key(ctx, p, key, b, o, mode, st);  // warm
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = launch_key(ctx, p, key, b, o, mode, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess) ms = std::min(ms, t);
        }
        if (e != cudaSuccess) { rc = cuda_err(ctx, e, "autotune"); break; }
        if (ms < best_ms) { best_ms = ms; best = key; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SALT_OK) return rc;
    *best_key = best;
    return SALT_OK;
}

// Graph replay for repeated plan calls. A call whose batch and output pointers
// equal those of an earlier call (same mode and configuration; up to
// kGraphSlots pointer sets are remembered) is captured once on the context's
// private stream (the launch's counter reset and kernel become a two-node
// graph) and replayed on the caller's stream from then on; a call with new
// pointers launches directly and takes the least recently used slot. Returns false when
// the caller should launch directly (never while the caller's stream is
// capturing: the caller's own graph then records the direct launch).
static bool replay_graph(salt_ctx *ctx, salt_plan *p, int key, const BatchDev &b, const OutDev &o, int mode,
                         cudaStream_t st, cudaError_t *err) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        (void)cudaGetLastError();
        return false;
    }
    salt_plan::GraphSet &S = p->graphs[mode * 256 + key];
    if (S.failed) return false;
    salt_plan::GraphEntry *G = nullptr;
    for (auto &x : S.e)
        if (x.seen && std::memcmp(&x.b, &b, sizeof b) == 0 && std::memcmp(&x.o, &o, sizeof o) == 0) {
            G = &x;
            break;
        }
    if (!G) {  // a new pointer set: record it in a free slot, else the least recently used one
        salt_plan::GraphEntry *v = &S.e[0];
        for (auto &x : S.e) {
            if (!x.seen) {
                v = &x;
                break;
            }
            if (x.used < v->used) v = &x;
        }
        if (v->exec) cudaGraphExecDestroy(v->exec);
        v->exec = nullptr;
        v->b = b;
        v->o = o;
        v->seen = true;
        v->used = ++S.tick;
        return false;
    }
    G->used = ++S.tick;
    if (!G->exec) {
        if (!ctx->capture_stream &&
            cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            S.failed = true;
            return false;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t el = launch_key(ctx, p, key, b, o, mode, ctx->capture_stream);
            e = cudaStreamEndCapture(ctx->capture_stream, &g);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            G->exec = nullptr;
            S.failed = true;
            return false;
        }
    }
    *err = cudaGraphLaunch(G->exec, st);
    return true;
}

// Drop a plan's work lists (and their scratch), captured graphs and tuned
// choices; the offsets stay. Used when the context's bands changed.
static void plan_reset_work(salt_plan *p) {
    for (auto &kv : p->graphs)
        for (auto &G : kv.second.e)
            if (G.exec) cudaGraphExecDestroy(G.exec);
    p->graphs.clear();
    for (auto &kv : p->lists) {
        if (kv.second.d) cudaFree(kv.second.d);
        if (kv.second.scratch) cudaFree(kv.second.scratch);
    }
    p->lists.clear();
    for (int &c : p->choice) c = -1;
}

int run_batch(salt_ctx *ctx, const BatchDev &b, const salt_plan *cplan, const OutDev &o, int mode,
              cudaStream_t st) {
    salt_plan *p = const_cast<salt_plan *>(cplan);  // tuning state and work lists are a cache
    if (p->band_gen != ctx->band_gen) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (cs != cudaStreamCaptureStatusNone)
            return set_err(ctx, SALT_ERR_INVALID, "bands changed: run the plan once outside stream capture");
        if (!p->temporary) plan_reset_work(p);
        p->band_gen = ctx->band_gen;
    }
    if (ctx->kernel == SALT_KERNEL_DIRECT) {
        ctx->last_kernel = SALT_KERNEL_DIRECT * 32;
        cudaError_t e = launch_direct(ctx, b, o, mode, st);
        return e == cudaSuccess ? SALT_OK : cuda_err(ctx, e, "kernel launch");
    }
    int key = 0;
    const int tile = ctx->tile_samples;
    if (ctx->kernel == SALT_KERNEL_FACTORISED) {
        key = cfg_key(FAM_CTA, tile > 0 ? tile : cfg_tile(default_config(ctx, p)));
    } else if (ctx->kernel == SALT_KERNEL_UNIT) {
        const int ts = tile == 2 ? 2 : 1;
        if (!unit_ok(ctx, p, ts))
            return set_err(ctx, SALT_ERR_INVALID, "warp-unit kernel: >128 phase nodes, no bands or scratch too large");
        key = cfg_key(FAM_UNIT, ts);
    } else if (ctx->kernel == SALT_KERNEL_BANDWARP) {
        if (ctx->mp.n_phase > bandwarp_max_phase())
            return set_err(ctx, SALT_ERR_INVALID, "band-warp kernel supports at most 128 phase nodes");
        key = cfg_key(FAM_WARP, tile == 2 ? 2 : 1);
    } else if (p->choice[mode] >= 0) {
        key = p->choice[mode];
    } else {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (p->temporary || cs != cudaStreamCaptureStatusNone) {
            key = default_config(ctx, p);
        } else {
            const std::string sig = plan_signature(ctx, p, mode);
            std::lock_guard<std::mutex> lk(g_tune.mu);
            g_tune.load();
            auto it = g_tune.best.find(sig);
            if (it != g_tune.best.end()) {
                key = it->second;
            } else {
                int rc = tune(ctx, p, b, o, mode, st, &key);
                if (rc != SALT_OK) return rc;
                g_tune.store(sig, key);
            }
            p->choice[mode] = key;
        }
    }
    if (!p->lists.count(key)) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (cs != cudaStreamCaptureStatusNone)
            return set_err(ctx, SALT_ERR_INVALID, "run a plan once outside stream capture before capturing it");
    }
    int rc = build_items(ctx, p, key, st);
    if (rc != SALT_OK) return rc;
    const int fam = cfg_family(key);
    ctx->last_kernel = (fam == FAM_UNIT ? SALT_KERNEL_UNIT : fam == FAM_WARP ? SALT_KERNEL_BANDWARP
                                                                             : SALT_KERNEL_FACTORISED) * 32 +
                       cfg_tile(key);
    cudaError_t e;
    if (ctx->use_graphs && !p->temporary && replay_graph(ctx, p, key, b, o, mode, st, &e))
        return e == cudaSuccess ? SALT_OK : cuda_err(ctx, e, "graph launch");
    e = launch_key(ctx, p, key, b, o, mode, st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "kernel launch");
    return SALT_OK;
}

// Launch a plan with a fixed configuration (no autotuning, no graph replay):
// for callers whose results must not depend on timing (the same kernel family
// and tile give bitwise the same results run to run).
int run_batch_fixed(salt_ctx *ctx, const BatchDev &b, salt_plan *p, const OutDev &o, int mode, cudaStream_t st,
                    int family, int tile) {
    if (p->band_gen != ctx->band_gen) {
        plan_reset_work(p);
        p->band_gen = ctx->band_gen;
    }
    const int key = cfg_key(family, tile);
    int rc = build_items(ctx, p, key, st);
    if (rc != SALT_OK) return rc;
    cudaError_t e = launch_key(ctx, p, key, b, o, mode, st);
    return e == cudaSuccess ? SALT_OK : cuda_err(ctx, e, "kernel launch");
}

}  // namespace salt

extern "C" int salt_plan_create(salt_ctx *ctx, int64_t n_sn, const int64_t *obs_off, const int64_t *par_off,
                                salt_plan **out) {
    if (!ctx || !out) return SALT_ERR_INVALID;
    *out = nullptr;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    salt_plan *p = new (std::nothrow) salt_plan();
    if (!p) return SALT_ERR_OOM;
    int rc = plan_build(ctx, n_sn, obs_off, par_off, 0, p, 0, false);
    if (rc == SALT_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "plan upload");
    }
    if (rc != SALT_OK) {
        plan_free(p, 0);
        delete p;
        return rc;
    }
    *out = p;
    return SALT_OK;
}

extern "C" void salt_plan_destroy(salt_plan *plan) {
    if (!plan) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(plan->device);
    plan_free(plan, 0);
    cudaSetDevice(prev);
    (void)cudaGetLastError();
    delete plan;
}

extern "C" int salt_bandflux_offsets(int64_t n_sn, const int64_t *obs_off, const int64_t *par_off,
                                     int64_t *bf_off) {
    if (n_sn < 0 || !bf_off || !offsets_ok(n_sn, obs_off) || !offsets_ok(n_sn, par_off)) return SALT_ERR_INVALID;
    bf_off[0] = 0;
    for (int64_t s = 0; s < n_sn; ++s)
        bf_off[s + 1] = bf_off[s] + (obs_off[s + 1] - obs_off[s]) * (par_off[s + 1] - par_off[s]);
    return SALT_OK;
}

// ------------------------------------------------------------------ batch calls

static int batch_call(salt_ctx *ctx, const salt_batch *bt, int mode, float *bf, double *chi2, float *grad,
                      void *stream) {
    if (!ctx || !bt) return SALT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (bt->n_sn < 0 || !bt->obs_off || !bt->par_off) return set_err(ctx, SALT_ERR_INVALID, "missing offsets");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const salt_plan *plan = bt->plan;
    salt_plan tmp;
    if (plan) {
        if (plan->ctx != ctx || plan->n_sn != bt->n_sn ||
            std::memcmp(plan->obs_off_h.data(), bt->obs_off, (bt->n_sn + 1) * 8) != 0 ||
            std::memcmp(plan->par_off_h.data(), bt->par_off, (bt->n_sn + 1) * 8) != 0)
            return set_err(ctx, SALT_ERR_INVALID, "plan does not match the batch offsets");
    }
    const int64_t n_obs = bt->n_sn ? bt->obs_off[bt->n_sn] : 0;
    const int64_t n_par = bt->n_sn ? bt->par_off[bt->n_sn] : 0;
    if (n_obs > 0 && (!bt->mjd || !bt->band || !bt->flux || !bt->fluxerr || !bt->zp))
        return set_err(ctx, SALT_ERR_INVALID, "missing observation arrays");
    if (n_par > 0 && (!bt->t0 || !bt->z || !bt->x0 || !bt->x1 || !bt->c))
        return set_err(ctx, SALT_ERR_INVALID, "missing parameter arrays");
    if (mode == MODE_BANDFLUX && !bf) {
        // an output is needed only when there is a bandflux to write
        int64_t n_bf = 0;
        for (int64_t s = 0; s < bt->n_sn && n_bf == 0; ++s)
            n_bf += (bt->obs_off[s + 1] - bt->obs_off[s]) * (bt->par_off[s + 1] - bt->par_off[s]);
        if (n_bf > 0) return set_err(ctx, SALT_ERR_INVALID, "missing output");
    }
    if (mode != MODE_BANDFLUX && !chi2 && n_par > 0) return set_err(ctx, SALT_ERR_INVALID, "missing output");
    if (mode == MODE_GRAD && !grad && n_par > 0) return set_err(ctx, SALT_ERR_INVALID, "missing output");
    if (!plan) {
        tmp.temporary = true;
        int rc = plan_build(ctx, bt->n_sn, bt->obs_off, bt->par_off, 0, &tmp, st, true);
        if (rc != SALT_OK) { plan_free(&tmp, st); return rc; }
        plan = &tmp;
    } else {
        if (!offsets_ok(bt->n_sn, bt->obs_off) || !offsets_ok(bt->n_sn, bt->par_off))
            return set_err(ctx, SALT_ERR_INVALID, "offsets must start at 0 and be nondecreasing");
    }
    BatchDev b{};
    b.n_sn = bt->n_sn;
    b.n_obs = n_obs;
    b.n_par = n_par;
    b.obs_off = plan->obs_off_d;
    b.par_off = plan->par_off_d;
    b.mjd = bt->mjd; b.band = bt->band; b.flux = bt->flux; b.fluxerr = bt->fluxerr; b.zp = bt->zp;
    b.t0 = bt->t0; b.z = bt->z; b.x0 = bt->x0; b.x1 = bt->x1; b.c = bt->c;
    int rc = SALT_OK;
    if (bt->validate) {
        cudaError_t e = cudaMemsetAsync(ctx->err_d + 1, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_validate(ctx, b, ctx->err_d + 1, st);
        int flag = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, ctx->err_d + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "validation");
        else if (flag) rc = set_err(ctx, SALT_ERR_INVALID, (flag & ERRBIT_BAND) ? "band id out of range"
                                                            : (flag & ERRBIT_SIGMA) ? "fluxerr must be > 0"
                                                                                    : "non-finite value or z <= -1");
    }
    if (rc == SALT_OK) {
        OutDev o{bf, plan->bf_off_d, chi2, grad, ctx->err_d};
        rc = run_batch(ctx, b, plan, o, mode, st);
    }
    if (plan == &tmp) plan_free(&tmp, st);
    return rc;
}

extern "C" int salt_bandflux(salt_ctx *ctx, const salt_batch *batch, float *out, void *cuda_stream) {
    return batch_call(ctx, batch, MODE_BANDFLUX, out, nullptr, nullptr, cuda_stream);
}

extern "C" int salt_chi2(salt_ctx *ctx, const salt_batch *batch, double *chi2, void *cuda_stream) {
    return batch_call(ctx, batch, MODE_CHI2, nullptr, chi2, nullptr, cuda_stream);
}

extern "C" int salt_chi2_grad(salt_ctx *ctx, const salt_batch *batch, double *chi2, float *grad,
                              void *cuda_stream) {
    return batch_call(ctx, batch, MODE_GRAD, nullptr, chi2, grad, cuda_stream);
}

extern "C" int salt_check(salt_ctx *ctx, void *cuda_stream) {
    if (!ctx) return SALT_ERR_INVALID;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, ctx->err_d, sizeof(int), cudaMemcpyDeviceToHost, st), "read error word");
    CK(cudaStreamSynchronize(st), "synchronize");
    CK(cudaMemsetAsync(ctx->err_d, 0, sizeof(int), st), "clear error word");
    CK(cudaStreamSynchronize(st), "synchronize");
    if (flag)
        return set_err(ctx, SALT_ERR_DATA,
                       (flag & ERRBIT_BAND)    ? "a kernel met a band id out of range"
                       : (flag & ERRBIT_SIGMA) ? "a kernel met fluxerr <= 0"
                       : (flag & ERRBIT_PARAM) ? "a kernel met non-finite parameters"
                                               : "a bandflux was not finite: FP32 overflow of the colour factor or "
                                                 "the surfaces (or a non-finite zero point)");
    return SALT_OK;
}

// ------------------------------------------------------------------ options

extern "C" int salt_set_option(salt_ctx *ctx, int32_t option, int64_t value) {
    if (!ctx) return SALT_ERR_INVALID;
    switch (option) {
        case SALT_OPT_KERNEL:
            if (value < 0 || value > 4) return SALT_ERR_INVALID;
            ctx->kernel = (int)value;
            return SALT_OK;
        case SALT_OPT_TILE_SAMPLES:
            if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
                return SALT_ERR_INVALID;
            ctx->tile_samples = (int)value;
            return SALT_OK;
        case SALT_OPT_GRAPHS:
            ctx->use_graphs = value ? 1 : 0;
            return SALT_OK;
        case SALT_OPT_SERVE_CHUNK:
            if (value < 1 || value > 4096) return SALT_ERR_INVALID;
            ctx->serve_chunk = (int)value;
            return SALT_OK;
    }
    return SALT_ERR_INVALID;
}

extern "C" int salt_get_option(const salt_ctx *ctx, int32_t option, int64_t *value) {
    if (!ctx || !value) return SALT_ERR_INVALID;
    switch (option) {
        case SALT_OPT_KERNEL: *value = ctx->kernel; return SALT_OK;
        case SALT_OPT_TILE_SAMPLES: *value = ctx->tile_samples; return SALT_OK;
        case SALT_OPT_GRAPHS: *value = ctx->use_graphs; return SALT_OK;
        case SALT_OPT_SERVE_CHUNK: *value = ctx->serve_chunk; return SALT_OK;
        case SALT_OPT_LAST_KERNEL: *value = ctx->last_kernel; return SALT_OK;
    }
    return SALT_ERR_INVALID;
}

// ------------------------------------------------------------------ serving

extern "C" int salt_serve_submit(salt_ctx *ctx, const salt_request *req, uint64_t *ticket) {
    if (!ctx || !ctx->serve) return SALT_ERR_INVALID;
    return serve_submit(ctx->serve, req, ticket);
}

extern "C" int salt_serve_poll(salt_ctx *ctx, uint64_t ticket, int32_t wait_ms, double *chi2, float *grad) {
    if (!ctx || !ctx->serve) return SALT_ERR_INVALID;
    return serve_poll(ctx->serve, ticket, wait_ms, chi2, grad);
}

extern "C" int salt_serve_cancel(salt_ctx *ctx, uint64_t ticket) {
    if (!ctx || !ctx->serve) return SALT_ERR_INVALID;
    return serve_cancel(ctx->serve, ticket);
}

extern "C" int salt_serve_stats_get(salt_ctx *ctx, salt_serve_stats *out) {
    if (!ctx || !ctx->serve || !out) return SALT_ERR_INVALID;
    return serve_stats(ctx->serve, out);
}

// ------------------------------------------------------------------ misc

extern "C" const char *salt_status_str(int status) {
    switch (status) {
        case SALT_OK: return "ok";
        case SALT_PENDING: return "pending";
        case SALT_ERR_INVALID: return "invalid argument or data";
        case SALT_ERR_OOM: return "out of memory";
        case SALT_ERR_CUDA: return "CUDA error";
        case SALT_ERR_TIMEOUT: return "timeout";
        case SALT_ERR_NOT_FOUND: return "ticket not found";
        case SALT_ERR_CANCELLED: return "cancelled";
        case SALT_ERR_DATA: return "invalid batch data met by a kernel";
    }
    return "unknown status";
}

extern "C" const char *salt_last_error(const salt_ctx *ctx) {
    if (!ctx) return "no context";
    return ctx->last_error.c_str();
}
