// chi^2 + gradient without device-memory allocation: the warp-unit kernel at
// one parameter sample per unit, with every piece of per-call scratch (the
// offset copies, the work list, the unit counter, the per-band partials and
// arrival counters) carved out of one statically sized device array instead
// of plan-owned or stream-ordered allocations. The paper has no counterpart:
// this serves callers that must not allocate device memory during a call.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "salt_internal.cuh"

// One array per device (a module global), zero at module load. Every call
// clears, on its stream, the parts that must start at zero.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SALT_NOALLOC_SCRATCH_BYTES];

namespace salt {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned char *g_addr[kMaxDevices];  // device address of the array, looked up once per device

// Look the array's address up on the current device (once per device).
cudaError_t scratch_address(int device, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

int fail(salt_ctx *ctx, int code, const std::string &msg) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_error = msg;
    return code;
}

int fail_cuda(salt_ctx *ctx, cudaError_t e, const char *what) {
    (void)cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? SALT_ERR_OOM : SALT_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }

bool offsets_valid(int64_t n_sn, const int64_t *off) {
    if (off[0] != 0) return false;
    for (int64_t s = 0; s < n_sn; ++s)
        if (off[s + 1] < off[s] || off[s + 1] - off[s] > INT32_MAX / 2) return false;
    return true;
}

// One work item per parameter sample j: its supernova s is the largest s with
// par_off[s] <= j (empty supernovae own no samples and are skipped).
__global__ void k_noalloc_items(const int64_t *obs_off, const int64_t *par_off, int64_t n_sn, int n_par,
                                WorkItem *items) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_par) return;
    int64_t lo = 0, hi = n_sn;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (par_off[mid] <= j) lo = mid; else hi = mid;
    }
    WorkItem w;
    w.obs0 = obs_off[lo];
    w.par0 = j;
    w.bf0 = 0;
    w.nobs = (int32_t)(obs_off[lo + 1] - obs_off[lo]);
    w.nj = 1;
    w.jloc0 = (int32_t)(j - par_off[lo]);
    w.pad = 0;
    items[j] = w;
}

}  // namespace
}  // namespace salt

using namespace salt;

extern "C" int salt_chi2_grad_noalloc(salt_ctx *ctx, const salt_batch *bt, double *chi2, float *grad,
                                      void *cuda_stream) {
    if (!ctx || !bt) return SALT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (bt->n_sn < 0 || !bt->obs_off || !bt->par_off) return fail(ctx, SALT_ERR_INVALID, "missing offsets");
    if (!offsets_valid(bt->n_sn, bt->obs_off) || !offsets_valid(bt->n_sn, bt->par_off))
        return fail(ctx, SALT_ERR_INVALID, "offsets must start at 0 and be nondecreasing");
    const int64_t n_sn = bt->n_sn;
    const int64_t n_obs = n_sn ? bt->obs_off[n_sn] : 0;
    const int64_t n_par = n_sn ? bt->par_off[n_sn] : 0;
    if (n_obs > 0 && (!bt->mjd || !bt->band || !bt->flux || !bt->fluxerr || !bt->zp))
        return fail(ctx, SALT_ERR_INVALID, "missing observation arrays");
    if (n_par > 0 && (!bt->t0 || !bt->z || !bt->x0 || !bt->x1 || !bt->c))
        return fail(ctx, SALT_ERR_INVALID, "missing parameter arrays");
    if (n_par > 0 && (!chi2 || !grad)) return fail(ctx, SALT_ERR_INVALID, "missing output");
    if (ctx->mp.n_phase > unit_max_phase() || ctx->mp.bands.n_bands < 1)
        return fail(ctx, SALT_ERR_INVALID, "the no-allocation call needs a model with at most " +
                                               std::to_string(unit_max_phase()) + " phase nodes and a band");
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return fail(ctx, SALT_ERR_INVALID, "device ordinal out of range for the no-allocation call");

    // scratch layout: unit counter | obs_off | par_off | work list | unit partials + arrival counters
    const int nb = ctx->mp.bands.n_bands;
    const size_t off_bytes = al256((size_t)(n_sn + 1) * sizeof(int64_t));
    const size_t o_obs = 256, o_par = o_obs + off_bytes, o_items = o_par + off_bytes;
    const size_t o_unit = o_items + al256((size_t)n_par * sizeof(WorkItem));
    const size_t unit_bytes = n_par <= INT32_MAX ? unit_scratch_bytes((int)n_par, 1, nb) : SIZE_MAX / 2;
    const size_t need = o_unit + unit_bytes;
    if (n_par > INT32_MAX || need > SALT_NOALLOC_SCRATCH_BYTES) {
        char msg[192];
        std::snprintf(msg, sizeof msg,
                      "batch needs %zu bytes of scratch; the no-allocation call has %zu "
                      "(SALT_NOALLOC_SCRATCH_BYTES)",
                      need, (size_t)SALT_NOALLOC_SCRATCH_BYTES);
        return fail(ctx, SALT_ERR_INVALID, msg);
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaSetDevice");
    if (n_par == 0) return SALT_OK;
    unsigned char *base = nullptr;
    if ((e = scratch_address(ctx->device, &base)) != cudaSuccess) return fail_cuda(ctx, e, "cudaGetSymbolAddress");

    int *counter = reinterpret_cast<int *>(base);
    int64_t *obs_off_d = reinterpret_cast<int64_t *>(base + o_obs);
    int64_t *par_off_d = reinterpret_cast<int64_t *>(base + o_par);
    WorkItem *items = reinterpret_cast<WorkItem *>(base + o_items);
    void *unit = base + o_unit;

    // pageable HOST offsets: staged before cudaMemcpyAsync returns
    if ((e = cudaMemcpyAsync(obs_off_d, bt->obs_off, (n_sn + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(par_off_d, bt->par_off, (n_sn + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return fail_cuda(ctx, e, "upload offsets");
    // the arrival counters must start at zero (the launcher clears the unit counter)
    if ((e = cudaMemsetAsync(unit, 0, unit_bytes, st)) != cudaSuccess) return fail_cuda(ctx, e, "clear scratch");
    const int threads = 256;
    k_noalloc_items<<<(unsigned)((n_par + threads - 1) / threads), threads, 0, st>>>(obs_off_d, par_off_d, n_sn,
                                                                                      (int)n_par, items);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(ctx, e, "work list");

    BatchDev b{};
    b.n_sn = n_sn;
    b.n_obs = n_obs;
    b.n_par = n_par;
    b.obs_off = obs_off_d;
    b.par_off = par_off_d;
    b.mjd = bt->mjd; b.band = bt->band; b.flux = bt->flux; b.fluxerr = bt->fluxerr; b.zp = bt->zp;
    b.t0 = bt->t0; b.z = bt->z; b.x0 = bt->x0; b.x1 = bt->x1; b.c = bt->c;
    if (bt->validate) {
        int flag = 0;
        e = cudaMemsetAsync(ctx->err_d + 1, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_validate(ctx, b, ctx->err_d + 1, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, ctx->err_d + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail_cuda(ctx, e, "validation");
        if (flag)
            return fail(ctx, SALT_ERR_INVALID, (flag & ERRBIT_BAND)    ? "band id out of range"
                                               : (flag & ERRBIT_SIGMA) ? "fluxerr must be > 0"
                                                                       : "non-finite value or z <= -1");
    }
    OutDev o{nullptr, nullptr, chi2, grad, ctx->err_d};
    e = launch_unit_items(ctx, 1, items, (int)n_par, counter, unit, b, o, MODE_GRAD, st);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "unit kernel");
    return SALT_OK;
}
