// Batched nested sampling of the SALT posterior, one independent run per
// supernova, all runs in lockstep on the device (the paper samples its
// posterior with nested sampling, Implementation, first paragraph: ns.py).
//
// Per supernova: N live points in a uniform prior box over the free
// parameters. An iteration orders them by log L = -chi^2/2 (ties by index),
// stops when they could add less than dlogz to log Z, else removes the k
// lowest (the j-th removal, with N - j points live, shrinks log X by
// 1/(N - j) and adds weight X_before - X_after to the evidence and the
// posterior moments) and replaces them: k random-walk chains, each started
// at a survivor picked uniformly, take M steps theta + f sigma * n (sigma the
// survivors' standard deviation, f a scale adapted by exp(acceptance - 1/2))
// and accept proposals inside the box above the k-th removed log L. The
// proposals of all chains of all supernovae form one batch per step: a
// chi^2 evaluation by the factorised kernels. At the stop the live points
// share the remaining volume. Random numbers: Philox4x32-10 (Salmon et al.,
// SC'11), counter (supernova, iteration or point, index, stream), key =
// the seed; evidence sums in FP64 with a running maximum. One iteration is
// captured as a CUDA graph and replayed.
#include <cmath>
#include <cstring>
#include <string>

#include "salt_internal.cuh"

namespace salt {
namespace nsd {

constexpr int NP = 5;
constexpr int NMAX = 1024;  // live points per supernova (one block sorts them)
enum { STREAM_INIT = 0, STREAM_START = 1, STREAM_STEP = 2 };

struct Sn {
    double logx, f, lstar;
    double m, s0, s1[NP], s2[NP], sl;  // evidence / moment sums, scaled by exp(-m)
    double sig[NP];
    double lo[NP], hi[NP];
    int it, done, status, n_acc;
};

struct Opts {
    int n_sn, N, k, M, mask, max_iter;
    unsigned long long seed;
    double dlogz;
};

struct Dev {
    Sn *sn;
    double *live_th, *live_l;          // [n_sn][N][5], [n_sn][N]
    double *chain_th, *chain_l;        // [n_sn][k][5], [n_sn][k]
    double *prop_th;                   // [n_sn][k][5]
    int *slot, *prop_in;               // [n_sn][k]
    double *t0i; float *zi, *x0i, *x1i, *ci;  // evaluation arrays, init layout [n_sn][N]
    double *t0c; float *zc, *x0c, *x1c, *cc;  // evaluation arrays, chain layout [n_sn][k]
    double *chi2i, *chi2c;
    int *n_done;
};

// ---- Philox4x32-10
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}
__device__ __forceinline__ uint4 draw(unsigned long long seed, unsigned s, unsigned a, unsigned b, int stream,
                                      int part) {
    return philox(make_uint4(s, a, b, 4u * stream + part), make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}
__device__ __forceinline__ double u01(unsigned x) { return ((double)x + 0.5) * 0x1p-32; }

__device__ void uniforms5(unsigned long long seed, int s, int a, int b, int stream, double u[NP]) {
    const uint4 w0 = draw(seed, s, a, b, stream, 0), w1 = draw(seed, s, a, b, stream, 1);
    u[0] = u01(w0.x); u[1] = u01(w0.y); u[2] = u01(w0.z); u[3] = u01(w0.w); u[4] = u01(w1.x);
}
__device__ void normals5(unsigned long long seed, int s, int a, int b, int stream, double n[NP]) {
    const uint4 w0 = draw(seed, s, a, b, stream, 0), w1 = draw(seed, s, a, b, stream, 1);
    const unsigned w[6] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
    double out[6];
#pragma unroll
    for (int q = 0; q < 3; ++q) {  // Box-Muller
        const double r = sqrt(-2.0 * log(u01(w[2 * q])));
        const double ang = 2.0 * M_PI * u01(w[2 * q + 1]);
        out[2 * q] = r * cos(ang);
        out[2 * q + 1] = r * sin(ang);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) n[i] = out[i];
}

// The kernels evaluate z, x0, x1, c in FP32 and t0 in FP64: keep points
// exactly at what gets evaluated.
__device__ __forceinline__ double fp32(double v, int i) { return i == 1 ? v : (double)(float)v; }

__device__ __forceinline__ bool free_p(int mask, int i) { return (mask >> i) & 1; }

__device__ void acc_add(Sn &st, double lwl, const double *th, double logl) {
    if (!(lwl > -INFINITY)) return;
    if (lwl > st.m) {
        const double r = st.m > -INFINITY ? exp(st.m - lwl) : 0.0;
        st.s0 *= r;
        st.sl *= r;
#pragma unroll
        for (int i = 0; i < NP; ++i) { st.s1[i] *= r; st.s2[i] *= r; }
        st.m = lwl;
    }
    const double e = exp(lwl - st.m);
    st.s0 += e;
    st.sl += e * logl;
#pragma unroll
    for (int i = 0; i < NP; ++i) { st.s1[i] += e * th[i]; st.s2[i] += e * th[i] * th[i]; }
}

__device__ __forceinline__ void write_eval(double *t0, float *z, float *x0, float *x1, float *c, size_t q,
                                           const double *th) {
    z[q] = (float)th[0];
    t0[q] = th[1];
    x0[q] = (float)th[2];
    x1[q] = (float)th[3];
    c[q] = (float)th[4];
}

__device__ __forceinline__ double logl_of(double chi2) { return isfinite(chi2) ? -0.5 * chi2 : -INFINITY; }

// Live points drawn uniformly in the box; thread per (supernova, point).
__global__ void k_init(Opts op, Dev d, const double *t0, const float *z, const float *x0, const float *x1,
                       const float *c, const double *lower, const double *upper) {
    const int s = blockIdx.y, p = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= op.n_sn || p >= op.N) return;
    const double ref[NP] = {(double)z[s], t0[s], (double)x0[s], (double)x1[s], (double)c[s]};
    double lo[NP], hi[NP];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        lo[i] = free_p(op.mask, i) ? lower[NP * s + i] : ref[i];
        hi[i] = free_p(op.mask, i) ? upper[NP * s + i] : ref[i];
        if (!(lo[i] <= hi[i]) || !isfinite(lo[i]) || !isfinite(hi[i])) ok = false;
    }
    double u[NP];
    uniforms5(op.seed, s, 0, p, STREAM_INIT, u);
    double th[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i)
        th[i] = fp32(free_p(op.mask, i) ? lo[i] + u[i] * (hi[i] - lo[i]) : ref[i], i);
    const size_t q = (size_t)s * op.N + p;
#pragma unroll
    for (int i = 0; i < NP; ++i) d.live_th[NP * q + i] = th[i];
    write_eval(d.t0i, d.zi, d.x0i, d.x1i, d.ci, q, th);
    if (p == 0) {
        Sn st;
        st.logx = 0.0;
        st.f = 1.0;
        st.lstar = -INFINITY;
        st.m = -INFINITY;
        st.s0 = st.sl = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            st.s1[i] = st.s2[i] = st.sig[i] = 0.0;
            st.lo[i] = lo[i];
            st.hi[i] = hi[i];
        }
        st.it = 0;
        st.done = ok ? 0 : 1;
        st.status = ok ? 0 : SALT_FIT_INVALID;
        st.n_acc = 0;
        d.sn[s] = st;
        if (!ok) atomicAdd(d.n_done, 1);  // an empty or non-finite box: nothing to sample
    }
}

__global__ void k_init_logl(Opts op, Dev d) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < (size_t)op.n_sn * op.N) d.live_l[q] = logl_of(d.chi2i[q]);
}

// Order, test for the stop, remove the k lowest, set up the chains; one block
// per supernova (blockDim = the power of two >= N).
__global__ void k_select(Opts op, Dev d) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int s = blockIdx.x, tid = threadIdx.x, P = blockDim.x;
    double *key = (double *)sm;
    int *idx = (int *)(key + P);
    __shared__ int s_done;
    __shared__ double s_sig[NP];
    Sn &st = d.sn[s];
    const double *ll = d.live_l + (size_t)s * op.N;
    const double *th = d.live_th + (size_t)s * op.N * NP;
    key[tid] = tid < op.N ? ll[tid] : INFINITY;
    idx[tid] = tid;
    __syncthreads();
    // bitonic sort ascending by (log L, index)
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int o = tid ^ stride;
            if (o > tid) {
                const bool up = (tid & size) == 0;
                const double ka = key[tid], kb = key[o];
                const int ia = idx[tid], ib = idx[o];
                const bool gt = ka > kb || (ka == kb && ia > ib);
                if (gt == up) {
                    key[tid] = kb; key[o] = ka;
                    idx[tid] = ib; idx[o] = ia;
                }
            }
            __syncthreads();
        }
    if (tid == 0) {
        int done = st.done;
        if (!done) {
            if (st.it > 0) {  // scale update from the last iteration's acceptance
                const double rate = (double)st.n_acc / ((double)op.k * op.M);
                st.f = fmin(fmax(st.f * exp(rate - 0.5), 1e-3), 10.0);
                st.n_acc = 0;
            }
            const double z_now = st.s0 > 0.0 ? st.m + log(st.s0) : -INFINITY;
            const double remain = key[op.N - 1] + st.logx;
            bool stop = false;
            if (z_now > -INFINITY) {
                const double hi = fmax(z_now, remain), lo = fmin(z_now, remain);
                stop = hi + log1p(exp(lo - hi)) - z_now < op.dlogz;
            }
            if (stop || st.it >= op.max_iter) {
                const double lw = st.logx - log((double)op.N);
                for (int p = 0; p < op.N; ++p) acc_add(st, lw + ll[p], th + (size_t)NP * p, ll[p]);
                st.done = 1;
                st.status = stop ? st.it : SALT_FIT_MAXITER;
                atomicAdd(d.n_done, 1);
                done = 1;
            } else {
                for (int j = 0; j < op.k; ++j) {
                    const double n_alive = (double)(op.N - j);
                    const double lw = st.logx + log(-expm1(-1.0 / n_alive));
                    const int p = idx[j];
                    acc_add(st, lw + ll[p], th + (size_t)NP * p, ll[p]);
                    st.logx -= 1.0 / n_alive;
                }
                st.lstar = key[op.k - 1];
            }
        }
        s_done = done;
    }
    __syncthreads();
    if (s_done) return;
    // survivors' standard deviation per parameter (two passes, fixed order)
    const int ns = op.N - op.k;
    if (tid < 32) {
        for (int i = 0; i < NP; ++i) {
            double a = 0.0;
            for (int r = op.k + tid; r < op.N; r += 32) a += th[(size_t)NP * idx[r] + i];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            const double mean = a / ns;
            double v = 0.0;
            for (int r = op.k + tid; r < op.N; r += 32) {
                const double e = th[(size_t)NP * idx[r] + i] - mean;
                v += e * e;
            }
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (tid == 0) s_sig[i] = sqrt(v / ns);
        }
    }
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < NP; ++i) st.sig[i] = s_sig[i];
    // chains: start at a survivor picked uniformly, replace the c-th lowest
    for (int c = tid; c < op.k; c += P) {
        const unsigned w = draw(op.seed, s, st.it, c, STREAM_START, 0).x;
        const int r = op.k + (int)(((unsigned long long)w * (unsigned)ns) >> 32);
        const int start = idx[r];
        const size_t q = (size_t)s * op.k + c;
#pragma unroll
        for (int i = 0; i < NP; ++i) d.chain_th[NP * q + i] = th[(size_t)NP * start + i];
        d.chain_l[q] = ll[start];
        d.slot[q] = idx[c];
    }
}

// One random-walk proposal per chain; thread per (supernova, chain).
__global__ void k_propose(Opts op, Dev d, int m) {
    const int s = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= op.n_sn || c >= op.k) return;
    const Sn &st = d.sn[s];
    const size_t q = (size_t)s * op.k + c;
    double th[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) th[i] = d.chain_th[NP * q + i];
    int in = 0;
    if (!st.done) {
        double n[NP];
        normals5(op.seed, s, st.it, m * op.k + c, STREAM_STEP, n);
        in = 1;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            if (free_p(op.mask, i)) th[i] = fp32(th[i] + st.f * st.sig[i] * n[i], i);
            if (!(th[i] >= st.lo[i] && th[i] <= st.hi[i])) in = 0;
        }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) d.prop_th[NP * q + i] = th[i];
    d.prop_in[q] = in;
    // a proposal outside the box is rejected whatever its likelihood: evaluate
    // the chain's current point in its place, so that no parameter far outside
    // the prior (a colour factor beyond the FP32 range, say) reaches the kernel
    if (!in)
#pragma unroll
        for (int i = 0; i < NP; ++i) th[i] = d.chain_th[NP * q + i];
    write_eval(d.t0c, d.zc, d.x0c, d.x1c, d.cc, q, th);
}

// Work items of finished supernovae get no samples, so the chi^2 launches of
// later iterations skip them (their proposals were never used).
__global__ void k_drop_done(WorkItem *items, int n_items, const Sn *sn, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_items && sn[items[i].par0 / k].done) items[i].nj = 0;
}

__global__ void k_accept(Opts op, Dev d) {
    const int s = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= op.n_sn || c >= op.k) return;
    Sn &st = d.sn[s];
    if (st.done) return;
    const size_t q = (size_t)s * op.k + c;
    const double lp = logl_of(d.chi2c[q]);
    if (d.prop_in[q] && lp > st.lstar) {
#pragma unroll
        for (int i = 0; i < NP; ++i) d.chain_th[NP * q + i] = d.prop_th[NP * q + i];
        d.chain_l[q] = lp;
        atomicAdd(&st.n_acc, 1);
    }
}

__global__ void k_commit(Opts op, Dev d) {
    const int s = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= op.n_sn || c >= op.k) return;
    Sn &st = d.sn[s];
    if (st.done) return;
    const size_t q = (size_t)s * op.k + c;
    const int p = d.slot[q];
    const size_t lq = (size_t)s * op.N + p;
#pragma unroll
    for (int i = 0; i < NP; ++i) d.live_th[NP * lq + i] = d.chain_th[NP * q + i];
    d.live_l[lq] = d.chain_l[q];
}

__global__ void k_next(Opts op, Dev d) {  // after the commit: count the iteration
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < op.n_sn && !d.sn[s].done) ++d.sn[s].it;
}

__global__ void k_output(Opts op, Dev d, double *logz, double *logz_err, double *mean, double *sd, int *status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= op.n_sn) return;
    const Sn &st = d.sn[s];
    const double lz = st.s0 > 0.0 ? st.m + log(st.s0) : -INFINITY;
    const double h = st.s0 > 0.0 ? st.sl / st.s0 - lz : 0.0;
    logz[s] = lz;
    logz_err[s] = sqrt(fmax(h, 0.0) / op.N);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const double mu = st.s0 > 0.0 ? st.s1[i] / st.s0 : NAN;
        mean[NP * s + i] = mu;
        sd[NP * s + i] = st.s0 > 0.0 ? sqrt(fmax(st.s2[i] / st.s0 - mu * mu, 0.0)) : NAN;
    }
    status[s] = st.done ? st.status : SALT_FIT_MAXITER;
}

}  // namespace nsd
}  // namespace salt

using namespace salt;

namespace {
int ns_fail(salt_ctx *ctx, int code, const std::string &msg) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_error = msg;
    return code;
}
int ns_cuda(salt_ctx *ctx, cudaError_t e, const char *what) {
    (void)cudaGetLastError();
    return ns_fail(ctx, e == cudaErrorMemoryAllocation ? SALT_ERR_OOM : SALT_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace

extern "C" int salt_nested(salt_ctx *ctx, const salt_batch *bt, const double *lower, const double *upper,
                           const salt_nested_opts *opts, double *logz, double *logz_err, double *mean,
                           double *std_out, int32_t *status, void *cuda_stream) {
    if (!ctx || !bt) return SALT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    salt_nested_opts o = opts ? *opts : salt_nested_opts{};
    if (o.n_live <= 0) o.n_live = 256;
    if (o.n_batch <= 0) o.n_batch = o.n_live / 4 > 0 ? o.n_live / 4 : 1;
    if (o.n_steps <= 0) o.n_steps = 20;
    if (o.max_iter <= 0) o.max_iter = 2000;
    if (o.free_mask == 0) o.free_mask = SALT_FIT_DEFAULT_MASK;
    if (o.dlogz <= 0.0) o.dlogz = 0.1;
    if (o.n_live < 2 || o.n_live > nsd::NMAX || o.n_batch >= o.n_live || (o.free_mask & ~0x1f) != 0)
        return ns_fail(ctx, SALT_ERR_INVALID, "nested: need 2 <= n_live <= 1024, n_batch < n_live, free_mask in 5 bits");
    if (bt->n_sn < 0 || !bt->obs_off || !bt->par_off) return ns_fail(ctx, SALT_ERR_INVALID, "missing offsets");
    const int64_t n_sn = bt->n_sn;
    for (int64_t s = 0; s <= n_sn; ++s)
        if (bt->par_off[s] != s)
            return ns_fail(ctx, SALT_ERR_INVALID, "nested: one parameter sample (the fixed values) per supernova");
    if (n_sn == 0) return SALT_OK;
    if (n_sn * (int64_t)o.n_live > INT32_MAX / 2 || n_sn > 65535)
        return ns_fail(ctx, SALT_ERR_INVALID, "nested: too many supernovae x live points");
    if (!lower || !upper || !logz || !logz_err || !mean || !std_out || !status)
        return ns_fail(ctx, SALT_ERR_INVALID, "nested: missing prior box or output");
    if (!bt->t0 || !bt->z || !bt->x0 || !bt->x1 || !bt->c)
        return ns_fail(ctx, SALT_ERR_INVALID, "missing parameter arrays");
    const int64_t n_obs = bt->obs_off[n_sn];
    if (n_obs > 0 && (!bt->mjd || !bt->band || !bt->flux || !bt->fluxerr || !bt->zp))
        return ns_fail(ctx, SALT_ERR_INVALID, "missing observation arrays");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return ns_cuda(ctx, e, "cudaSetDevice");
    const int n = (int)n_sn, N = o.n_live, k = o.n_batch, M = o.n_steps;

    // plans: N samples per supernova (the initial live points), k per supernova (the chains)
    std::vector<int64_t> off_i(n + 1), off_c(n + 1);
    for (int s = 0; s <= n; ++s) { off_i[s] = (int64_t)s * N; off_c[s] = (int64_t)s * k; }
    salt_plan plan_i, plan_c;
    int rc = plan_build(ctx, n_sn, bt->obs_off, off_i.data(), 0, &plan_i, st, false);
    if (rc == SALT_OK) rc = plan_build(ctx, n_sn, bt->obs_off, off_c.data(), 0, &plan_c, st, false);
    nsd::Dev d{};
    std::vector<void *> owned;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        cudaStreamSynchronize(st);
        for (void *q : owned) cudaFree(q);
        plan_free(&plan_i, st);
        plan_free(&plan_c, st);
    };
    if (rc != SALT_OK) {
        cleanup();
        return rc;
    }
    auto alloc = [&](void **p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(p, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) owned.push_back(*p);
    };
    const size_t nN = (size_t)n * N, nk = (size_t)n * k;
    alloc((void **)&d.sn, n * sizeof(nsd::Sn));
    alloc((void **)&d.live_th, nN * 5 * sizeof(double));
    alloc((void **)&d.live_l, nN * sizeof(double));
    alloc((void **)&d.chain_th, nk * 5 * sizeof(double));
    alloc((void **)&d.chain_l, nk * sizeof(double));
    alloc((void **)&d.prop_th, nk * 5 * sizeof(double));
    alloc((void **)&d.slot, nk * sizeof(int));
    alloc((void **)&d.prop_in, nk * sizeof(int));
    alloc((void **)&d.t0i, nN * sizeof(double));
    alloc((void **)&d.zi, nN * sizeof(float));
    alloc((void **)&d.x0i, nN * sizeof(float));
    alloc((void **)&d.x1i, nN * sizeof(float));
    alloc((void **)&d.ci, nN * sizeof(float));
    alloc((void **)&d.t0c, nk * sizeof(double));
    alloc((void **)&d.zc, nk * sizeof(float));
    alloc((void **)&d.x0c, nk * sizeof(float));
    alloc((void **)&d.x1c, nk * sizeof(float));
    alloc((void **)&d.cc, nk * sizeof(float));
    alloc((void **)&d.chi2i, nN * sizeof(double));
    alloc((void **)&d.chi2c, nk * sizeof(double));
    alloc((void **)&d.n_done, sizeof(int));
    float *grad_dummy = nullptr;  // the chi^2 mode writes no gradient
    if (e == cudaSuccess) e = cudaMemsetAsync(d.n_done, 0, sizeof(int), st);
    if (e != cudaSuccess) {
        rc = ns_cuda(ctx, e, "nested scratch");
        cleanup();
        return rc;
    }
    nsd::Opts op{n, N, k, M, o.free_mask, o.max_iter, (unsigned long long)o.seed, o.dlogz};
    auto batch_of = [&](const salt_plan &p, const double *t0, const float *z, const float *x0, const float *x1,
                        const float *c, int per) {
        BatchDev b{};
        b.n_sn = n_sn;
        b.n_obs = n_obs;
        b.n_par = n_sn * per;
        b.obs_off = p.obs_off_d;
        b.par_off = p.par_off_d;
        b.mjd = bt->mjd; b.band = bt->band; b.flux = bt->flux; b.fluxerr = bt->fluxerr; b.zp = bt->zp;
        b.t0 = t0; b.z = z; b.x0 = x0; b.x1 = x1; b.c = c;
        return b;
    };
    const BatchDev bi = batch_of(plan_i, d.t0i, d.zi, d.x0i, d.x1i, d.ci, N);
    const BatchDev bc = batch_of(plan_c, d.t0c, d.zc, d.x0c, d.x1c, d.cc, k);
    const OutDev oi{nullptr, plan_i.bf_off_d, d.chi2i, grad_dummy, ctx->err_d};
    const OutDev oc{nullptr, plan_c.bf_off_d, d.chi2c, grad_dummy, ctx->err_d};
    // a fixed kernel configuration: results reproduce run to run for a given seed
    const int tile_i = 8, tile_c = k >= 8 ? 8 : k >= 4 ? 4 : k >= 2 ? 2 : 1;

    const dim3 gi((N + 127) / 128, n), gc((k + 127) / 128, n);
    nsd::k_init<<<gi, 128, 0, st>>>(op, d, bt->t0, bt->z, bt->x0, bt->x1, bt->c, lower, upper);
    if ((e = cudaGetLastError()) != cudaSuccess) { rc = ns_cuda(ctx, e, "nested init"); cleanup(); return rc; }
    rc = run_batch_fixed(ctx, bi, &plan_i, oi, MODE_CHI2, st, FAM_CTA, tile_i);
    if (rc == SALT_OK) {
        nsd::k_init_logl<<<(unsigned)((nN + 255) / 256), 256, 0, st>>>(op, d);
        if ((e = cudaGetLastError()) != cudaSuccess) rc = ns_cuda(ctx, e, "nested init");
    }
    int P = 1;
    while (P < N) P <<= 1;
    const size_t sel_smem = (size_t)P * (sizeof(double) + sizeof(int));
    WorkItem *items_c = nullptr;  // the chain plan's work list, once built
    int n_items_c = 0;
    auto iteration = [&](cudaStream_t s) -> int {
        nsd::k_select<<<n, P, sel_smem, s>>>(op, d);
        cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess) return ns_cuda(ctx, e2, "nested select");
        if (items_c) {
            nsd::k_drop_done<<<(n_items_c + 255) / 256, 256, 0, s>>>(items_c, n_items_c, d.sn, k);
            if ((e2 = cudaGetLastError()) != cudaSuccess) return ns_cuda(ctx, e2, "nested drop");
        }
        for (int m = 0; m < M; ++m) {
            nsd::k_propose<<<gc, 128, 0, s>>>(op, d, m);
            if ((e2 = cudaGetLastError()) != cudaSuccess) return ns_cuda(ctx, e2, "nested propose");
            const int r = run_batch_fixed(ctx, bc, &plan_c, oc, MODE_CHI2, s, FAM_CTA, tile_c);
            if (r != SALT_OK) return r;
            nsd::k_accept<<<gc, 128, 0, s>>>(op, d);
            if ((e2 = cudaGetLastError()) != cudaSuccess) return ns_cuda(ctx, e2, "nested accept");
        }
        nsd::k_commit<<<gc, 128, 0, s>>>(op, d);
        nsd::k_next<<<(n + 127) / 128, 128, 0, s>>>(op, d);
        e2 = cudaGetLastError();
        return e2 == cudaSuccess ? SALT_OK : ns_cuda(ctx, e2, "nested commit");
    };
    // first iteration directly (it builds the chain plan's work list), then a captured graph
    if (rc == SALT_OK) rc = iteration(st);
    if (rc == SALT_OK) {
        const auto it = plan_c.lists.find(cfg_key(FAM_CTA, tile_c));
        if (it != plan_c.lists.end()) {
            items_c = it->second.d;
            n_items_c = it->second.n;
        }
    }
    if (rc == SALT_OK && !ctx->capture_stream &&
        (e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        rc = ns_cuda(ctx, e, "nested stream");
    if (rc == SALT_OK) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
        int rc_cap = e == cudaSuccess ? iteration(ctx->capture_stream) : SALT_OK;
        const cudaError_t e_end = e == cudaSuccess ? cudaStreamEndCapture(ctx->capture_stream, &g) : e;
        if (e == cudaSuccess) e = e_end;
        if (e == cudaSuccess && rc_cap == SALT_OK) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || rc_cap != SALT_OK) {
            (void)cudaGetLastError();
            exec = nullptr;
        }
    }
    int done = 0;
    for (int it = 1; rc == SALT_OK && it <= o.max_iter + 1; ++it) {
        if (exec) {
            if ((e = cudaGraphLaunch(exec, st)) != cudaSuccess) { rc = ns_cuda(ctx, e, "nested graph"); break; }
        } else if ((rc = iteration(st)) != SALT_OK) {
            break;
        }
        if ((it & 3) == 0 || it == o.max_iter + 1) {
            e = cudaMemcpyAsync(&done, d.n_done, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { rc = ns_cuda(ctx, e, "nested progress"); break; }
            if (done >= n) break;
        }
    }
    // stragglers (the iteration limit) are finalised by one more selection pass
    if (rc == SALT_OK && done < n) {
        nsd::k_select<<<n, P, sel_smem, st>>>(op, d);
        if ((e = cudaGetLastError()) != cudaSuccess) rc = ns_cuda(ctx, e, "nested finish");
    }
    if (rc == SALT_OK) {
        nsd::k_output<<<(n + 127) / 128, 128, 0, st>>>(op, d, logz, logz_err, mean, std_out, status);
        if ((e = cudaGetLastError()) != cudaSuccess) rc = ns_cuda(ctx, e, "nested output");
    }
    cleanup();
    return rc;
}
