// Microbenchmarks of the device's FP32 FMA rate, L2 read bandwidth and
// shared-memory read bandwidth: the measured side of the roofline
// denominators (the FP32 peak the bench divides by is derived from the SM
// count and clock; this checks it on the device at hand). Not part of the
// photometry path.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "salt_internal.cuh"

namespace salt {
namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

// 8 independent FMA chains per thread, 128 FMAs per iteration; the final
// comparison never holds for these inputs but keeps every chain live.
__global__ void __launch_bounds__(kThreads) k_peak_fma(float *sink, int iters) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1e-3f * (float)threadIdx.x + (float)j;
    const float mul = 0.9999999f, add = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], mul, add);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == -1.0f) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

// `passes` reads of n float4 through L2 only (ld.global.cg), grid-strided.
__global__ void __launch_bounds__(kThreads) k_peak_l2(const float4 *__restrict__ buf, size_t n, int passes,
                                                      float *sink) {
    const size_t stride = (size_t)gridDim.x * kThreads;
    float acc = 0.f;
    for (int p = 0; p < passes; ++p)
        for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    if (acc == -1.0f) sink[blockIdx.x * kThreads + threadIdx.x] = acc;
}

// Conflict-free 16-byte shared-memory reads: each quarter warp reads 128
// consecutive bytes.
__global__ void __launch_bounds__(kThreads) k_peak_smem(int iters, float *sink) {
    __shared__ float4 tile[2048];
    for (int i = threadIdx.x; i < 2048; i += kThreads)
        tile[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float4 v = tile[(idx + r * kThreads) & 2047];
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        idx = (idx + 32) & 2047;
    }
    const float s = (acc.x + acc.y) + (acc.z + acc.w);
    if (s == -1.0f) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

int peak_fail(salt_ctx *ctx, cudaError_t e, const char *what) {
    (void)cudaGetLastError();
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SALT_ERR_OOM : SALT_ERR_CUDA;
}

// Best of `reps` timed launches (after one warm-up) in milliseconds.
template <class F>
cudaError_t best_ms(F launch, cudaStream_t st, int reps, float *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch();
    float best = 1e30f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess) best = std::min(best, t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ms = best;
    return e;
}

}  // namespace
}  // namespace salt

extern "C" int salt_measure_peaks(salt_ctx *ctx, salt_peaks *out) {
    using namespace salt;
    if (!ctx || !out) return SALT_ERR_INVALID;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return peak_fail(ctx, e, "cudaSetDevice");
    const int grid = ctx->num_sms * kBlocksPerSM;
    constexpr size_t kL2Bytes = (size_t)32 << 20;  // well inside the L2
    cudaStream_t st = nullptr;
    float *sink = nullptr;
    float4 *buf = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)grid * kThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&buf, kL2Bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, kL2Bytes, st);
    float ms_fma = 0.f, ms_l2 = 0.f, ms_smem = 0.f;
    const int fma_iters = 4096, l2_passes = 200, smem_iters = 8192;
    if (e == cudaSuccess)
        e = best_ms([&] { k_peak_fma<<<grid, kThreads, 0, st>>>(sink, fma_iters); return cudaGetLastError(); },
                    st, 3, &ms_fma);
    const size_t n4 = kL2Bytes / sizeof(float4);
    if (e == cudaSuccess)
        e = best_ms([&] { k_peak_l2<<<grid, kThreads, 0, st>>>(buf, n4, l2_passes, sink); return cudaGetLastError(); },
                    st, 3, &ms_l2);
    if (e == cudaSuccess)
        e = best_ms([&] { k_peak_smem<<<grid, kThreads, 0, st>>>(smem_iters, sink); return cudaGetLastError(); },
                    st, 3, &ms_smem);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return peak_fail(ctx, e, "peak microbenchmarks");
    const double threads = (double)grid * kThreads;
    out->fp32_tflops = 2.0 * 128.0 * fma_iters * threads / (ms_fma * 1e-3) / 1e12;
    out->l2_read_gbs = (double)kL2Bytes * l2_passes / (ms_l2 * 1e-3) / 1e9;
    out->smem_read_gbs = 16.0 * 8.0 * smem_iters * threads / (ms_smem * 1e-3) / 1e9;
    int khz = 0;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device) != cudaSuccess) khz = 0;
    out->sm_clock_max_mhz = khz / 1000.0;
    out->num_sms = ctx->num_sms;
    return SALT_OK;
}
