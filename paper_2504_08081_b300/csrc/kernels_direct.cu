// Direct kernels: every (sample, observation, band sample) evaluated straight
// from the model form (Eq. 1) and the trapezoid band integral (Eq. 2), plus the
// validation pass. One warp per parameter sample; lanes stride over the band's
// wavelength samples; a warp reduction closes each band integral.
#include <cstdio>

#include "device_math.cuh"

namespace salt {

__device__ __forceinline__ int64_t sn_of_sample(const int64_t *off, int64_t n_sn, int64_t j) {
    // largest s with off[s] <= j (then off[s+1] > j; empty supernovae are skipped)
    int64_t lo = 0, hi = n_sn;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool params_ok(float z, double t0, float x0, float x1, float c) {
    return isfinite(z) && z > -1.0f && isfinite(t0) && isfinite(x0) && isfinite(x1) && isfinite(c);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_direct(ModelParams m, BatchDev b, OutDev o) {
    constexpr bool GRAD = MODE == MODE_GRAD;
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= b.n_par) return;
    const int64_t s = sn_of_sample(b.par_off, b.n_sn, j);
    const int64_t i0 = b.obs_off[s], i1 = b.obs_off[s + 1];
    const int64_t jl = j - b.par_off[s];
    const float z = b.z[j], x0 = b.x0[j], x1 = b.x1[j], c = b.c[j];
    const double t0 = b.t0[j];
    bool bad = !params_ok(z, t0, x0, x1, c);
    float a;
    const float4 pm = phase_map(m, bad ? 0.f : z, bad ? 0.0 : t0, a);
    double chi2 = 0.0;
    float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t i = i0; i < i1; ++i) {
        const int bnd = b.band[i];
        const float sig = b.fluxerr[i];
        if (bnd < 0 || bnd >= m.bands.n_bands || !(sig > 0.0f) || bad) {
            if (lane == 0 && !bad) atomicOr(o.err, (bnd < 0 || bnd >= m.bands.n_bands) ? ERRBIT_BAND : ERRBIT_SIGMA);
            bad = true;
            if (MODE == MODE_BANDFLUX && lane == 0)
                o.bandflux[o.bf_off[s] + jl * (i1 - i0) + (i - i0)] = __int_as_float(0x7fc00000);
            continue;
        }
        Taps4 tp;
        float p;
        phase_taps<GRAD>(m, split_f2(b.mjd[i]), pm, tp, p);
        float accB = 0.f, acc1 = 0.f, accC = 0.f, accP = 0.f, accL = 0.f;
        const int off = m.bands.off[bnd], K = m.bands.n[bnd];
        for (int k = lane; k < K; k += 32) {
            const float lam = __ldg(m.band_lam + off + k);
            const float wk = __ldg(m.band_w + off + k);
            const float lr = lam * a;
            Taps4 tl;
            wave_taps<GRAD>(m, lr, tl);
            float dcl;
            const float cl = colour_law(m, lr, dcl);
            const float C = exp2f(kColour * c * cl);
            float M0 = 0.f, M1 = 0.f, M0p = 0.f, M1p = 0.f, M0l = 0.f, M1l = 0.f;
#pragma unroll
            for (int ra = 0; ra < 4; ++ra) {
                const float2 *row = m.g01 + (size_t)(tp.first + ra) * m.nw_pitch + tl.first;
                float r0 = 0.f, r1 = 0.f, rl0 = 0.f, rl1 = 0.f;
#pragma unroll
                for (int cb = 0; cb < 4; ++cb) {
                    const float2 gv = __ldg(row + cb);
                    r0 = fmaf(tl.w[cb], gv.x, r0);
                    r1 = fmaf(tl.w[cb], gv.y, r1);
                    if (GRAD) {
                        rl0 = fmaf(tl.dw[cb], gv.x, rl0);
                        rl1 = fmaf(tl.dw[cb], gv.y, rl1);
                    }
                }
                M0 = fmaf(tp.w[ra], r0, M0);
                M1 = fmaf(tp.w[ra], r1, M1);
                if (GRAD) {
                    M0p = fmaf(tp.dw[ra], r0, M0p);
                    M1p = fmaf(tp.dw[ra], r1, M1p);
                    M0l = fmaf(tp.w[ra], rl0, M0l);
                    M1l = fmaf(tp.w[ra], rl1, M1l);
                }
            }
            const float S = fmaf(x1, M1, M0);
            const float wC = wk * C;
            accB = fmaf(wC, S, accB);
            if (GRAD) {
                acc1 = fmaf(wC, M1, acc1);
                accC = fmaf(wC * S, kColourLn * cl, accC);
                accP = fmaf(wC, fmaf(x1, M1p, M0p), accP);
                accL = fmaf(wC * lr, fmaf(S, kColourLn * c * dcl, fmaf(x1, M1l, M0l)), accL);
            }
        }
        accB = warp_sum(accB);
        const float zpf = zp_scale(b.zp[i]);
        const float pre = x0 * a * zpf;
        const float B = pre * accB;
        if (lane == 0 && !isfinite(B)) atomicOr(o.err, ERRBIT_RANGE);
        if (MODE == MODE_BANDFLUX) {
            if (lane == 0) o.bandflux[o.bf_off[s] + jl * (i1 - i0) + (i - i0)] = B;
        } else {
            const float r = (b.flux[i] - B) / sig;
            chi2 = fma((double)r, (double)r, chi2);
            if (GRAD) {
                acc1 = warp_sum(acc1);
                accC = warp_sum(accC);
                accP = warp_sum(accP);
                accL = warp_sum(accL);
                const float gi = -2.0f * r / sig;
                g[0] += gi * (-a * B - pre * a * fmaf(p, accP, accL));
                g[1] += gi * pre * accP * (-a);
                g[2] += gi * a * zpf * accB;
                g[3] += gi * pre * acc1;
                g[4] += gi * pre * accC;
            }
        }
    }
    if (bad && lane == 0 && !params_ok(z, t0, x0, x1, c)) atomicOr(o.err, ERRBIT_PARAM);
    if (MODE != MODE_BANDFLUX && lane == 0) {
        const double qn = __longlong_as_double(0x7ff8000000000000ll);
        o.chi2[j] = bad ? qn : chi2;
        if (GRAD) {
#pragma unroll
            for (int q = 0; q < 5; ++q) o.grad[5 * j + q] = bad ? __int_as_float(0x7fc00000) : g[q];
        }
    }
    if (MODE == MODE_BANDFLUX && bad && lane == 0) {
        for (int64_t i = i0; i < i1; ++i)
            o.bandflux[o.bf_off[s] + jl * (i1 - i0) + (i - i0)] = __int_as_float(0x7fc00000);
    }
}

// Validation pass: band ids in range, fluxerr > 0, finite values, z > -1.
__global__ void k_validate(int n_bands, BatchDev b, int *flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bits = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b.n_obs; i += stride) {
        const int bd = b.band[i];
        if (bd < 0 || bd >= n_bands) bits |= ERRBIT_BAND;
        const float e = b.fluxerr[i];
        if (!(e > 0.0f) || !isfinite(e)) bits |= ERRBIT_SIGMA;
        if (!isfinite(b.mjd[i]) || !isfinite(b.flux[i]) || !isfinite(b.zp[i])) bits |= ERRBIT_PARAM;
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < b.n_par; j += stride)
        if (!params_ok(b.z[j], b.t0[j], b.x0[j], b.x1[j], b.c[j])) bits |= ERRBIT_PARAM;
    if (bits) atomicOr(flag, bits);
}

cudaError_t launch_direct(const salt_ctx *ctx, const BatchDev &b, const OutDev &o, int mode,
                          cudaStream_t st) {
    if (b.n_par == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (b.n_par * 32 + threads - 1) / threads;
    switch (mode) {
        case MODE_BANDFLUX: k_direct<MODE_BANDFLUX><<<(unsigned)blocks, threads, 0, st>>>(ctx->mp, b, o); break;
        case MODE_CHI2: k_direct<MODE_CHI2><<<(unsigned)blocks, threads, 0, st>>>(ctx->mp, b, o); break;
        default: k_direct<MODE_GRAD><<<(unsigned)blocks, threads, 0, st>>>(ctx->mp, b, o); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_validate(const salt_ctx *ctx, const BatchDev &b, int *flag, cudaStream_t st) {
    const int64_t n = b.n_obs > b.n_par ? b.n_obs : b.n_par;
    int blocks = (int)((n + 255) / 256);
    if (blocks > ctx->num_sms * 8) blocks = ctx->num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_validate<<<blocks, 256, 0, st>>>(ctx->mp.bands.n_bands, b, flag);
    return cudaGetLastError();
}

}  // namespace salt
