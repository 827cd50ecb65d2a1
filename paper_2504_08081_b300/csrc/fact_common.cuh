// Device helpers shared by the factorised kernels (column-response build).
#pragma once

#include "device_math.cuh"

namespace salt {
namespace fk {

constexpr int FSPAN = 64;  // first-lane table span per 32-sample chunk

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__device__ __forceinline__ float qnanf() { return __int_as_float(0x7fc00000); }

__device__ __forceinline__ int first_tap(int iv, int n) {
    return iv == 0 ? 0 : (iv == n - 2 ? n - 4 : iv - 1);
}

// Column-response build for one sample over band samples [kf, kl], columns
// [cc, cc + W) of the current chunk, by one warp (chunks of 32 band samples
// strided by `stride`). Per band sample k (one per lane): rest wavelength,
// Keys taps, colour law, colour factor and trapezoid weight. Band sample k
// contributes to columns first_k .. first_k + 3 and first_k is nondecreasing
// in k, so for each tap the lanes sharing a column form contiguous runs: a
// segmented inclusive scan (shuffles, fixed tree, as many steps as the
// longest run needs) sums each run and its last lane adds the total to the
// column. e0 points at column cc, columns `estride` apart.
__device__ __forceinline__ void ebuild(const ModelParams &m, const float *lam, const float *wk, int kl, int k_begin,
                                       int stride, float a, float c, int cc, int W, int lane, float *e0,
                                       int estride) {
    const int NW = m.n_wave;
    for (int k0 = k_begin; k0 <= kl; k0 += stride) {
        const int k = k0 + lane;
        const bool act = k <= kl;
        int first = 0x40000000 + lane;  // inactive lanes: a run of their own, never written
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (act) {
            const float lr = lam[k] * a;
            int iv;
            float t;
            float iw;
            wave_find(m, lr, iv, t, iw);
            Taps4 tl;
            axis_taps_from<false>(iv, t, NW, iw, tl);
            float dcl;
            const float cl = colour_law(m, lr, dcl);
            const float A = wk[k] * exp2f(kColour * c * cl);
            first = tl.first;
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = A * tl.w[q];
        }
        const int fprev = __shfl_up_sync(0xffffffffu, first, 1);
        const int fnext = __shfl_down_sync(0xffffffffu, first, 1);
        const bool head = lane == 0 || fprev != first;
        const bool tail = lane == 31 || fnext != first;
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of my run
        const int runlen = __reduce_max_sync(0xffffffffu, (unsigned)(lane - start + 1));
        // segmented sums over each run sharing `first`, the 4 tap columns in the
        // same shuffle rounds (same additions, in the same order, as one at a time)
        for (int d = 1; d < runlen; d <<= 1) {
            float y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) y[q] = __shfl_up_sync(0xffffffffu, v[q], d);
            if (lane - d >= start)
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] += y[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int col = first + q;
            if (act && tail && col >= cc && col < cc + W) e0[(col - cc) * estride] += v[q];
            __syncwarp();
        }
    }
}

// Forward-mode column responses for one sample: E as ebuild, plus
//   E_c[col] = sum_k dA_k/dc psi_col(t_k)                          (d E / d c)
//   E_z[col] = sum_k dlambda'_k/dz (A_k psi'_col + dA_k/dlambda' psi_col)   (d E / d z through lambda')
// (A_k = w_k C_k), built with the same segmented scan. e0/e1/e2 point at
// column cc of E, E_c, E_z, columns `estride` apart.
__device__ __forceinline__ void ebuild3(const ModelParams &m, const float *lam, const float *wk, int kl, int k_begin,
                                        int stride, float a, float c, int cc, int W, int lane, float *e0, float *e1,
                                        float *e2, int estride) {
    const int NW = m.n_wave;
    for (int k0 = k_begin; k0 <= kl; k0 += stride) {
        const int k = k0 + lane;
        const bool act = k <= kl;
        int first = 0x40000000 + lane;
        float v[3][4];
#pragma unroll
        for (int e = 0; e < 3; ++e)
#pragma unroll
            for (int q = 0; q < 4; ++q) v[e][q] = 0.f;
        if (act) {
            const float lr = lam[k] * a;
            int iv;
            float t;
            float iw;
            wave_find(m, lr, iv, t, iw);
            Taps4 tl;
            axis_taps_from<true>(iv, t, NW, iw, tl);
            float dcl;
            const float cl = colour_law(m, lr, dcl);
            const float A = wk[k] * exp2f(kColour * c * cl);
            const float Ac = A * (kColourLn * cl);
            const float Zs = -A * lr * a;
            const float Zv = Zs * (kColourLn * c * dcl);
            first = tl.first;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[0][q] = A * tl.w[q];
                v[1][q] = Ac * tl.w[q];
                v[2][q] = fmaf(Zs, tl.dw[q], Zv * tl.w[q]);
            }
        }
        const int fprev = __shfl_up_sync(0xffffffffu, first, 1);
        const int fnext = __shfl_down_sync(0xffffffffu, first, 1);
        const bool head = lane == 0 || fprev != first;
        const bool tail = lane == 31 || fnext != first;
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const int runlen = __reduce_max_sync(0xffffffffu, (unsigned)(lane - start + 1));
        // segmented sums over each run of band samples sharing `first`: the runs
        // are the same for all 4 tap columns, so the 12 values share each shuffle
        // round (same additions, in the same order, as one column at a time)
        for (int d = 1; d < runlen; d <<= 1) {
            float y[3][4];
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int q = 0; q < 4; ++q) y[e][q] = __shfl_up_sync(0xffffffffu, v[e][q], d);
            if (lane - d >= start)
#pragma unroll
                for (int e = 0; e < 3; ++e)
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[e][q] += y[e][q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int col = first + q;
            if (act && tail && col >= cc && col < cc + W) {
                const int ci = (col - cc) * estride;
                e0[ci] += v[0][q];
                e1[ci] += v[1][q];
                e2[ci] += v[2][q];
            }
            __syncwarp();
        }
    }
}

// Adjoint of the column response for one sample. With Q[col] = dchi2/dE[col]
// (the adjoint rows back-projected through the grid) on columns [cc, cc + W),
// accumulate over band samples [k_begin.., kl] (stride `stride`)
//   gc += sum_k dA_k/dc        sum_m psi_m(t_k)  Q[first_k + m],
//   gz += sum_k [ dlambda'_k/dz A_k sum_m dpsi_m/dlambda' Q + dA_k/dz|lambda' sum_m psi_m Q ],
// i.e. dchi2/dc and the rest-wavelength part of dchi2/dz (A_k = w_k C_k).
// Lane partials; the caller reduces them.
__device__ __forceinline__ void eadjoint(const ModelParams &m, const float *lam, const float *wk, int kl, int k_begin,
                                         int stride, float a, float c, int cc, int W, int lane, const float *Q,
                                         int qstride, float &gc, float &gz) {
    const int NW = m.n_wave;
    for (int k0 = k_begin; k0 <= kl; k0 += stride) {
        const int k = k0 + lane;
        if (k > kl) continue;
        const float lr = lam[k] * a;
        int iv;
        float t;
        float iw;
            wave_find(m, lr, iv, t, iw);
        Taps4 tl;
        axis_taps_from<true>(iv, t, NW, iw, tl);
        float dcl;
        const float cl = colour_law(m, lr, dcl);
        const float A = wk[k] * exp2f(kColour * c * cl);
        float qs = 0.f, qd = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int col = tl.first + q - cc;
            const float qv = (col >= 0 && col < W) ? Q[col * qstride] : 0.f;
            qs = fmaf(tl.w[q], qv, qs);
            qd = fmaf(tl.dw[q], qv, qd);
        }
        const float Zs = -A * lr * a;  // d lambda'/dz = -lambda' a
        gc = fmaf(A * (kColourLn * cl), qs, gc);
        gz = fmaf(Zs, fmaf(kColourLn * c * dcl, qs, qd), gz);
    }
}

}  // namespace fk
}  // namespace salt
