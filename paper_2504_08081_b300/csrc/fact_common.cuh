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
// [cc, cc + W) of the current chunk, by one warp (k-chunks of 32 strided by
// `stride`). Per k: rest wavelength, Keys taps, colour law, colour factor and
// trapezoid weight (staged per lane); then per column the contributions of
// the k whose 4 taps cover it, in increasing k. NEB selects E only (1) or
// E, E_c, E_z (3); WANT0 = false skips E (rebuild of E_c, E_z only).
template <int NEB, bool WANT0>
__device__ __forceinline__ void ebuild(const ModelParams &m, const float *lam, const float *wk, int kf,
                                       int kl, int k_begin, int stride, float a, float c, int cc, int W,
                                       int lane, int *kc, int *F, float *kw, float *e0, float *e1,
                                       float *e2, int estride) {
    constexpr bool GRAD = NEB == 3;
    const int NW = m.n_wave;
    for (int k0 = k_begin; k0 <= kl; k0 += stride) {
        const int nk = min(32, kl - k0 + 1);
        if (lane < nk) {
            const int k = k0 + lane;
            const float lr = lam[k] * a;
            int iv;
            float t;
            axis_locate(lr, m.wave0, m.inv_dwave, m.wave_max, NW, iv, t);
            Taps4 tl;
            axis_taps_from<GRAD>(iv, t, NW, m.inv_dwave, tl);
            float dcl;
            const float cl = colour_law(m, lr, dcl);
            const float C = exp2f(kColour * c * cl);
            const float A = wk[k] * C;
            kc[lane] = tl.first;
            float *kwl = kw + lane * 4 * NEB;
#pragma unroll
            for (int q = 0; q < 4; ++q) kwl[q] = A * tl.w[q];
            if (GRAD) {
                const float Ac = A * (kColourLn * cl);
                const float Zs = -A * lr * a;  // d lambda'/dz = -lambda' a
                const float Zv = Zs * (kColourLn * c * dcl);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    kwl[4 + q] = Ac * tl.w[q];
                    kwl[8 + q] = fmaf(Zs, tl.dw[q], Zv * tl.w[q]);
                }
            }
        }
        __syncwarp();
        const int c0 = kc[0], cl_ = kc[nk - 1];
        const int span = cl_ - c0;
        const bool table = span < FSPAN - 1;
        if (table) {
            // F[c - c0] = first lane whose first column is >= c, for c in [c0, cl_ + 1]
            if (lane < nk) {
                const int prev = lane == 0 ? c0 - 1 : kc[lane - 1];
                for (int cq = prev + 1; cq <= kc[lane]; ++cq) F[cq - c0] = lane;
            }
            if (lane == 0) F[span + 1] = nk;
        }
        __syncwarp();
        for (int col = c0 + lane; col <= cl_ + 3; col += 32) {
            if (col < cc || col >= cc + W) continue;
            int lo, hi;
            if (table) {
                lo = (col - 3 <= c0) ? 0 : F[col - 3 - c0];
                hi = (col + 1 - c0 > span + 1) ? nk : F[col + 1 - c0];
            } else {
                lo = 0; hi = nk;
                while (lo < hi) { const int md = (lo + hi) >> 1; if (kc[md] >= col - 3) hi = md; else lo = md + 1; }
                hi = lo;
                while (hi < nk && kc[hi] <= col) ++hi;
            }
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            for (int q = lo; q < hi; ++q) {
                const int mc = col - kc[q];
                const float *kwq = kw + q * 4 * NEB;
                if (WANT0) s0 += kwq[mc];
                if (GRAD) {
                    s1 += kwq[4 + mc];
                    s2 += kwq[8 + mc];
                }
            }
            const int ci = (col - cc) * estride;
            if (WANT0) e0[ci] += s0;
            if (GRAD) {
                e1[ci] += s1;
                e2[ci] += s2;
            }
        }
        __syncwarp();
    }
}

}  // namespace fk
}  // namespace salt
