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

// 2^x by the special-function unit (PTX ex2.approx.ftz.f32, relative error
// about 2^-22 over the normal range). The colour factors 10^(-0.4 c CL) it
// serves are far from the denormal range, where exp2f's extra scaling steps
// would matter.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One band sample's contribution to the column response: its first tap column
// and the 4 weighted taps w_k C_k psi_m(lambda'_k) (rest wavelength a lambda_k).
__device__ __forceinline__ void ebuild_point(const ModelParams &m, const float *lam, const float *wk, int k, float a,
                                             float c, int &first, float (&v)[4]) {
    const float lr = lam[k] * a;
    int iv;
    float t, iw;
    wave_find(m, lr, iv, t, iw);
    Taps4 tl;
    axis_taps_from<false>(iv, t, m.n_wave, iw, tl);
    float dcl;
    const float cl = colour_law(m, lr, dcl);
    const float A = wk[k] * ex2_approx(kColour * c * cl);
    first = tl.first;
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = A * tl.w[q];
}

// ---- Two band samples at once through the packed FP32 instructions
// (fma/mul/add .f32x2): each half is the IEEE operation of the scalar code,
// in the same order, so the values are those of one band sample at a time.

// colour_law on both halves (value; with DERIV also dCL/dlambda).
template <bool DERIV>
__device__ __forceinline__ float2 colour_law2(const ModelParams &m, float2 lam, float2 &dcl) {
    const float2 x = __fmul2_rn(__fadd2_rn(lam, f2(-m.cl_lamB)), f2(m.cl_inv_span));
    const float *p = m.cl_p;
    const float2 Pin = __fmul2_rn(
        x, __ffma2_rn(x, __ffma2_rn(x, __ffma2_rn(x, __ffma2_rn(x, f2(p[4]), f2(p[3])), f2(p[2])), f2(p[1])),
                      f2(p[0])));
    const float2 Plo = __ffma2_rn(f2(m.cl_dPlo), __fadd2_rn(x, f2(-m.cl_xlo)), f2(m.cl_Plo));
    const float2 Phi = __ffma2_rn(f2(m.cl_dPhi), __fadd2_rn(x, f2(-m.cl_xhi)), f2(m.cl_Phi));
    const bool la = lam.x < m.cl_lo, lb = lam.y < m.cl_lo, ha = lam.x > m.cl_hi, hb = lam.y > m.cl_hi;
    if (DERIV) {
        const float2 dPin = __ffma2_rn(
            x, __ffma2_rn(x, __ffma2_rn(x, __ffma2_rn(x, f2(5.f * p[4]), f2(4.f * p[3])), f2(3.f * p[2])),
                          f2(2.f * p[1])),
            f2(p[0]));
        const float2 dP = make_float2(la ? m.cl_dPlo : (ha ? m.cl_dPhi : dPin.x),
                                      lb ? m.cl_dPlo : (hb ? m.cl_dPhi : dPin.y));
        dcl = __fmul2_rn(dP, f2(-m.cl_inv_span));
    }
    return make_float2(-(la ? Plo.x : (ha ? Phi.x : Pin.x)), -(lb ? Plo.y : (hb ? Phi.y : Pin.y)));
}

// Interval and fraction of both halves on the uniform wavelength axis
// (in-grid wavelengths: the arithmetic of axis_locate).
__device__ __forceinline__ float2 wave_locate2(const ModelParams &m, float2 lr, int &ia, int &ib) {
    const float2 u = __fmul2_rn(__fadd2_rn(lr, f2(-m.wave0)), f2(m.inv_dwave));
    ia = min(max(__float2int_rd(u.x), 0), m.n_wave - 2);
    ib = min(max(__float2int_rd(u.y), 0), m.n_wave - 2);
    return __fadd2_rn(u, make_float2(-(float)ia, -(float)ib));
}

// ebuild_point for two in-grid band samples (uniform wavelength axis), kc =
// kColour * c: first tap columns fa, fb and the weighted taps, halves (a, b).
__device__ __forceinline__ void ebuild_point2(const ModelParams &m, float2 lamk, float2 wkk, float a, float kc,
                                              int &fa, int &fb, float2 (&v)[4]) {
    const int NW = m.n_wave;
    const float2 lr = __fmul2_rn(lamk, f2(a));
    int ia, ib;
    const float2 t = wave_locate2(m, lr, ia, ib);
    float2 w[4], dw_[4];
    axis_taps_from2<false>(ia, ib, t, NW, f2(0.f), fa, fb, w, dw_);
    float2 dcl_;
    const float2 cl = colour_law2<false>(m, lr, dcl_);
    const float2 arg = __fmul2_rn(f2(kc), cl);
    const float2 A = __fmul2_rn(wkk, make_float2(ex2_approx(arg.x), ex2_approx(arg.y)));
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = __fmul2_rn(A, w[q]);
}

// The column-response build of ebuild with two consecutive band samples per
// lane (k = k0 + 2 lane and k0 + 2 lane + 1, chunks of 64 strided by
// `stride`, k0 even, so each lane reads its two band samples with one 8-byte
// load: every band starts on an even index of the padded tables; samples below
// k_lo or above kl are inactive): a lane whose two samples share their first
// tap column adds them locally; a lane whose pair straddles two columns hands
// its first sample to the previous lane when that lane's run has the same
// first column (the run then ends there), and otherwise writes it alone after
// the main pass. The segmented scan and the column writes then run once per 64
// band samples. Columns `estride` apart from e0 (column cc).
// FULL: the chunk [cc, cc + W) holds every column the band samples touch (a
// single chunk), so the column checks are left out.
template <bool FULL = false>
__device__ __forceinline__ void ebuild_pair(const ModelParams &m, const float *lam, const float *wk, int k_lo, int kl,
                                            int k_begin, int stride, float a, float c, int cc, int W, int lane,
                                            float *e0, int estride) {
    for (int k0 = k_begin; k0 <= kl; k0 += stride) {
        const int ka = k0 + 2 * lane, kb = ka + 1;
        const bool acta = ka >= k_lo && ka <= kl, actb = kb >= k_lo && kb <= kl;
        int fa = 0x40000000 + 2 * lane, fb = fa + 1;  // inactive: keys of their own, never written
        float va[4] = {0.f, 0.f, 0.f, 0.f}, vb[4] = {0.f, 0.f, 0.f, 0.f};
        if (m.wnode) {  // node axis: binary searches, one band sample at a time
            if (acta) ebuild_point(m, lam, wk, ka, a, c, fa, va);
            if (actb) ebuild_point(m, lam, wk, kb, a, c, fb, vb);
        } else if (acta || actb) {
            // (ka, ka + 1) lie inside the band's padded run of samples
            const float2 l2 = *reinterpret_cast<const float2 *>(lam + ka);
            const float2 w2 = *reinterpret_cast<const float2 *>(wk + ka);
            int f0, f1;
            float2 v2[4];
            ebuild_point2(m, l2, w2, a, kColour * c, f0, f1, v2);
            if (acta) {
                fa = f0;
#pragma unroll
                for (int q = 0; q < 4; ++q) va[q] = v2[q].x;
            }
            if (actb) {
                fb = f1;
#pragma unroll
                for (int q = 0; q < 4; ++q) vb[q] = v2[q].y;
            }
        }
        const bool split = acta && actb && fa != fb;
        const int key = actb ? fb : fa;
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (acta && actb && !split) ? va[q] + vb[q] : (actb ? vb[q] : va[q]);
        // a straddling pair's first sample joins the previous lane's run when
        // that run has its first column
        const int prevkey = __shfl_up_sync(0xffffffffu, key, 1);
        const bool give = split && lane > 0 && prevkey == fa;
        const bool alone = split && !give;
        const bool take = __shfl_down_sync(0xffffffffu, (int)give, 1) != 0 && lane < 31;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float y = __shfl_down_sync(0xffffffffu, va[q], 1);
            if (take) v[q] += y;
        }
        const bool act = acta || actb;
        const int fprev = __shfl_up_sync(0xffffffffu, key, 1);
        const int fnext = __shfl_down_sync(0xffffffffu, key, 1);
        const bool head = lane == 0 || fprev != key;
        const bool tail = lane == 31 || fnext != key;
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const int runlen = __reduce_max_sync(0xffffffffu, (unsigned)(lane - start + 1));
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
            const int col = key + q;
            if (act && tail && (FULL || (col >= cc && col < cc + W))) e0[(col - cc) * estride] += v[q];
            __syncwarp();
        }
        // first samples that stand alone (a run of one band sample, or the
        // chunk's first lane continuing the previous chunk's run)
        if (__any_sync(0xffffffffu, alone)) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int col = fa + q;
                if (alone && (FULL || (col >= cc && col < cc + W))) e0[(col - cc) * estride] += va[q];
                __syncwarp();
            }
        }
    }
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
            const float A = wk[k] * ex2_approx(kColour * c * cl);
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
// column cc of E, E_c, E_z, columns `estride` apart in E and `estride12`
// apart in E_c and E_z (the same as in E when estride12 is 0).
__device__ __forceinline__ void ebuild3(const ModelParams &m, const float *lam, const float *wk, int kl, int k_begin,
                                        int stride, float a, float c, int cc, int W, int lane, float *e0, float *e1,
                                        float *e2, int estride, int estride12 = 0) {
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
            const float A = wk[k] * ex2_approx(kColour * c * cl);
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
                const int ci12 = estride12 ? (col - cc) * estride12 : ci;
                e0[ci] += v[0][q];
                e1[ci12] += v[1][q];
                e2[ci12] += v[2][q];
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
        // Q interpolated at lambda'_k and its slope: on an interior interval the
        // Keys a = -1/2 (Catmull-Rom) cubic through Q at nodes iv-1 .. iv+2,
        //   Q1 + t (Q2 - Q0)/2 + t^2 (Q0 - 5/2 Q1 + 2 Q2 - Q3/2)
        //      + t^3 ((Q3 - Q0)/2 + 3/2 (Q1 - Q2)),
        // on the first / last interval the straight line through its two nodes
        const int first = first_tap(iv, NW);
        float qv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int col = first + q - cc;
            qv[q] = (col >= 0 && col < W) ? Q[col * qstride] : 0.f;
        }
        const bool lo = iv == 0, hi = iv == NW - 2;
        float c0, c1, c2, c3;
        if (lo || hi) {
            const float p0 = lo ? qv[0] : qv[2], p1 = lo ? qv[1] : qv[3];
            c0 = p0;
            c1 = p1 - p0;
            c2 = 0.f;
            c3 = 0.f;
        } else {
            c0 = qv[1];
            c1 = 0.5f * (qv[2] - qv[0]);
            c2 = fmaf(-0.5f, qv[3], fmaf(2.0f, qv[2], fmaf(-2.5f, qv[1], qv[0])));
            c3 = fmaf(0.5f, qv[3] - qv[0], 1.5f * (qv[1] - qv[2]));
        }
        const float qs = fmaf(fmaf(fmaf(c3, t, c2), t, c1), t, c0);
        const float qd = fmaf(fmaf(3.0f * c3, t, 2.0f * c2), t, c1) * iw;
        float dcl;
        const float cl = colour_law(m, lr, dcl);
        const float A = wk[k] * ex2_approx(kColour * c * cl);
        const float Zs = -A * lr * a;  // d lambda'/dz = -lambda' a
        gc = fmaf(A * (kColourLn * cl), qs, gc);
        gz = fmaf(Zs, fmaf(kColourLn * c * dcl, qs, qd), gz);
    }
}

// eadjoint with two band samples per lane, k and k + 32 of chunks of 64
// strided by `stride`, through the packed FP32 instructions on the uniform
// wavelength axis; each lane adds k's terms, then k + 32's, so with one warp
// per sample (stride 64) the lane sums are those of eadjoint with stride 32.
template <bool FULL = false>
__device__ __forceinline__ void eadjoint_pair(const ModelParams &m, const float *lam, const float *wk, int kl,
                                              int k_begin, int stride, float a, float c, int cc, int W, int lane,
                                              const float *Q, int qstride, float &gc, float &gz) {
    if (m.wnode) {  // node axis: one band sample at a time
        for (int k0 = k_begin; k0 <= kl; k0 += stride) {
            eadjoint(m, lam, wk, min(kl, k0 + 31), k0, 64, a, c, cc, W, lane, Q, qstride, gc, gz);
            eadjoint(m, lam, wk, min(kl, k0 + 63), k0 + 32, 64, a, c, cc, W, lane, Q, qstride, gc, gz);
        }
        return;
    }
    const int NW = m.n_wave;
    const float kc = kColour * c, kcl = kColourLn * c;
    for (int k0 = k_begin; k0 <= kl; k0 += stride) {
        const int ka = k0 + lane, kb = ka + 32;
        if (ka > kl) continue;
        const bool actb = kb <= kl;
        const int kb2 = actb ? kb : ka;
        const float2 lr = __fmul2_rn(make_float2(lam[ka], lam[kb2]), f2(a));
        int ia, ib;
        const float2 t = wave_locate2(m, lr, ia, ib);
        const int fa = first_tap(ia, NW), fb = first_tap(ib, NW);
        float2 qv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ca = fa + q - cc, cb = fb + q - cc;
            qv[q] = FULL ? make_float2(Q[ca * qstride], Q[cb * qstride])
                         : make_float2((ca >= 0 && ca < W) ? Q[ca * qstride] : 0.f,
                                       (cb >= 0 && cb < W) ? Q[cb * qstride] : 0.f);
        }
        // Catmull-Rom coefficients (interior) or the straight line (edge interval), per half
        float2 c0 = qv[1];
        float2 c1 = __fmul2_rn(f2(0.5f), __fadd2_rn(qv[2], make_float2(-qv[0].x, -qv[0].y)));
        float2 c2 = __ffma2_rn(f2(-0.5f), qv[3], __ffma2_rn(f2(2.0f), qv[2], __ffma2_rn(f2(-2.5f), qv[1], qv[0])));
        float2 c3 = __ffma2_rn(f2(0.5f), __fadd2_rn(qv[3], make_float2(-qv[0].x, -qv[0].y)),
                               __fmul2_rn(f2(1.5f), __fadd2_rn(qv[1], make_float2(-qv[2].x, -qv[2].y))));
        const bool loa = ia == 0, hia = ia == NW - 2, lob = ib == 0, hib = ib == NW - 2;
        if (loa || hia) {
            const float p0 = loa ? qv[0].x : qv[2].x, p1 = loa ? qv[1].x : qv[3].x;
            c0.x = p0; c1.x = p1 - p0; c2.x = 0.f; c3.x = 0.f;
        }
        if (lob || hib) {
            const float p0 = lob ? qv[0].y : qv[2].y, p1 = lob ? qv[1].y : qv[3].y;
            c0.y = p0; c1.y = p1 - p0; c2.y = 0.f; c3.y = 0.f;
        }
        const float2 qs = __ffma2_rn(__ffma2_rn(__ffma2_rn(c3, t, c2), t, c1), t, c0);
        const float2 iw = f2(m.inv_dwave);
        const float2 qd =
            __fmul2_rn(__ffma2_rn(__ffma2_rn(__fmul2_rn(f2(3.0f), c3), t, __fmul2_rn(f2(2.0f), c2)), t, c1), iw);
        float2 dcl;
        const float2 cl = colour_law2<true>(m, lr, dcl);
        const float2 arg = __fmul2_rn(f2(kc), cl);
        const float2 A = __fmul2_rn(make_float2(wk[ka], wk[kb2]), make_float2(ex2_approx(arg.x), ex2_approx(arg.y)));
        const float2 Zs = __fmul2_rn(__fmul2_rn(make_float2(-A.x, -A.y), lr), f2(a));
        const float2 Ac = __fmul2_rn(A, __fmul2_rn(f2(kColourLn), cl));
        const float2 Zt = __ffma2_rn(__fmul2_rn(f2(kcl), dcl), qs, qd);
        gc = fmaf(Ac.x, qs.x, gc);
        gz = fmaf(Zs.x, Zt.x, gz);
        if (actb) {
            gc = fmaf(Ac.y, qs.y, gc);
            gz = fmaf(Zs.y, Zt.y, gz);
        }
    }
}

}  // namespace fk
}  // namespace salt
