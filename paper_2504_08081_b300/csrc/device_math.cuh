// Per-element device arithmetic of the SALT photometry path (FP32).
#pragma once

#include <cuda_runtime.h>

#include "salt_internal.cuh"

namespace salt {

// Tap set of one interpolation axis: 4 consecutive nodes starting at `first`
// (first in [0, n-4]), their weights and the weights' derivatives with respect
// to the axis coordinate. Keys cubic convolution (a = -1/2) on interior
// intervals; on the first / last interval the two end nodes carry the linear
// weights and the other two carry 0; outside the axis every weight is 0.
struct Taps4 {
    int first;
    float w[4];
    float dw[4];
};

// Keys a = -1/2 weights of nodes (i-1, i, i+1, i+2) at fraction t of interval i,
// expanded as polynomials in t (value and d/dt).
__device__ __forceinline__ void keys_weights(float t, float w[4]) {
    float t2 = t * t;
    w[0] = t * fmaf(t, fmaf(-0.5f, t, 1.0f), -0.5f);
    w[1] = fmaf(t2, fmaf(1.5f, t, -2.5f), 1.0f);
    w[2] = t * fmaf(t, fmaf(-1.5f, t, 2.0f), 0.5f);
    w[3] = t2 * fmaf(0.5f, t, -0.5f);
}

__device__ __forceinline__ void keys_dweights(float t, float d[4]) {
    d[0] = fmaf(t, fmaf(-1.5f, t, 2.0f), -0.5f);
    d[1] = t * fmaf(4.5f, t, -5.0f);
    d[2] = fmaf(t, fmaf(-4.5f, t, 4.0f), 0.5f);
    d[3] = t * fmaf(1.5f, t, -1.0f);
}

// Interval index and fraction of coordinate x on a uniform axis of n >= 4
// nodes. Returns false outside [x0, xmax].
__device__ __forceinline__ bool axis_locate(float x, float x0, float inv_dx, float xmax, int n,
                                            int &i, float &t) {
    if (!(x >= x0 && x <= xmax)) return false;
    float u = (x - x0) * inv_dx;
    i = __float2int_rd(u);
    i = min(max(i, 0), n - 2);
    t = u - (float)i;
    return true;
}

// Interval i, fraction t and the interval's inverse width iw (for the
// derivatives) of x on a model axis: the uniform axis when node is NULL (the
// arithmetic of axis_locate), else by binary search over the ascending node
// positions, t being the fraction of the local interval (the index-space
// reading of the Keys kernel on a non-uniform axis). False outside the axis.
__device__ __forceinline__ bool axis_find(float x, float x0, float inv_dx, float xmax, int n, const float *node,
                                          const float *inv, int &i, float &t, float &iw) {
    if (!node) {
        iw = inv_dx;
        return axis_locate(x, x0, inv_dx, xmax, n, i, t);
    }
    if (!(x >= x0 && x <= xmax)) return false;
    int lo = 0, hi = n - 1;  // node[lo] <= x <= node[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(node + mid) <= x) lo = mid; else hi = mid;
    }
    i = lo;
    iw = __ldg(inv + lo);
    t = fminf((x - __ldg(node + lo)) * iw, 1.0f);
    return true;
}

// Weights (and optionally derivatives w.r.t. x) for a located interval.
// Written with selects only (no runtime index into the tap arrays), so the
// taps stay in registers.
template <bool DERIV>
__device__ __forceinline__ void axis_taps_from(int i, float t, int n, float inv_dx, Taps4 &tp) {
    tp.first = i - 1;
    keys_weights(t, tp.w);
    if (DERIV) {
        keys_dweights(t, tp.dw);
#pragma unroll
        for (int q = 0; q < 4; ++q) tp.dw[q] *= inv_dx;
    }
    if (i == 0 || i == n - 2) {  // first interval: linear weights on nodes 0, 1; last: on n-2, n-1
        const bool lo = i == 0;
        const float l0 = 1.0f - t;
        tp.first = lo ? 0 : n - 4;
        tp.w[0] = lo ? l0 : 0.f;
        tp.w[1] = lo ? t : 0.f;
        tp.w[2] = lo ? 0.f : l0;
        tp.w[3] = lo ? 0.f : t;
        if (DERIV) {
            tp.dw[0] = lo ? -inv_dx : 0.f;
            tp.dw[1] = lo ? inv_dx : 0.f;
            tp.dw[2] = lo ? 0.f : -inv_dx;
            tp.dw[3] = lo ? 0.f : inv_dx;
        }
    }
}

template <bool DERIV>
__device__ __forceinline__ void axis_taps(float x, float x0, float inv_dx, float xmax, int n,
                                          Taps4 &tp) {
    int i;
    float t;
    if (!axis_locate(x, x0, inv_dx, xmax, n, i, t)) {
        tp.first = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) { tp.w[m] = 0.f; if (DERIV) tp.dw[m] = 0.f; }
        return;
    }
    axis_taps_from<DERIV>(i, t, n, inv_dx, tp);
}

// ---- Packed FP32 (fma/mul/add .f32x2) forms of the tap arithmetic: two
// coordinates at once, each half the IEEE operation of the scalar code.

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
// a - b, exactly rounded as the scalar subtraction
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }

// keys_weights on both halves.
__device__ __forceinline__ void keys_weights2(float2 t, float2 (&w)[4]) {
    const float2 t2 = __fmul2_rn(t, t);
    w[0] = __fmul2_rn(t, __ffma2_rn(t, __ffma2_rn(f2(-0.5f), t, f2(1.0f)), f2(-0.5f)));
    w[1] = __ffma2_rn(t2, __ffma2_rn(f2(1.5f), t, f2(-2.5f)), f2(1.0f));
    w[2] = __fmul2_rn(t, __ffma2_rn(t, __ffma2_rn(f2(-1.5f), t, f2(2.0f)), f2(0.5f)));
    w[3] = __fmul2_rn(t2, __ffma2_rn(f2(0.5f), t, f2(-0.5f)));
}

// keys_dweights on both halves.
__device__ __forceinline__ void keys_dweights2(float2 t, float2 (&d)[4]) {
    d[0] = __ffma2_rn(t, __ffma2_rn(f2(-1.5f), t, f2(2.0f)), f2(-0.5f));
    d[1] = __fmul2_rn(t, __ffma2_rn(f2(4.5f), t, f2(-5.0f)));
    d[2] = __ffma2_rn(t, __ffma2_rn(f2(-4.5f), t, f2(4.0f)), f2(0.5f));
    d[3] = __fmul2_rn(t, __ffma2_rn(f2(1.5f), t, f2(-1.0f)));
}

// Taps of two located intervals (ia, t.x) and (ib, t.y) on an axis of n
// nodes, inverse widths iw: axis_taps_from on each half.
template <bool DERIV>
__device__ __forceinline__ void axis_taps_from2(int ia, int ib, float2 t, int n, float2 iw, int &fa, int &fb,
                                                float2 (&w)[4], float2 (&dw)[4]) {
    fa = ia - 1;
    fb = ib - 1;
    keys_weights2(t, w);
    if (DERIV) {
        keys_dweights2(t, dw);
#pragma unroll
        for (int q = 0; q < 4; ++q) dw[q] = __fmul2_rn(dw[q], iw);
    }
    const bool ea = ia == 0 || ia == n - 2, eb = ib == 0 || ib == n - 2;
    if (ea || eb) {  // first / last interval: linear weights on its two nodes
        const float2 l0 = fsub2(f2(1.0f), t);
        if (ea) {
            const bool lo = ia == 0;
            fa = lo ? 0 : n - 4;
            w[0].x = lo ? l0.x : 0.f; w[1].x = lo ? t.x : 0.f; w[2].x = lo ? 0.f : l0.x; w[3].x = lo ? 0.f : t.x;
            if (DERIV) {
                dw[0].x = lo ? -iw.x : 0.f; dw[1].x = lo ? iw.x : 0.f;
                dw[2].x = lo ? 0.f : -iw.x; dw[3].x = lo ? 0.f : iw.x;
            }
        }
        if (eb) {
            const bool lo = ib == 0;
            fb = lo ? 0 : n - 4;
            w[0].y = lo ? l0.y : 0.f; w[1].y = lo ? t.y : 0.f; w[2].y = lo ? 0.f : l0.y; w[3].y = lo ? 0.f : t.y;
            if (DERIV) {
                dw[0].y = lo ? -iw.y : 0.f; dw[1].y = lo ? iw.y : 0.f;
                dw[2].y = lo ? 0.f : -iw.y; dw[3].y = lo ? 0.f : iw.y;
            }
        }
    }
}

// ---- The phase coordinate as a float pair.
// The rest-frame phase (mjd - t0) / (1 + z) is a difference of epochs ~5e4 d
// apart by tens of days. Formed in FP32, the phase (or its grid coordinate
// near the end of a 70-node axis) carries ~4e-6 d of rounding, which the steep
// ends of a surface turn into ~1e-5 of bandflux. So the observation time is
// held as a float pair (hi + lo = mjd to ~1e-10 d), each sample has an origin
// O and a scale S (FP64 per sample, stored as float pairs) with
// u = (mjd - O) S, and u is formed as a float pair by error-free
// transformations (Knuth's two-sum, the FMA product error): FP32 arithmetic
// throughout, no FP64 per (observation, sample) pair. On a uniform axis u is
// the grid coordinate (O = t0 + phase0 (1 + z), S = 1 / ((1 + z) dphase));
// on a node axis it is the phase itself (O = t0, S = 1 / (1 + z)).

// x as hi + lo, hi = x rounded to FP32.
__device__ __forceinline__ float2 split_f2(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// Per-sample phase map (O hi, O lo, S hi, S lo); a = 1 / (1 + z) rounded once.
__device__ __forceinline__ float4 phase_map(const ModelParams &m, float z, double t0, float &a) {
    const double zp1 = 1.0 + (double)z;
    const double ad = 1.0 / zp1;
    a = __double2float_rn(ad);
    double o = t0, s = ad;
    if (!m.pnode) { o = fma(m.phase0_d, zp1, t0); s = ad * m.inv_dphase_d; }
    const float2 O = split_f2(o), S = split_f2(s);
    return make_float4(O.x, O.y, S.x, S.y);
}

// u = (tm - O) S as a normalised float pair (x + y, |y| <= ulp(x) / 2 when
// |u| is not tiny). The _rn intrinsics keep the compiler from fusing the
// products into the sums the error terms are taken from.
__device__ __forceinline__ float2 phase_u(float2 tm, float4 pm) {
    const float dh = __fadd_rn(tm.x, -pm.x);                // two-sum of tm.x and -O.x
    const float bv = __fadd_rn(dh, -tm.x);
    const float de = __fadd_rn(__fadd_rn(tm.x, -__fadd_rn(dh, -bv)), -__fadd_rn(pm.x, bv));
    const float dl = __fadd_rn(de, __fadd_rn(tm.y, -pm.y)); // tm - O = dh + dl
    const float uh = __fmul_rn(dh, pm.z);
    float ue = fmaf(dh, pm.z, -uh);                         // exact error of dh S.hi
    ue = fmaf(dh, pm.w, ue);
    ue = fmaf(dl, pm.z, ue);
    const float s = __fadd_rn(uh, ue);                      // fast two-sum
    return make_float2(s, __fadd_rn(ue, -__fadd_rn(s, -uh)));
}

// Interval i, fraction t and inverse width iw (as axis_find) of the phase of
// observation time tm under the sample's phase map pm, the interval chosen
// and t formed from the float pair; p is the phase in FP32 (for the gradient
// terms). False outside the phase axis.
__device__ __forceinline__ bool phase_find(const ModelParams &m, float2 tm, float4 pm, int &i, float &t, float &iw,
                                           float &p) {
    const float2 u = phase_u(tm, pm);
    if (!m.pnode) {
        const float top = (float)(m.n_phase - 1);
        if (!((u.x > 0.f || (u.x == 0.f && u.y >= 0.f)) && (u.x < top || (u.x == top && u.y <= 0.f))))
            return false;
        i = min(__float2int_rd(u.x), m.n_phase - 2);
        t = __fadd_rn(u.x, -(float)i) + u.y;  // u.x - i is exact
        iw = m.inv_dphase;
        p = fmaf(u.x, m.dphase, m.phase0);
        return true;
    }
    const int n = m.n_phase;
    const float n0 = __ldg(m.pnode), n1 = __ldg(m.pnode + n - 1);
    const float l0 = __ldg(m.pnode_lo), l1 = __ldg(m.pnode_lo + n - 1);
    if (!((u.x > n0 || (u.x == n0 && u.y >= l0)) && (u.x < n1 || (u.x == n1 && u.y <= l1)))) return false;
    int lo = 0, hi = n - 1;  // node[lo] <= u.x <= node[hi] (float parts)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(m.pnode + mid) <= u.x) lo = mid; else hi = mid;
    }
    i = lo;
    iw = __ldg(m.pinv + lo);
    // (u - node) from the pairs: the hi difference is exact or rounded relative
    // to itself (at most one interval)
    t = fminf((__fadd_rn(u.x, -__ldg(m.pnode + lo)) + (u.y - __ldg(m.pnode_lo + lo))) * iw, 1.0f);
    p = u.x;
    return true;
}

// phase_find for two observation times under one phase map: on a uniform
// axis the float-pair arithmetic of phase_u runs on both halves at once; on a
// node axis it is phase_find twice. oka / okb say whether each phase is on
// the axis (ia, ib, t, iw, p are then set for that half).
__device__ __forceinline__ void phase_find2(const ModelParams &m, float2 tma, float2 tmb, float4 pm, bool &oka,
                                            bool &okb, int &ia, int &ib, float2 &t, float2 &iw, float2 &p) {
    if (m.pnode) {
        oka = phase_find(m, tma, pm, ia, t.x, iw.x, p.x);
        okb = phase_find(m, tmb, pm, ib, t.y, iw.y, p.y);
        return;
    }
    const float2 th = make_float2(tma.x, tmb.x), tl = make_float2(tma.y, tmb.y);
    const float2 dh = __fadd2_rn(th, f2(-pm.x));  // two-sum of the hi parts and -O.x
    const float2 bv = fsub2(dh, th);
    const float2 de = fsub2(fsub2(th, fsub2(dh, bv)), __fadd2_rn(f2(pm.x), bv));
    const float2 dl = __fadd2_rn(de, __fadd2_rn(tl, f2(-pm.y)));
    const float2 uh = __fmul2_rn(dh, f2(pm.z));
    float2 ue = __ffma2_rn(dh, f2(pm.z), make_float2(-uh.x, -uh.y));
    ue = __ffma2_rn(dh, f2(pm.w), ue);
    ue = __ffma2_rn(dl, f2(pm.z), ue);
    const float2 s = __fadd2_rn(uh, ue);
    const float2 e = fsub2(ue, fsub2(s, uh));
    const float top = (float)(m.n_phase - 1);
    oka = (s.x > 0.f || (s.x == 0.f && e.x >= 0.f)) && (s.x < top || (s.x == top && e.x <= 0.f));
    okb = (s.y > 0.f || (s.y == 0.f && e.y >= 0.f)) && (s.y < top || (s.y == top && e.y <= 0.f));
    ia = min(max(__float2int_rd(s.x), 0), m.n_phase - 2);
    ib = min(max(__float2int_rd(s.y), 0), m.n_phase - 2);
    t = __fadd2_rn(__fadd2_rn(s, make_float2(-(float)ia, -(float)ib)), e);
    iw = f2(m.inv_dphase);
    p = __ffma2_rn(s, f2(m.dphase), f2(m.phase0));
}

__device__ __forceinline__ bool wave_find(const ModelParams &m, float lam, int &i, float &t, float &iw) {
    return axis_find(lam, m.wave0, m.inv_dwave, m.wave_max, m.n_wave, m.wnode, m.winv, i, t, iw);
}

// Taps on a model axis (all weights zero outside it).
template <bool DERIV>
__device__ __forceinline__ void phase_taps(const ModelParams &m, float2 tm, float4 pm, Taps4 &tp, float &p) {
    int i;
    float t, iw;
    p = 0.f;
    if (!phase_find(m, tm, pm, i, t, iw, p)) {
        tp.first = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) { tp.w[q] = 0.f; if (DERIV) tp.dw[q] = 0.f; }
        return;
    }
    axis_taps_from<DERIV>(i, t, m.n_phase, iw, tp);
}
template <bool DERIV>
__device__ __forceinline__ void wave_taps(const ModelParams &m, float lam, Taps4 &tp) {
    int i;
    float t, iw;
    if (!wave_find(m, lam, i, t, iw)) {
        tp.first = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) { tp.w[q] = 0.f; if (DERIV) tp.dw[q] = 0.f; }
        return;
    }
    axis_taps_from<DERIV>(i, t, m.n_wave, iw, tp);
}

// SALT2-form colour law CL(lambda) and dCL/dlambda (linear outside [cl_lo, cl_hi]).
__device__ __forceinline__ float colour_law(const ModelParams &m, float lam, float &dcl) {
    float x = (lam - m.cl_lamB) * m.cl_inv_span;
    float P, dP;
    if (lam < m.cl_lo) {
        dP = m.cl_dPlo;
        P = fmaf(dP, x - m.cl_xlo, m.cl_Plo);
    } else if (lam > m.cl_hi) {
        dP = m.cl_dPhi;
        P = fmaf(dP, x - m.cl_xhi, m.cl_Phi);
    } else {
        const float *p = m.cl_p;
        P = x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, p[4], p[3]), p[2]), p[1]), p[0]);
        dP = fmaf(x, fmaf(x, fmaf(x, fmaf(x, 5.f * p[4], 4.f * p[3]), 3.f * p[2]), 2.f * p[1]),
                  p[0]);
    }
    dcl = -dP * m.cl_inv_span;
    return -P;
}

// 0.4 * log2(10) split into a float head and tail (Cody-Waite style).
constexpr float kZpHi = 1.3287712335586548f;
constexpr float kZpLo = 4.3962899987093351e-09f;

// 10^(0.4 zp) in FP32 with the exponent argument carried in two parts, so the
// rounding of 0.4*log2(10)*zp (|arg| ~ 37) does not cost ~1e-6 relative.
__device__ __forceinline__ float zp_scale(float zp) {
    float th = zp * kZpHi;
    float te = fmaf(zp, kZpHi, -th) + zp * kZpLo;  // exact product error + tail
    float n = rintf(th);
    float f = (th - n) + te;
    return ldexpf(exp2f(f), (int)n);
}

// -0.4 * log2(10): colour factor 10^(-0.4 c CL) = exp2(kColour * c * CL).
constexpr float kColour = -1.32877123795494492f;
// -0.4 * ln(10): d/dc of log of the colour factor per unit CL.
constexpr float kColourLn = -0.921034037197618f;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace salt

namespace salt {

// Prefetch [p, p + bytes) into L2 with bulk prefetches (TMA engine); only the
// 16-byte aligned interior is requested, so nothing outside the range is touched.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
    uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    while (a < e) {
        const uint32_t n = (uint32_t)((e - a) < (uintptr_t)(1u << 16) ? (e - a) : (uintptr_t)(1u << 16));
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
        a += n;
    }
}

// L2 prefetch of one work item's observation and parameter ranges.
__device__ __forceinline__ void prefetch_item(const BatchDev &b, const WorkItem &w) {
    const int64_t n = w.nobs, s = w.nj;
    prefetch_l2(b.mjd + w.obs0, 8 * n);
    prefetch_l2(b.band + w.obs0, 4 * n);
    prefetch_l2(b.flux + w.obs0, 4 * n);
    prefetch_l2(b.fluxerr + w.obs0, 4 * n);
    prefetch_l2(b.zp + w.obs0, 4 * n);
    prefetch_l2(b.t0 + w.par0, 8 * s);
    prefetch_l2(b.z + w.par0, 4 * s);
    prefetch_l2(b.x0 + w.par0, 4 * s);
    prefetch_l2(b.x1 + w.par0, 4 * s);
    prefetch_l2(b.c + w.par0, 4 * s);
}

}  // namespace salt
