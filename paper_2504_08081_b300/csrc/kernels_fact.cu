// Fused factorised kernel: chi^2, its gradient, or the bandfluxes of a ragged
// batch, by a persistent grid that pulls (supernova, sample-range) work items
// from a cost-sorted list.
//
// The bandflux of observation i (band b, phase p) for sample j is
//   B_ij = x0 a zpf_i  sum_r phi_r(p_ij) sum_col (G0 + x1 G1)[r][col] E_jb[col],
//   E_jb[col] = sum_k w_k C_k(c, lambda'_k) psi_col(lambda'_k),   lambda'_k = a lambda_k,
// which is the band integral of Eq. 2 with the model of Eq. 1 reassociated:
// the tensor-product interpolation is linear in the grid values, so the
// wavelength taps, colour factors and trapezoid weights of one (sample, band)
// collapse into one column response E shared by every observation in that band.
// Per (band, sample tile) the kernel
//   1. builds E (and, for the gradient, E_c = dE/dc and E_z = dE/dz through
//      lambda') for the union column window of the tile,
//   2. forms the row dots D[r][j] = sum_col G[r][col] E_j[col] for every phase
//      row touched by an observation (a small GEMM, FP32 FMA),
//   3. finishes each (observation, sample) pair from 4 row dots: bandflux,
//      residual, FP64 chi^2 and the direct gradient terms,
//   4. (gradient) back-projects the adjoint Y[r][j] = sum_i g_ij pre_ij phi_r
//      through the grid, Q_j[col] = sum_r Y[r][j] H_j[r][col], and dots Q with
//      E_c and E_z for dchi2/dc and the lambda' part of dchi2/dz.
// Every sum has a fixed order, so results are bitwise reproducible for a
// given tile size.
#include <cstdio>

#include "device_math.cuh"

namespace salt {
namespace fk {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int OBS_MAX = 1024;  // observations of one supernova staged per pass
constexpr int PCAP = 256;      // (observation x sample) pairs per epilogue sub-chunk
constexpr int WMAX = 256;      // union window columns per column chunk
constexpr int LPR = 4;         // lanes per row in the forward GEMM
constexpr int NPH_MAX = 256;   // phase nodes supported

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

struct Lay {
    size_t ord, zpf, bstart, pj, rowmask, rows, misc, E, Ep, D, Y, pf, pt, pc, kst, red, total;
    __host__ __device__ Lay(int tj, bool grad, int n_phase) {
        const int ne = grad ? 3 : 1;
        const int wps = WARPS / tj;
        size_t o = 0;
        ord = o;     o = al16(o + 4 * OBS_MAX);
        zpf = o;     o = al16(o + 4 * OBS_MAX);
        bstart = o;  o = al16(o + 4 * (2 * SALT_MAX_BANDS + 2));
        pj = o;      o = al16(o + 4 * 16 * tj);  // per-sample scalars (see kernel)
        rowmask = o; o = al16(o + 4 * (NPH_MAX / 32));
        rows = o;    o = al16(o + 4 * NPH_MAX);
        misc = o;    o = al16(o + 4 * 16);
        E = o;       o = al16(o + 4 * (size_t)WMAX * tj * ne);
        Ep = o;      o = al16(o + (wps > 1 ? 4 * (size_t)WARPS * WMAX * ne : 0));
        D = o;       o = al16(o + 4 * (size_t)n_phase * tj * 2);
        Y = o;       o = al16(o + (grad ? 4 * (size_t)n_phase * tj : 0));
        pf = o;      o = al16(o + 4 * (size_t)PCAP);
        pt = o;      o = al16(o + 4 * (size_t)PCAP);
        pc = o;      o = al16(o + (grad ? 4 * (size_t)PCAP : 0));
        kst = o;     o = al16(o + (size_t)WARPS * 32 * 4 * (1 + 4 * ne));
        red = o;     o = al16(o + 8 * (size_t)WARPS * (8 + 2 * tj));
        total = o;
    }
};

// per-sample scalar slots in Lay::pj (float unless noted)
enum { PJ_A = 0, PJ_X0, PJ_X1, PJ_C, PJ_Z, PJ_OK, PJ_KF, PJ_KL, PJ_T0LO, PJ_T0HI, PJ_NUM };

__device__ __forceinline__ float qnanf() { return __int_as_float(0x7fc00000); }

// Keys / linear weight (and derivative in the fraction t) of tap m for the
// interval of type `edge` (0 interior, 1 first, 2 last).
__device__ __forceinline__ void tap_weight(int m, float t, int edge, float &w, float &dw) {
    if (edge == 1) {
        w = (m == 0) ? 1.f - t : (m == 1 ? t : 0.f);
        dw = (m == 0) ? -1.f : (m == 1 ? 1.f : 0.f);
        return;
    }
    if (edge == 2) {
        w = (m == 2) ? 1.f - t : (m == 3 ? t : 0.f);
        dw = (m == 2) ? -1.f : (m == 3 ? 1.f : 0.f);
        return;
    }
    float ww[4], dd[4];
    keys_weights(t, ww);
    keys_dweights(t, dd);
    w = ww[m];
    dw = dd[m];
}

template <int TJ, int MODE>
__global__ void __launch_bounds__(THREADS, 2)
k_fact(ModelParams m, BatchDev b, OutDev o, const WorkItem *__restrict__ items, int n_items,
       int *counter) {
    constexpr bool GRAD = MODE == MODE_GRAD;
    constexpr int NE = GRAD ? 3 : 1;
    constexpr int WPS = WARPS / TJ;  // warps per sample
    extern __shared__ __align__(16) unsigned char smem[];
    const Lay L(TJ, GRAD, m.n_phase);
    int *sOrd = (int *)(smem + L.ord);
    float *sZpf = (float *)(smem + L.zpf);
    int *sBst = (int *)(smem + L.bstart);  // [0..NB] starts, [NB+1..] running positions
    float *sPj = (float *)(smem + L.pj);   // [PJ_NUM][TJ]
    unsigned *sRowMask = (unsigned *)(smem + L.rowmask);
    int *sRows = (int *)(smem + L.rows);
    int *sMisc = (int *)(smem + L.misc);
    float *sE = (float *)(smem + L.E);     // [NE][WMAX][TJ]
    float *sEp = (float *)(smem + L.Ep);   // [NE][WARPS][WMAX] (WPS > 1)
    float *sD = (float *)(smem + L.D);     // [n_phase][TJ][2]
    float *sY = (float *)(smem + L.Y);     // [n_phase][TJ]
    int *sPf = (int *)(smem + L.pf);       // pair: interval index or -1
    float *sPt = (float *)(smem + L.pt);   // pair: fraction
    float *sPc = (float *)(smem + L.pc);   // pair: g * pre (adjoint coefficient)
    int *sKc = (int *)(smem + L.kst);      // [WARPS][32] first column
    float *sKw = (float *)(smem + L.kst + 4 * WARPS * 32);  // [WARPS][32][4*NE]
    double *sRed = (double *)(smem + L.red);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NB = m.bands.n_bands;
    const int NW = m.n_wave;

    for (;;) {
        __syncthreads();
        if (tid == 0) sMisc[0] = atomicAdd(counter, 1);
        __syncthreads();
        const int it = sMisc[0];
        if (it >= n_items) break;
        const WorkItem wi = items[it];
        const int64_t ob0 = wi.obs0;
        const int64_t nobs = wi.nobs;

        for (int jt = 0; jt < wi.nj; jt += TJ) {
            const int nj = min(TJ, wi.nj - jt);
            const int64_t pj0 = wi.par0 + jt;  // global index of tile sample 0
            const int jloc0 = wi.jloc0 + jt;   // local index of tile sample 0

            // ---- per-sample parameters
            __syncthreads();
            if (tid < TJ) {
                const int j = tid;
                float z = 0.f, x0 = 0.f, x1 = 0.f, c = 0.f;
                double t0 = 0.0;
                int ok = 0;
                if (j < nj) {
                    z = b.z[pj0 + j]; x0 = b.x0[pj0 + j]; x1 = b.x1[pj0 + j]; c = b.c[pj0 + j];
                    t0 = b.t0[pj0 + j];
                    ok = isfinite(z) && z > -1.f && isfinite(x0) && isfinite(x1) && isfinite(c) &&
                         isfinite(t0);
                    if (!ok) atomicOr(o.err, ERRBIT_PARAM);
                }
                if (!ok) { z = 0.f; x0 = 0.f; x1 = 0.f; c = 0.f; t0 = 0.0; }
                sPj[PJ_A * TJ + j] = 1.0f / (1.0f + z);
                sPj[PJ_X0 * TJ + j] = x0;
                sPj[PJ_X1 * TJ + j] = x1;
                sPj[PJ_C * TJ + j] = c;
                sPj[PJ_Z * TJ + j] = z;
                sPj[PJ_OK * TJ + j] = (j < nj && ok) ? 1.f : 0.f;
                ((double *)(sPj + PJ_T0LO * TJ))[j] = t0;  // occupies T0LO..T0HI rows
            }
            if (tid == 0) sMisc[2] = 0;  // any invalid observation in this supernova
            // per-thread accumulators, fixed assignment -> deterministic sums
            double chi_acc = 0.0;            // epilogue owner (warp -> sample warp / WPS)
            float gacc[4] = {0.f, 0.f, 0.f, 0.f};  // z(prefactor+phase), t0, x0, x1
            float gc_acc[TJ], gz_acc[TJ];    // reverse GEMM partials, all samples
#pragma unroll
            for (int j = 0; j < TJ; ++j) { gc_acc[j] = 0.f; gz_acc[j] = 0.f; }

            for (int64_t oc = 0; oc < nobs; oc += OBS_MAX) {
                const int nc = (int)min((int64_t)OBS_MAX, nobs - oc);
                const int64_t obase = ob0 + oc;
                // ---- stage zero-point scales, validate, stable counting sort by band
                __syncthreads();
                for (int i = tid; i < 2 * SALT_MAX_BANDS + 2; i += THREADS) sBst[i] = 0;
                __syncthreads();
                for (int i = tid; i < nc; i += THREADS) {
                    const int bd = b.band[obase + i];
                    const float e = b.fluxerr[obase + i];
                    const bool okb = bd >= 0 && bd < NB;
                    if (!okb || !(e > 0.f)) {
                        atomicOr(o.err, okb ? ERRBIT_SIGMA : ERRBIT_BAND);
                        sMisc[2] = 1;
                    }
                    sZpf[i] = zp_scale(b.zp[obase + i]);
                }
                __syncthreads();
                if (warp == 0) {
                    int *cnt = sBst + 1;  // counts at [1..NB]
                    for (int base = 0; base < nc; base += 32) {
                        const int i = base + lane;
                        int bd = -1;
                        if (i < nc) {
                            bd = b.band[obase + i];
                            if (bd < 0 || bd >= NB || !(b.fluxerr[obase + i] > 0.f)) bd = -1;
                        }
                        const unsigned mm = __match_any_sync(0xffffffffu, bd);
                        if (bd >= 0 && lane == __ffs(mm) - 1) cnt[bd] += __popc(mm);
                        __syncwarp();
                    }
                    if (lane == 0) {
                        int acc = 0;
                        for (int q = 0; q <= NB; ++q) {
                            const int v = (q < NB) ? sBst[q + 1] : 0;
                            sBst[q] = acc;
                            sBst[NB + 1 + q] = acc;  // running position
                            acc += v;
                        }
                    }
                    __syncwarp();
                    int *pos = sBst + NB + 1;
                    for (int base = 0; base < nc; base += 32) {
                        const int i = base + lane;
                        int bd = -1;
                        if (i < nc) {
                            bd = b.band[obase + i];
                            if (bd < 0 || bd >= NB || !(b.fluxerr[obase + i] > 0.f)) bd = -1;
                        }
                        const unsigned mm = __match_any_sync(0xffffffffu, bd);
                        const int rank = __popc(mm & ((1u << lane) - 1u));
                        if (bd >= 0) sOrd[pos[bd] + rank] = i;
                        __syncwarp();
                        if (bd >= 0 && lane == __ffs(mm) - 1) pos[bd] += __popc(mm);
                        __syncwarp();
                    }
                }
                __syncthreads();

                for (int bd = 0; bd < NB; ++bd) {
                    const int nb_obs = sBst[bd + 1] - sBst[bd];
                    if (nb_obs == 0) continue;  // uniform: sBst is shared
                    const int* ordb = sOrd + sBst[bd];
                    const int K = m.bands.n[bd], koff = m.bands.off[bd];
                    const float *blam = m.band_lam + koff;
                    const float *bw = m.band_w + koff;

                    // ---- 1. in-grid band-sample range and column window per sample
                    __syncthreads();
                    if (tid == 0) { sMisc[4] = 0x7fffffff; sMisc[5] = -1; sMisc[6] = 0; }
                    for (int q = tid; q < NPH_MAX / 32; q += THREADS) sRowMask[q] = 0u;
                    __syncthreads();
                    if (warp == 0 && lane < nj) {
                        const int j = lane;
                        const float a = sPj[PJ_A * TJ + j];
                        int kf = K, kl = -1;
                        if (sPj[PJ_OK * TJ + j] != 0.f) {
                            // first k with a*lambda_k >= wave0; last with a*lambda_k <= wave_max
                            int lo = 0, hi = K;
                            while (lo < hi) { int md = (lo + hi) >> 1; if (__ldg(blam + md) * a >= m.wave0) hi = md; else lo = md + 1; }
                            kf = lo;
                            lo = 0; hi = K;
                            while (lo < hi) { int md = (lo + hi) >> 1; if (__ldg(blam + md) * a <= m.wave_max) lo = md + 1; else hi = md; }
                            kl = lo - 1;
                        }
                        sPj[PJ_KF * TJ + j] = __int_as_float(kf);
                        sPj[PJ_KL * TJ + j] = __int_as_float(kl);
                        if (kf <= kl) {
                            int iv; float t;
                            Taps4 tp;
                            axis_locate(__ldg(blam + kf) * a, m.wave0, m.inv_dwave, m.wave_max, NW, iv, t);
                            axis_taps_from<false>(iv, t, NW, m.inv_dwave, tp);
                            atomicMin(&sMisc[4], tp.first);
                            axis_locate(__ldg(blam + kl) * a, m.wave0, m.inv_dwave, m.wave_max, NW, iv, t);
                            axis_taps_from<false>(iv, t, NW, m.inv_dwave, tp);
                            atomicMax(&sMisc[5], tp.first + 3);
                        }
                    }
                    // ---- 2. touched phase rows (all obs of the band, all samples)
                    for (int q = tid; q < nb_obs * nj; q += THREADS) {
                        const int il = q / nj, j = q - il * nj;
                        if (sPj[PJ_OK * TJ + j] == 0.f) continue;
                        const int i = ordb[il];
                        const double t0 = ((const double *)(sPj + PJ_T0LO * TJ))[j];
                        const float p = (float)(b.mjd[obase + i] - t0) * sPj[PJ_A * TJ + j];
                        int iv; float t;
                        if (axis_locate(p, m.phase0, m.inv_dphase, m.phase_max, m.n_phase, iv, t)) {
                            const int first = (iv == 0) ? 0 : (iv == m.n_phase - 2 ? m.n_phase - 4 : iv - 1);
#pragma unroll
                            for (int mm = 0; mm < 4; ++mm)
                                atomicOr(&sRowMask[(first + mm) >> 5], 1u << ((first + mm) & 31));
                        }
                    }
                    __syncthreads();
                    if (warp == 0) {
                        int base = 0;
                        for (int wd = 0; wd < (m.n_phase + 31) / 32; ++wd) {
                            const unsigned word = sRowMask[wd];
                            const bool on = (word >> lane) & 1u;
                            const unsigned bal = __ballot_sync(0xffffffffu, on);
                            if (on) sRows[base + __popc(bal & ((1u << lane) - 1u))] = wd * 32 + lane;
                            base += __popc(bal);
                        }
                        if (lane == 0) sMisc[6] = base;
                    }
                    __syncthreads();
                    const int nrows = sMisc[6];
                    const int C_lo = sMisc[4], C_hi = sMisc[5];

                    // zero the row dots of the touched rows
                    for (int q = tid; q < nrows * TJ * 2; q += THREADS) {
                        const int rr = q / (TJ * 2);
                        sD[sRows[rr] * TJ * 2 + (q - rr * TJ * 2)] = 0.f;
                    }
                    const int n_cchunks = (C_hi >= C_lo) ? (C_hi - C_lo + WMAX) / WMAX : 0;

                    // ---- E build + forward GEMM, per column chunk
                    for (int ch = 0; ch < n_cchunks; ++ch) {
                        const int cc = C_lo + ch * WMAX;
                        const int W = min(WMAX, C_hi - cc + 1);
                        const bool want_grad_E = GRAD && n_cchunks == 1;
                        const int ne_now = want_grad_E ? NE : 1;
                        __syncthreads();
                        for (int q = tid; q < ne_now * WMAX * TJ; q += THREADS) sE[q] = 0.f;
                        if (WPS > 1)
                            for (int q = tid; q < ne_now * WARPS * WMAX; q += THREADS) sEp[q] = 0.f;
                        __syncthreads();
                        // warp -> (sample j, k-chunk subset)
                        {
                            const int j = warp / WPS, sub = warp % WPS;
                            if (j < nj && sPj[PJ_OK * TJ + j] != 0.f) {
                                const int kf = __float_as_int(sPj[PJ_KF * TJ + j]);
                                const int kl = __float_as_int(sPj[PJ_KL * TJ + j]);
                                const float a = sPj[PJ_A * TJ + j];
                                const float c = sPj[PJ_C * TJ + j];
                                int *kc = sKc + warp * 32;
                                float *kw = sKw + warp * 32 * 4 * NE;
                                for (int k0 = kf + 32 * sub; k0 <= kl; k0 += 32 * WPS) {
                                    const int k = k0 + lane;
                                    const int nk = min(32, kl - k0 + 1);
                                    if (lane < nk) {
                                        const float lr = __ldg(blam + k) * a;
                                        int iv; float t;
                                        axis_locate(lr, m.wave0, m.inv_dwave, m.wave_max, NW, iv, t);
                                        Taps4 tl;
                                        axis_taps_from<GRAD>(iv, t, NW, m.inv_dwave, tl);
                                        float dcl;
                                        const float cl = colour_law(m, lr, dcl);
                                        const float C = exp2f(kColour * c * cl);
                                        const float A = __ldg(bw + k) * C;
                                        kc[lane] = tl.first;
#pragma unroll
                                        for (int q = 0; q < 4; ++q) kw[lane * 4 * NE + q] = A * tl.w[q];
                                        if (GRAD && want_grad_E) {
                                            const float Ac = A * (kColourLn * cl);
                                            const float Zs = -A * lr * a;  // d lambda'/dz = -lambda' a
                                            const float Zv = Zs * (kColourLn * c * dcl);
#pragma unroll
                                            for (int q = 0; q < 4; ++q) {
                                                kw[lane * 4 * NE + 4 + q] = Ac * tl.w[q];
                                                kw[lane * 4 * NE + 8 + q] = fmaf(Zs, tl.dw[q], Zv * tl.w[q]);
                                            }
                                        }
                                    }
                                    __syncwarp();
                                    // gather: columns covered by this chunk of band samples
                                    const int cfirst = kc[0], clast = kc[nk - 1] + 3;
                                    for (int col = cfirst + lane; col <= clast; col += 32) {
                                        if (col < cc || col >= cc + W) continue;
                                        // contributing k: kc[k] in [col-3, col] (kc nondecreasing)
                                        int lo = 0, hi = nk;
                                        while (lo < hi) { int md = (lo + hi) >> 1; if (kc[md] >= col - 3) hi = md; else lo = md + 1; }
                                        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
                                        for (int q = lo; q < nk && kc[q] <= col; ++q) {
                                            const int mcol = col - kc[q];
                                            e0 += kw[q * 4 * NE + mcol];
                                            if (GRAD && want_grad_E) {
                                                e1 += kw[q * 4 * NE + 4 + mcol];
                                                e2 += kw[q * 4 * NE + 8 + mcol];
                                            }
                                        }
                                        const int cl_ = col - cc;
                                        if (WPS == 1) {
                                            sE[cl_ * TJ + j] += e0;
                                            if (GRAD && want_grad_E) {
                                                sE[WMAX * TJ + cl_ * TJ + j] += e1;
                                                sE[2 * WMAX * TJ + cl_ * TJ + j] += e2;
                                            }
                                        } else {
                                            sEp[warp * WMAX + cl_] += e0;
                                            if (GRAD && want_grad_E) {
                                                sEp[WARPS * WMAX + warp * WMAX + cl_] += e1;
                                                sEp[2 * WARPS * WMAX + warp * WMAX + cl_] += e2;
                                            }
                                        }
                                    }
                                    __syncwarp();
                                }
                            }
                        }
                        __syncthreads();
                        if (WPS > 1) {
                            for (int q = tid; q < ne_now * W * TJ; q += THREADS) {
                                const int e = q / (W * TJ), rem = q - e * W * TJ;
                                const int col = rem / TJ, j = rem - col * TJ;
                                float acc = 0.f;
#pragma unroll
                                for (int sb = 0; sb < WPS; ++sb) acc += sEp[e * WARPS * WMAX + (j * WPS + sb) * WMAX + col];
                                sE[e * WMAX * TJ + col * TJ + j] = acc;
                            }
                            __syncthreads();
                        }
                        // forward GEMM over the touched rows: LPR lanes per row
                        {
                            constexpr int RPW = 32 / LPR;  // rows per warp per pass
                            const int l4 = lane % LPR;
                            for (int rbase = 0; rbase < nrows; rbase += WARPS * RPW) {
                                const int rr = rbase + warp * RPW + lane / LPR;
                                const bool valid = rr < nrows;
                                const int r = valid ? sRows[rr] : 0;
                                float acc0[TJ], acc1[TJ];
#pragma unroll
                                for (int j = 0; j < TJ; ++j) { acc0[j] = 0.f; acc1[j] = 0.f; }
                                if (valid) {
                                    const float2 *grow = m.g01 + (size_t)r * NW + cc;
                                    for (int col = l4; col < W; col += LPR) {
                                        const float2 gv = __ldg(grow + col);
                                        const float *ev = sE + col * TJ;
                                        if (TJ % 4 == 0) {
#pragma unroll
                                            for (int j = 0; j < TJ; j += 4) {
                                                const float4 e4 = *reinterpret_cast<const float4 *>(ev + j);
                                                acc0[j] = fmaf(gv.x, e4.x, acc0[j]); acc1[j] = fmaf(gv.y, e4.x, acc1[j]);
                                                acc0[j + 1] = fmaf(gv.x, e4.y, acc0[j + 1]); acc1[j + 1] = fmaf(gv.y, e4.y, acc1[j + 1]);
                                                acc0[j + 2] = fmaf(gv.x, e4.z, acc0[j + 2]); acc1[j + 2] = fmaf(gv.y, e4.z, acc1[j + 2]);
                                                acc0[j + 3] = fmaf(gv.x, e4.w, acc0[j + 3]); acc1[j + 3] = fmaf(gv.y, e4.w, acc1[j + 3]);
                                            }
                                        } else {
#pragma unroll
                                            for (int j = 0; j < TJ; ++j) {
                                                acc0[j] = fmaf(gv.x, ev[j], acc0[j]);
                                                acc1[j] = fmaf(gv.y, ev[j], acc1[j]);
                                            }
                                        }
                                    }
                                }
#pragma unroll
                                for (int sh = 1; sh < LPR; sh <<= 1) {
#pragma unroll
                                    for (int j = 0; j < TJ; ++j) {
                                        acc0[j] += __shfl_xor_sync(0xffffffffu, acc0[j], sh);
                                        acc1[j] += __shfl_xor_sync(0xffffffffu, acc1[j], sh);
                                    }
                                }
                                if (valid && l4 == 0) {
#pragma unroll
                                    for (int j = 0; j < TJ; ++j) {
                                        sD[(r * TJ + j) * 2] += acc0[j];
                                        sD[(r * TJ + j) * 2 + 1] += acc1[j];
                                    }
                                }
                            }
                        }
                    }  // column chunks
                    __syncthreads();

                    // ---- 3. epilogue per (observation, sample) pair, in sub-chunks
                    if (GRAD)
                        for (int q = tid; q < nrows * TJ; q += THREADS) {
                            const int rr = q / TJ;
                            sY[sRows[rr] * TJ + (q - rr * TJ)] = 0.f;
                        }
                    const int sub_obs = PCAP / TJ;
                    for (int ib = 0; ib < nb_obs; ib += sub_obs) {
                        const int nsub = min(sub_obs, nb_obs - ib);
                        __syncthreads();
                        {
                            const int j = warp / WPS, sub = warp % WPS;
                            if (j < nj) {
                                const bool okj = sPj[PJ_OK * TJ + j] != 0.f;
                                const float a = sPj[PJ_A * TJ + j], x0 = sPj[PJ_X0 * TJ + j];
                                const float x1 = sPj[PJ_X1 * TJ + j];
                                const double t0 = ((const double *)(sPj + PJ_T0LO * TJ))[j];
                                for (int il = sub * 32 + lane; il < nsub; il += 32 * WPS) {
                                    const int i = ordb[ib + il];
                                    const int64_t gi = obase + i;
                                    const float p = (float)(b.mjd[gi] - t0) * a;
                                    int iv = -1; float t = 0.f;
                                    float Bs = 0.f, Bp = 0.f, B1 = 0.f;
                                    if (okj && axis_locate(p, m.phase0, m.inv_dphase, m.phase_max, m.n_phase, iv, t)) {
                                        Taps4 tp;
                                        axis_taps_from<GRAD>(iv, t, m.n_phase, m.inv_dphase, tp);
#pragma unroll
                                        for (int mm = 0; mm < 4; ++mm) {
                                            const float2 dv = *reinterpret_cast<const float2 *>(sD + ((tp.first + mm) * TJ + j) * 2);
                                            const float h = fmaf(x1, dv.y, dv.x);
                                            Bs = fmaf(tp.w[mm], h, Bs);
                                            if (GRAD) {
                                                Bp = fmaf(tp.dw[mm], h, Bp);
                                                B1 = fmaf(tp.w[mm], dv.y, B1);
                                            }
                                        }
                                    } else {
                                        iv = -1;
                                    }
                                    const float zpf = sZpf[i];
                                    const float pre = x0 * a * zpf;
                                    const float B = pre * Bs;
                                    if (MODE == MODE_BANDFLUX) {
                                        o.bandflux[wi.bf0 + (int64_t)(jloc0 + j) * nobs + (oc + i)] = B;
                                    } else {
                                        const float sig = b.fluxerr[gi];
                                        const float r = (b.flux[gi] - B) / sig;
                                        chi_acc = fma((double)r, (double)r, chi_acc);
                                        if (GRAD) {
                                            const float g = -2.0f * r / sig;
                                            gacc[0] += g * (-a * B - pre * a * p * Bp);
                                            gacc[1] += g * pre * Bp * (-a);
                                            gacc[2] += g * a * zpf * Bs;
                                            gacc[3] += g * pre * B1;
                                            sPf[il * TJ + j] = iv;
                                            sPt[il * TJ + j] = t;
                                            sPc[il * TJ + j] = g * pre;
                                        }
                                    }
                                }
                            }
                        }
                        if (GRAD) {
                            __syncthreads();
                            // adjoint rows, gathered per (row, sample) in observation order
                            for (int q = tid; q < nrows * nj; q += THREADS) {
                                const int rr = q / nj, j = q - rr * nj;
                                const int r = sRows[rr];
                                float y = 0.f;
                                for (int il = 0; il < nsub; ++il) {
                                    const int iv = sPf[il * TJ + j];
                                    if (iv < 0) continue;
                                    const int edge = (iv == 0) ? 1 : (iv == m.n_phase - 2 ? 2 : 0);
                                    const int first = (edge == 1) ? 0 : (edge == 2 ? m.n_phase - 4 : iv - 1);
                                    const int mm = r - first;
                                    if (mm < 0 || mm > 3) continue;
                                    float w, dw;
                                    tap_weight(mm, sPt[il * TJ + j], edge, w, dw);
                                    y = fmaf(sPc[il * TJ + j], w, y);
                                }
                                sY[r * TJ + j] += y;
                            }
                        }
                    }
                    // ---- 4. reverse GEMM: Q_j[col] = sum_r Y[r][j] H_j[r][col], dotted with E_c, E_z
                    if (GRAD) {
                        for (int ch = 0; ch < n_cchunks; ++ch) {
                            const int cc = C_lo + ch * WMAX;
                            const int W = min(WMAX, C_hi - cc + 1);
                            __syncthreads();
                            if (n_cchunks > 1) {
                                // rebuild E_c, E_z for this chunk (wide windows only)
                                for (int q = tid; q < 2 * WMAX * TJ; q += THREADS) sE[WMAX * TJ + q] = 0.f;
                                if (WPS > 1)
                                    for (int q = tid; q < 2 * WARPS * WMAX; q += THREADS) sEp[WARPS * WMAX + q] = 0.f;
                                __syncthreads();
                                const int j = warp / WPS, sub = warp % WPS;
                                if (j < nj && sPj[PJ_OK * TJ + j] != 0.f) {
                                    const int kf = __float_as_int(sPj[PJ_KF * TJ + j]);
                                    const int kl = __float_as_int(sPj[PJ_KL * TJ + j]);
                                    const float a = sPj[PJ_A * TJ + j];
                                    const float c = sPj[PJ_C * TJ + j];
                                    int *kc = sKc + warp * 32;
                                    float *kw = sKw + warp * 32 * 4 * NE;
                                    for (int k0 = kf + 32 * sub; k0 <= kl; k0 += 32 * WPS) {
                                        const int k = k0 + lane;
                                        const int nk = min(32, kl - k0 + 1);
                                        if (lane < nk) {
                                            const float lr = __ldg(blam + k) * a;
                                            int iv; float t;
                                            axis_locate(lr, m.wave0, m.inv_dwave, m.wave_max, NW, iv, t);
                                            Taps4 tl;
                                            axis_taps_from<true>(iv, t, NW, m.inv_dwave, tl);
                                            float dcl;
                                            const float cl = colour_law(m, lr, dcl);
                                            const float C = exp2f(kColour * c * cl);
                                            const float A = __ldg(bw + k) * C;
                                            const float Ac = A * (kColourLn * cl);
                                            const float Zs = -A * lr * a;
                                            const float Zv = Zs * (kColourLn * c * dcl);
                                            kc[lane] = tl.first;
#pragma unroll
                                            for (int q = 0; q < 4; ++q) {
                                                kw[lane * 4 * NE + 4 + q] = Ac * tl.w[q];
                                                kw[lane * 4 * NE + 8 + q] = fmaf(Zs, tl.dw[q], Zv * tl.w[q]);
                                            }
                                        }
                                        __syncwarp();
                                        const int cfirst = kc[0], clast = kc[nk - 1] + 3;
                                        for (int col = cfirst + lane; col <= clast; col += 32) {
                                            if (col < cc || col >= cc + W) continue;
                                            int lo = 0, hi = nk;
                                            while (lo < hi) { int md = (lo + hi) >> 1; if (kc[md] >= col - 3) hi = md; else lo = md + 1; }
                                            float e1 = 0.f, e2 = 0.f;
                                            for (int q = lo; q < nk && kc[q] <= col; ++q) {
                                                const int mcol = col - kc[q];
                                                e1 += kw[q * 4 * NE + 4 + mcol];
                                                e2 += kw[q * 4 * NE + 8 + mcol];
                                            }
                                            const int cl_ = col - cc;
                                            if (WPS == 1) {
                                                sE[WMAX * TJ + cl_ * TJ + j] += e1;
                                                sE[2 * WMAX * TJ + cl_ * TJ + j] += e2;
                                            } else {
                                                sEp[WARPS * WMAX + warp * WMAX + cl_] += e1;
                                                sEp[2 * WARPS * WMAX + warp * WMAX + cl_] += e2;
                                            }
                                        }
                                        __syncwarp();
                                    }
                                }
                                __syncthreads();
                                if (WPS > 1) {
                                    for (int q = tid; q < 2 * W * TJ; q += THREADS) {
                                        const int e = 1 + q / (W * TJ), rem = q % (W * TJ);
                                        const int col = rem / TJ, jj = rem - col * TJ;
                                        float acc = 0.f;
#pragma unroll
                                        for (int sb = 0; sb < WPS; ++sb) acc += sEp[e * WARPS * WMAX + (jj * WPS + sb) * WMAX + col];
                                        sE[e * WMAX * TJ + col * TJ + jj] = acc;
                                    }
                                }
                            }
                            __syncthreads();
                            // threads: column = tid % Wp, row subset = tid / Wp
                            const int Wp = (W + 31) & ~31;
                            const int nrs = max(1, THREADS / Wp);
                            const int col = tid % Wp, rs = tid / Wp;
                            if (col < W && rs < nrs) {
                                float q0[TJ], q1[TJ];
#pragma unroll
                                for (int j = 0; j < TJ; ++j) { q0[j] = 0.f; q1[j] = 0.f; }
                                const float2 *gcol = m.g01 + cc + col;
                                for (int rr = rs; rr < nrows; rr += nrs) {
                                    const int r = sRows[rr];
                                    const float2 gv = __ldg(gcol + (size_t)r * NW);
                                    const float *yv = sY + r * TJ;
#pragma unroll
                                    for (int j = 0; j < TJ; ++j) {
                                        q0[j] = fmaf(yv[j], gv.x, q0[j]);
                                        q1[j] = fmaf(yv[j], gv.y, q1[j]);
                                    }
                                }
#pragma unroll
                                for (int j = 0; j < TJ; ++j) {
                                    const float qv = fmaf(sPj[PJ_X1 * TJ + j], q1[j], q0[j]);
                                    gc_acc[j] = fmaf(qv, sE[WMAX * TJ + col * TJ + j], gc_acc[j]);
                                    gz_acc[j] = fmaf(qv, sE[2 * WMAX * TJ + col * TJ + j], gz_acc[j]);
                                }
                            }
                        }
                    }
                }  // bands
            }  // observation chunks

            // ---- per-sample reductions in a fixed order, outputs
            if (MODE != MODE_BANDFLUX) {
                __syncthreads();
                // epilogue partials: warp-level butterfly, then across the sample's warps
                chi_acc = warp_sum_d(chi_acc);
                float gr[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) gr[q] = GRAD ? warp_sum(gacc[q]) : 0.f;
                double *red = sRed;  // [WARPS][8 + 2*TJ]
                const int RS = 8 + 2 * TJ;
                if (lane == 0) {
                    red[warp * RS + 0] = chi_acc;
#pragma unroll
                    for (int q = 0; q < 4; ++q) red[warp * RS + 1 + q] = gr[q];
                }
                if (GRAD) {
#pragma unroll
                    for (int j = 0; j < TJ; ++j) {
                        const float vc = warp_sum(gc_acc[j]);
                        const float vz = warp_sum(gz_acc[j]);
                        if (lane == 0) { red[warp * RS + 8 + 2 * j] = vc; red[warp * RS + 8 + 2 * j + 1] = vz; }
                    }
                }
                __syncthreads();
                if (tid < nj) {
                    const int j = tid;
                    double x2 = 0.0;
                    float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                    for (int sb = 0; sb < WPS; ++sb) {
                        const int w = j * WPS + sb;
                        x2 += red[w * RS + 0];
                        g[0] += (float)red[w * RS + 1];
                        g[1] += (float)red[w * RS + 2];
                        g[2] += (float)red[w * RS + 3];
                        g[3] += (float)red[w * RS + 4];
                    }
                    if (GRAD) {
                        float gc = 0.f, gz = 0.f;
                        for (int w = 0; w < WARPS; ++w) {
                            gc += (float)red[w * RS + 8 + 2 * j];
                            gz += (float)red[w * RS + 8 + 2 * j + 1];
                        }
                        g[0] += gz;
                        g[4] = gc;
                    }
                    const bool bad = sPj[PJ_OK * TJ + j] == 0.f || sMisc[2] != 0;
                    o.chi2[pj0 + j] = bad ? __longlong_as_double(0x7ff8000000000000ll) : x2;
                    if (GRAD) {
#pragma unroll
                        for (int q = 0; q < 5; ++q) o.grad[5 * (pj0 + j) + q] = bad ? qnanf() : g[q];
                    }
                }
            } else {
                __syncthreads();
                // invalid supernova or sample: overwrite its bandfluxes with NaN
                for (int j = 0; j < nj; ++j) {
                    const bool bad = sPj[PJ_OK * TJ + j] == 0.f || sMisc[2] != 0;
                    if (bad)
                        for (int64_t i = tid; i < nobs; i += THREADS)
                            o.bandflux[wi.bf0 + (int64_t)(jloc0 + j) * nobs + i] = qnanf();
                }
            }
        }  // tiles
    }
}

}  // namespace fk

int factorised_smem_bytes(int tile, int mode) {
    return (int)fk::Lay(tile, mode == MODE_GRAD, fk::NPH_MAX).total;
}

int factorised_max_tile() { return 8; }

template <int TJ, int MODE>
static cudaError_t launch_fk(const salt_ctx *ctx, const WorkItem *items_d, int n_items, int *counter_d,
                             const BatchDev &b, const OutDev &o, cudaStream_t st) {
    const size_t smem = fk::Lay(TJ, MODE == MODE_GRAD, ctx->mp.n_phase).total;
    // one-time per (process, instantiation): opt in to the large dynamic shared memory
    static std::atomic<int> attr_done[64];
    cudaError_t e;
    const int dv = ctx->device & 63;
    if (!attr_done[dv].load()) {
        e = cudaFuncSetAttribute(fk::k_fact<TJ, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fk::Lay(TJ, MODE == MODE_GRAD, fk::NPH_MAX).total);
        if (e != cudaSuccess) return e;
        attr_done[dv].store(1);
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fk::k_fact<TJ, MODE>, fk::THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = ctx->num_sms * per_sm;
    if (grid > n_items) grid = n_items;
    if (grid < 1) return cudaSuccess;
    e = cudaMemsetAsync(counter_d, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    fk::k_fact<TJ, MODE><<<grid, fk::THREADS, smem, st>>>(ctx->mp, b, o, items_d, n_items, counter_d);
    return cudaGetLastError();
}

template <int TJ>
static cudaError_t launch_fk_mode(const salt_ctx *ctx, const WorkItem *items_d, int n_items, int *counter_d,
                                  const BatchDev &b, const OutDev &o, int mode, cudaStream_t st) {
    switch (mode) {
        case MODE_BANDFLUX: return launch_fk<TJ, MODE_BANDFLUX>(ctx, items_d, n_items, counter_d, b, o, st);
        case MODE_CHI2: return launch_fk<TJ, MODE_CHI2>(ctx, items_d, n_items, counter_d, b, o, st);
        default: return launch_fk<TJ, MODE_GRAD>(ctx, items_d, n_items, counter_d, b, o, st);
    }
}

cudaError_t launch_factorised_items(const salt_ctx *ctx, int tile, const WorkItem *items_d, int n_items,
                                    int *counter_d, const BatchDev &b, const OutDev &o, int mode,
                                    cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    switch (tile) {
        case 1: return launch_fk_mode<1>(ctx, items_d, n_items, counter_d, b, o, mode, st);
        case 2: return launch_fk_mode<2>(ctx, items_d, n_items, counter_d, b, o, mode, st);
        case 4: return launch_fk_mode<4>(ctx, items_d, n_items, counter_d, b, o, mode, st);
        default: return launch_fk_mode<8>(ctx, items_d, n_items, counter_d, b, o, mode, st);
    }
}

cudaError_t launch_factorised(const salt_ctx *ctx, const salt_plan *plan, const BatchDev &b,
                              const OutDev &o, int mode, cudaStream_t st) {
    return launch_factorised_items(ctx, plan->tile, plan->items_d, plan->n_items, plan->counter_d, b, o,
                                   mode, st);
}

}  // namespace salt
