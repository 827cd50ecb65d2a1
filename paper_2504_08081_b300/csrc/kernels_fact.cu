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
// Per (sample tile, band) the kernel
//   1. builds E (and, for the gradient, E_c = dE/dc and E_z, the lambda' part
//      of dE/dz) over the tile's union column window,
//   2. forms the row dots D[r][j] = sum_col G[r][col] E_j[col] for every phase
//      row an observation touches (a small GEMM on packed FP32 FMA),
//   3. finishes each (observation, sample) pair from 4 row dots: bandflux,
//      residual, FP64 chi^2 and the direct gradient terms, and scatters the
//      adjoint weights Y[r][j] += g_ij pre_ij phi_r(p_ij),
//   4. (gradient) back-projects Q_j[col] = sum_r Y[r][j] (G0 + x1 G1)[r][col]
//      and dots Q with E_c and E_z for dchi2/dc and the lambda' part of dchi2/dz.
// Tiles take an item's samples in t0 order, so their phase rows mostly
// coincide. Every sum has a fixed order, so results are bitwise reproducible
// for a given tile size.
#include <cstdio>

#include "fact_common.cuh"

namespace salt {
namespace fk {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int OBS_MAX = 512;   // observations of one supernova staged per pass
constexpr int WMAX = 256;      // union window columns per column chunk
constexpr int LPR = 4;         // lanes per row in the forward GEMM
constexpr int NPH_MAX = 256;   // phase nodes supported
constexpr int KTOT = 2048;     // band samples (all bands) staged in shared memory per CTA
constexpr int ITEM_MAX = 128;  // samples ordered together (a multiple of every tile)
// Row stride of the sample-major column arrays (the build's staging rows, Q):
// WMAX + 4 columns, 4 modulo 32 banks, so that a warp reading 4 consecutive
// columns of 8 samples, or 32 consecutive columns of one sample, touches 32
// distinct banks.
constexpr int ES = WMAX + 4;


struct Lay {
    size_t ord, zpf, band, mjd, flux, sig, bst, lam, wk, pj, pm, rowmask, rows, misc, E, Q, D, Yw, kst, red, key,
        perm, total;
    __host__ __device__ Lay(int tj, bool grad, int n_phase) {
        const int nslot = tj > WARPS ? tj : WARPS;  // (warp, sample) slots
        const bool stage = tj <= 8;                 // 16-sample tiles read band samples through L1
        size_t o = 0;
        ord = o;     o = al16(o + 4 * OBS_MAX);
        zpf = o;     o = al16(o + 4 * OBS_MAX);
        band = o;    o = al16(o + 4 * OBS_MAX);
        mjd = o;     o = al16(o + 8 * OBS_MAX);
        flux = o;    o = al16(o + 4 * OBS_MAX);
        sig = o;     o = al16(o + 4 * OBS_MAX);
        bst = o;     o = al16(o + 4 * (2 * SALT_MAX_BANDS + 2));
        lam = o;     o = al16(o + (stage ? 4 * KTOT : 0));
        wk = o;      o = al16(o + (stage ? 4 * KTOT : 0));
        pj = o;      o = al16(o + 4 * 8 * tj);
        pm = o;      o = al16(o + 16 * tj);
        rowmask = o; o = al16(o + 4 * (NPH_MAX / 32));
        rows = o;    o = al16(o + 4 * NPH_MAX);
        misc = o;    o = al16(o + 4 * 16);
        E = o;       o = al16(o + 4 * (size_t)ES * tj);
        // the column-response staging rows [slot][ES] share their space with the
        // reverse GEMM partials (never live at the same time)
        const size_t nq = grad ? (size_t)THREADS * tj : 0, nst = (size_t)nslot * ES;
        Q = o;       o = al16(o + 4 * (nq > nst ? nq : nst));
        D = o;       o = al16(o + 4 * (size_t)n_phase * tj * 2);
        Yw = o;      o = al16(o + (grad ? 4 * (size_t)nslot * n_phase : 0));
        kst = o;     o = al16(o + 4 * (size_t)WARPS * 128);
        red = o;     o = al16(o + 8 * (size_t)nslot * 8);
        key = o;     o = al16(o + 8 * ITEM_MAX);
        perm = o;    o = al16(o + 4 * ITEM_MAX);
        total = o;
    }
};

// per-sample scalar slots in Lay::pj
enum { PJ_A = 0, PJ_X0, PJ_X1, PJ_C, PJ_OK, PJ_KF, PJ_KL, PJ_NUM };

// Row dot of one touched row against the column responses of the tile:
// acc[j] += sum_col G[row][col] E[col][j] over this lane's columns. For an
// even tile the samples go in pairs through the packed FP32 FMA (acc[p] holds
// samples 2p and 2p + 1; the grid value is broadcast to both halves): per
// column and pair one instruction per surface instead of two. Each half is
// an ordinary fused multiply-add, so the sums are those of the scalar loop.
template <int TJ, bool SMEM>
__device__ __forceinline__ void fwd_row_dot(const float2 *grow, int W, int l4, const float *sE, float2 *acc0,
                                            float2 *acc1) {
    static_assert(TJ % 2 == 0, "packed row dot needs an even tile");
    constexpr int U = 8;
    for (int col0 = l4; col0 < W; col0 += U * LPR) {
        float2 gv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int col = col0 + u * LPR;
            gv[u] = col < W ? (SMEM ? grow[col] : __ldg(grow + col)) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int col = col0 + u * LPR;
            if (col >= W) break;  // the last pass's slots past the window (all lanes but a column's worth)
            const float2 gx = make_float2(gv[u].x, gv[u].x), gy = make_float2(gv[u].y, gv[u].y);
            if (TJ % 4 == 0) {
                const float4 *ev = reinterpret_cast<const float4 *>(sE + col * TJ);
#pragma unroll
                for (int p4 = 0; p4 < TJ / 4; ++p4) {
                    const float4 e4 = ev[p4];
                    const float2 ea = make_float2(e4.x, e4.y), eb = make_float2(e4.z, e4.w);
                    acc0[2 * p4] = __ffma2_rn(gx, ea, acc0[2 * p4]);
                    acc1[2 * p4] = __ffma2_rn(gy, ea, acc1[2 * p4]);
                    acc0[2 * p4 + 1] = __ffma2_rn(gx, eb, acc0[2 * p4 + 1]);
                    acc1[2 * p4 + 1] = __ffma2_rn(gy, eb, acc1[2 * p4 + 1]);
                }
            } else {
                const float2 *ev = reinterpret_cast<const float2 *>(sE + col * TJ);
#pragma unroll
                for (int p = 0; p < TJ / 2; ++p) {
                    const float2 e = ev[p];
                    acc0[p] = __ffma2_rn(gx, e, acc0[p]);
                    acc1[p] = __ffma2_rn(gy, e, acc1[p]);
                }
            }
        }
    }
}

// The same for a one-sample tile (scalar FMAs).
template <bool SMEM>
__device__ __forceinline__ void fwd_row_dot1(const float2 *grow, int W, int l4, const float *sE, float &acc0,
                                             float &acc1) {
    constexpr int U = 8;
    for (int col0 = l4; col0 < W; col0 += U * LPR) {
        float2 gv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int col = col0 + u * LPR;
            gv[u] = col < W ? (SMEM ? grow[col] : __ldg(grow + col)) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float e = sE[min(col0 + u * LPR, W - 1)];
            acc0 = fmaf(gv[u].x, e, acc0);
            acc1 = fmaf(gv[u].y, e, acc1);
        }
    }
}

// Back-projection of the adjoint rows onto one column, over the rows
// rs, rs + nrs, ...: q[j] += sum_r Y[r][j] G[r][col], samples in pairs
// through the packed FMA as in fwd_row_dot (q[p] holds samples 2p, 2p + 1).
// With SMEM the grid rows are the staged window's slots (slot = position in
// the touched-row list).
template <int TJ, bool SMEM>
__device__ __forceinline__ void rev_col_dot(const float2 *gcol, size_t stride, const int *sRows, int rs, int nrs,
                                            int nrows, const float *sY, float2 *q0, float2 *q1) {
    static_assert(TJ % 2 == 0, "packed column dot needs an even tile");
    constexpr int U = 8;
    for (int rr0 = rs; rr0 < nrows; rr0 += U * nrs) {
        float2 gv[U];
        int rv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int rr = rr0 + u * nrs;
            rv[u] = rr < nrows ? sRows[rr] : -1;
            gv[u] = rv[u] < 0 ? make_float2(0.f, 0.f)
                              : (SMEM ? gcol[(size_t)rr * stride] : __ldg(gcol + (size_t)rv[u] * stride));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (rv[u] < 0) continue;
            const float2 gx = make_float2(gv[u].x, gv[u].x), gy = make_float2(gv[u].y, gv[u].y);
            if (TJ % 4 == 0) {
                const float4 *yv = reinterpret_cast<const float4 *>(sY + rv[u] * TJ);
#pragma unroll
                for (int p4 = 0; p4 < TJ / 4; ++p4) {
                    const float4 y4 = yv[p4];
                    const float2 ya = make_float2(y4.x, y4.y), yb = make_float2(y4.z, y4.w);
                    q0[2 * p4] = __ffma2_rn(ya, gx, q0[2 * p4]);
                    q1[2 * p4] = __ffma2_rn(ya, gy, q1[2 * p4]);
                    q0[2 * p4 + 1] = __ffma2_rn(yb, gx, q0[2 * p4 + 1]);
                    q1[2 * p4 + 1] = __ffma2_rn(yb, gy, q1[2 * p4 + 1]);
                }
            } else {
                const float2 *yv = reinterpret_cast<const float2 *>(sY + rv[u] * TJ);
#pragma unroll
                for (int p = 0; p < TJ / 2; ++p) {
                    const float2 y = yv[p];
                    q0[p] = __ffma2_rn(y, gx, q0[p]);
                    q1[p] = __ffma2_rn(y, gy, q1[p]);
                }
            }
        }
    }
}

// The same for a one-sample tile.
template <bool SMEM>
__device__ __forceinline__ void rev_col_dot1(const float2 *gcol, size_t stride, const int *sRows, int rs, int nrs,
                                             int nrows, const float *sY, float &q0, float &q1) {
    constexpr int U = 8;
    for (int rr0 = rs; rr0 < nrows; rr0 += U * nrs) {
        float2 gv[U];
        int rv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int rr = rr0 + u * nrs;
            rv[u] = rr < nrows ? sRows[rr] : -1;
            gv[u] = rv[u] < 0 ? make_float2(0.f, 0.f)
                              : (SMEM ? gcol[(size_t)rr * stride] : __ldg(gcol + (size_t)rv[u] * stride));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (rv[u] < 0) continue;
            const float y = sY[rv[u]];
            q0 = fmaf(y, gv[u].x, q0);
            q1 = fmaf(y, gv[u].y, q1);
        }
    }
}

// Y[first + m] += v_m for the 4 taps of each lane (first < 0: nothing).
// Lanes with the same first row form one group for all 4 taps; each group's
// sums run in lane order (deterministic) and its lowest lane adds them, tap
// by tap, so groups whose rows overlap add in a fixed order too. yval: 32
// float4 of the warp's staging.
__device__ __forceinline__ void y_scatter(float *yw, float *yval, int lane, int first, float4 yv) {
    const bool has = first >= 0;
    const int key = has ? first : -1 - lane;
    if (!has) yv = make_float4(0.f, 0.f, 0.f, 0.f);
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const bool lead = has && lane == __ffs(grp) - 1;
    if (!__all_sync(0xffffffffu, grp == (1u << lane))) {
        reinterpret_cast<float4 *>(yval)[lane] = yv;
        __syncwarp();
        if (lead) {
            float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
            unsigned g2 = grp;
            while (g2) {
                const float4 v = reinterpret_cast<const float4 *>(yval)[__ffs(g2) - 1];
                s4.x += v.x; s4.y += v.y; s4.z += v.z; s4.w += v.w;
                g2 &= g2 - 1;
            }
            yv = s4;
        }
        __syncwarp();
    }
    const float ys[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) {
        if (lead) yw[key + mm] += ys[mm];
        __syncwarp();
    }
}

template <int TJ, int MODE>
__global__ void __launch_bounds__(THREADS, 3)
k_fact(ModelParams m, BatchDev b, OutDev o, const WorkItem *__restrict__ items, int n_items,
       int *counter) {
    constexpr bool GRAD = MODE == MODE_GRAD;
    constexpr int WPS = TJ >= WARPS ? 1 : WARPS / TJ;  // warps per sample
    constexpr int SPW = TJ > WARPS ? TJ / WARPS : 1;   // samples per warp
    // (warp, jj) -> sample (warp / WPS) * SPW + jj, slot warp * SPW + jj
    extern __shared__ __align__(16) unsigned char smem[];
    const Lay L(TJ, GRAD, m.n_phase);
    int *sOrd = (int *)(smem + L.ord);
    float *sZpf = (float *)(smem + L.zpf);
    int *sBst = (int *)(smem + L.bst);  // [0..NB] band starts, [NB+1..] running positions
    float *sLam = (float *)(smem + L.lam);
    float *sWk = (float *)(smem + L.wk);
    float *sPj = (float *)(smem + L.pj);    // [PJ_NUM][TJ]
    float4 *sPm = (float4 *)(smem + L.pm);  // [TJ] phase maps
    unsigned *sRowMask = (unsigned *)(smem + L.rowmask);
    int *sRows = (int *)(smem + L.rows);
    int *sMisc = (int *)(smem + L.misc);
    float *sE = (float *)(smem + L.E);     // [WMAX][TJ] column responses (then Q as [TJ][ES])
    float *sSt = (float *)(smem + L.Q);    // [slot][ES] column-response staging rows, one per (warp, sample)
    float *sQ = (float *)(smem + L.Q);     // [TJ/2][THREADS] float2 reverse-GEMM partials (after the build)
    float *sD = (float *)(smem + L.D);     // [n_phase][TJ][2]
    float *sYw = (float *)(smem + L.Yw);   // [slots][n_phase] adjoint rows per (warp, sample)
    float2 *sMjd = (float2 *)(smem + L.mjd);  // observation times as float pairs
    int *sBand = (int *)(smem + L.band);
    float *sFlux = (float *)(smem + L.flux);
    float *sSig = (float *)(smem + L.sig);  // 1 / fluxerr
    double *sRed = (double *)(smem + L.red);
    double *sKey = (double *)(smem + L.key);  // [ITEM_MAX] t0 of the item's samples
    int *sPerm = (int *)(smem + L.perm);      // [ITEM_MAX] samples in t0 order

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NB = m.bands.n_bands;
    const int NW = m.n_wave;
    const int NP = m.n_phase;
    // per-warp staging for the column-response build and the adjoint scatter
    float *yval = (float *)(smem + L.kst) + warp * 128;  // per-warp adjoint scatter staging (32 float4)
    // every band's samples stay in shared memory for the CTA's lifetime
    const bool bands_staged = TJ <= 8 && m.bands.k_total <= KTOT;
    if (bands_staged)
        for (int k = tid; k < m.bands.k_total; k += THREADS) {
            sLam[k] = __ldg(m.band_lam + k);
            sWk[k] = __ldg(m.band_w + k);
        }

    if (tid == 0) sMisc[1] = atomicAdd(counter, 1);
    for (;;) {
        __syncthreads();
        const int it = sMisc[1];
        __syncthreads();
        if (it >= n_items) break;
        const WorkItem wi = items[it];
        if (tid == 0) {
            // claim the next item now and pull its data into L2 while this one runs
            const int nxt = atomicAdd(counter, 1);
            sMisc[1] = nxt;
            if (nxt < n_items) prefetch_item(b, items[nxt]);
        }
        const int64_t ob0 = wi.obs0;
        const int64_t nobs = wi.nobs;
        if (tid == 0) sMisc[2] = 0;  // any invalid observation in this supernova

        const bool one_obs_chunk = nobs <= OBS_MAX;

        for (int jt = 0; jt < wi.nj; jt += TJ) {
            const int nj = min(TJ, wi.nj - jt);
            // the item's samples are taken in t0 order within groups of ITEM_MAX (ties
            // by position, non-finite last): a tile's samples then share most of their
            // phase rows, so the row dots run over smaller row unions; each sample's
            // outputs still go to its own place
            const int g0 = jt - jt % ITEM_MAX;  // first sample of this tile's group
            if (jt == g0) {
                const int gn = min(ITEM_MAX, wi.nj - g0);
                __syncthreads();  // the previous group's readers of sPerm are done
                if (tid < gn) {
                    const double t = b.t0[wi.par0 + g0 + tid];
                    sKey[tid] = isfinite(t) ? t : __longlong_as_double(0x7ff0000000000000ll);
                }
                __syncthreads();
                if (tid < gn) {
                    const double k = sKey[tid];
                    int r = 0;
                    for (int i = 0; i < gn; ++i) {
                        const double ki = sKey[i];
                        r += (ki < k) || (ki == k && i < tid);
                    }
                    sPerm[r] = g0 + tid;
                }
            }
            const int *tperm = sPerm + (jt - g0);  // tile slot -> the sample's position in the item

            // ---- per-sample parameters
            __syncthreads();
            if (tid < TJ) {
                const int j = tid;
                float z = 0.f, x0 = 0.f, x1 = 0.f, c = 0.f;
                double t0 = 0.0;
                int ok = 0;
                if (j < nj) {
                    const int64_t pj = wi.par0 + tperm[j];
                    z = b.z[pj]; x0 = b.x0[pj]; x1 = b.x1[pj]; c = b.c[pj];
                    t0 = b.t0[pj];
                    ok = isfinite(z) && z > -1.f && isfinite(x0) && isfinite(x1) && isfinite(c) &&
                         isfinite(t0);
                    if (!ok) atomicOr(o.err, ERRBIT_PARAM);
                }
                if (!ok) { z = 0.f; x0 = 0.f; x1 = 0.f; c = 0.f; t0 = 0.0; }
                float a;
                sPm[j] = phase_map(m, z, t0, a);
                sPj[PJ_A * TJ + j] = a;
                sPj[PJ_X0 * TJ + j] = x0;
                sPj[PJ_X1 * TJ + j] = x1;
                sPj[PJ_C * TJ + j] = c;
                sPj[PJ_OK * TJ + j] = (j < nj && ok) ? 1.f : 0.f;
            }
            // per-lane accumulators with a fixed assignment (deterministic sums):
            // warp w owns sample w / WPS in the epilogue and the reverse dot
            double chi_acc[SPW];
            float gacc[SPW][6];  // z(prefactor+phase), t0, x0, x1, c, z(lambda')
#pragma unroll
            for (int jj = 0; jj < SPW; ++jj) {
                chi_acc[jj] = 0.0;
#pragma unroll
                for (int q = 0; q < 6; ++q) gacc[jj][q] = 0.f;
            }

            for (int64_t oc = 0; oc < nobs; oc += OBS_MAX) {
                const int nc = (int)min((int64_t)OBS_MAX, nobs - oc);
                const int64_t obase = ob0 + oc;
                // ---- observations to shared memory, validation, stable counting sort by
                // band (once per item when they fit in one pass)
                if (!one_obs_chunk || jt == 0) {
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
                    sBand[i] = (okb && e > 0.f) ? bd : -1;
                }
                __syncthreads();
                if (warp == 0) {
                    int *cnt = sBst + 1;  // counts at [1..NB]
                    for (int base = 0; base < nc; base += 32) {
                        const int i = base + lane;
                        int bd = -1;
                        if (i < nc) {
                            bd = sBand[i];
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
                            bd = sBand[i];
                        }
                        const unsigned mm = __match_any_sync(0xffffffffu, bd);
                        const int rank = __popc(mm & ((1u << lane) - 1u));
                        if (bd >= 0) {
                            const int ps = pos[bd] + rank;
                            sOrd[ps] = i;
                            sBand[i] = ps;  // from here on: the observation's sorted position
                        }
                        __syncwarp();
                        if (bd >= 0 && lane == __ffs(mm) - 1) pos[bd] += __popc(mm);
                        __syncwarp();
                    }
                }
                __syncthreads();
                // the valid observations' values staged in band-sorted order: a band's
                // observations are then consecutive (conflict-free reads in the epilogue)
                for (int i = tid; i < nc; i += THREADS) {
                    const int ps = sBand[i];
                    if (ps < 0) continue;
                    sZpf[ps] = zp_scale(b.zp[obase + i]);
                    sMjd[ps] = split_f2(b.mjd[obase + i]);
                    sFlux[ps] = b.flux[obase + i];
                    sSig[ps] = 1.0f / b.fluxerr[obase + i];
                }
                __syncthreads();
                }

                for (int bd = 0; bd < NB; ++bd) {
                    const int nb_obs = sBst[bd + 1] - sBst[bd];
                    if (nb_obs == 0) continue;  // uniform: sBst is shared
                    const int ob0s = sBst[bd];  // the band's first observation in sorted order
                    const int K = m.bands.n[bd], koff = m.bands.off[bd];
                    const float *lam = (bands_staged ? sLam : m.band_lam) + koff;
                    const float *wk = (bands_staged ? sWk : m.band_w) + koff;

                    // ---- 1. band samples to shared memory; window and rows
                    __syncthreads();
                    if (tid == 0) { sMisc[4] = 0x7fffffff; sMisc[5] = -1; sMisc[6] = 0; }
                    for (int q = tid; q < NPH_MAX / 32; q += THREADS) sRowMask[q] = 0u;
                    if (GRAD)
                        for (int q = tid; q < WARPS * SPW * NP; q += THREADS) sYw[q] = 0.f;
                    __syncthreads();
                    // the window on the last warp: the row marking below starts at warp 0
                    if (warp == WARPS - 1 && lane < nj) {
                        const int j = lane;
                        const float a = sPj[PJ_A * TJ + j];
                        int kf = K, kl = -1;
                        if (sPj[PJ_OK * TJ + j] != 0.f && lam[0] * a >= m.wave0 && lam[K - 1] * a <= m.wave_max) {
                            kf = 0;  // lambda ascending: both ends inside means every sample is
                            kl = K - 1;
                        } else if (sPj[PJ_OK * TJ + j] != 0.f) {
                            // first k with a*lambda_k >= wave0; last with a*lambda_k <= wave_max
                            int lo = 0, hi = K;
                            while (lo < hi) { const int md = (lo + hi) >> 1; if (lam[md] * a >= m.wave0) hi = md; else lo = md + 1; }
                            kf = lo;
                            lo = kf; hi = K;
                            while (lo < hi) { const int md = (lo + hi) >> 1; if (lam[md] * a <= m.wave_max) lo = md + 1; else hi = md; }
                            kl = lo - 1;
                        }
                        sPj[PJ_KF * TJ + j] = __int_as_float(kf);
                        sPj[PJ_KL * TJ + j] = __int_as_float(kl);
                        if (kf <= kl) {
                            int iv; float t;
                            { float iw_; wave_find(m, lam[kf] * a, iv, t, iw_); }
                            atomicMin(&sMisc[4], first_tap(iv, NW));
                            { float iw_; wave_find(m, lam[kl] * a, iv, t, iw_); }
                            atomicMax(&sMisc[5], first_tap(iv, NW) + 3);
                        }
                    }
                    // touched phase rows (all obs of the band, all samples of the tile): each
                    // lane's 4-row pattern is OR-reduced over the warp, one shared atomic per word
                    for (int qb = warp * 32; qb < nb_obs * nj; qb += THREADS) {
                        const int q = qb + lane;
                        int first = -1;
                        if (q < nb_obs * nj) {
                            const int il = q / nj, j = q - il * nj;
                            if (sPj[PJ_OK * TJ + j] != 0.f) {
                                const int i = ob0s + il;
                                int iv; float t, iwp, p;
                                if (phase_find(m, sMjd[i], sPm[j], iv, t, iwp, p))
                                    first = first_tap(iv, NP);
                            }
                        }
                        for (int wd = 0; wd < (NP + 31) / 32; ++wd) {
                            unsigned bits = 0u;
                            if (first >= 0) {
                                const int lo = first - wd * 32;  // rows first..first+3 relative to word wd
                                if (lo >= 0 && lo < 32) bits |= 0xfu << lo;
                                else if (lo < 0 && lo > -4) bits |= 0xfu >> (-lo);
                            }
                            const unsigned word = __reduce_or_sync(0xffffffffu, bits);
                            if (lane == 0 && word) atomicOr(&sRowMask[wd], word);
                        }
                    }
                    __syncthreads();
                    if (warp == 0) {
                        int base = 0;
                        for (int wd = 0; wd < (NP + 31) / 32; ++wd) {
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
                    for (int q = tid; q < nrows * TJ * 2; q += THREADS) {
                        const int rr = q / (TJ * 2), jj2 = q - rr * TJ * 2;  // (sample, surface)
                        sD[((jj2 >> 1) * NP + sRows[rr]) * 2 + (jj2 & 1)] = 0.f;
                    }
                    const int n_cchunks = (C_hi >= C_lo) ? (C_hi - C_lo + WMAX) / WMAX : 0;
                    // ---- 2. column response + forward GEMM, per column chunk
                    for (int ch = 0; ch < n_cchunks; ++ch) {
                        const int cc = C_lo + ch * WMAX;
                        const int W = min(WMAX, C_hi - cc + 1);
                        __syncthreads();
                        // each (warp, sample) slot builds into its own staging row, column
                        // after column (consecutive banks for the runs' column adds), then
                        // the rows are summed over a sample's warps in order and transposed
                        // to E[col][j]
#pragma unroll
                        for (int jj = 0; jj < SPW; ++jj) {
                            const int j = (warp / WPS) * SPW + jj, sub = warp % WPS;
                            float *e0 = sSt + (warp * SPW + jj) * ES;
                            for (int q = lane; q < W; q += 32) e0[q] = 0.f;
                            __syncwarp();
                            if (j < nj && sPj[PJ_OK * TJ + j] != 0.f) {
                                const int kf = __float_as_int(sPj[PJ_KF * TJ + j]);
                                const int kl = __float_as_int(sPj[PJ_KL * TJ + j]);
                                const float a = sPj[PJ_A * TJ + j], c = sPj[PJ_C * TJ + j];
                                const int k0 = (kf & ~1) + 64 * sub;  // even: one 8-byte load per lane's pair
                                if (n_cchunks == 1)
                                    ebuild_pair<true>(m, lam, wk, kf, kl, k0, 64 * WPS, a, c, cc, W, lane, e0, 1);
                                else
                                    ebuild_pair<false>(m, lam, wk, kf, kl, k0, 64 * WPS, a, c, cc, W, lane, e0, 1);
                            }
                        }
                        __syncthreads();
                        for (int q = tid; q < W * TJ; q += THREADS) {
                            const int col = q / TJ, j = q - col * TJ;
                            float acc = 0.f;
#pragma unroll
                            for (int sb = 0; sb < WPS; ++sb) acc += sSt[(j * WPS + sb) * ES + col];
                            sE[col * TJ + j] = acc;
                        }
                        __syncthreads();
                        // forward GEMM over the touched rows: LPR lanes per row, 8 columns in flight
                        {
                            constexpr int RPW = 32 / LPR;
                            const int l4 = lane % LPR;
                            // few rows (an 8-sample tile's usual case): two warps per row group,
                            // each over half the columns, so every warp has work; the first
                            // half's sums are added to D before the second's (a fixed order)
                            const bool split = TJ == 8 && nrows <= (WARPS / 2) * RPW;
                            const int half = split ? warp / (WARPS / 2) : 0;
                            const int wrow = split ? warp % (WARPS / 2) : warp;
                            const int Wh = (W + 1) / 2;
                            const int c0 = split && half ? Wh : 0;
                            const int c1 = split && !half ? Wh : W;
                            for (int rbase = 0; rbase < nrows; rbase += (split ? WARPS / 2 : WARPS) * RPW) {
                                const int rr = rbase + wrow * RPW + lane / LPR;
                                const bool valid = rr < nrows;
                                const int r = valid ? sRows[rr] : 0;
                                float acc0[TJ], acc1[TJ];  // per sample: M0 and M1 row dots
                                if constexpr (TJ == 1) {
                                    acc0[0] = 0.f; acc1[0] = 0.f;
                                    if (valid)
                                        fwd_row_dot1<false>(m.g01 + (size_t)r * m.nw_pitch + cc, W, l4, sE, acc0[0],
                                                            acc1[0]);
                                } else {
                                    float2 a0[TJ / 2], a1[TJ / 2];
#pragma unroll
                                    for (int p = 0; p < TJ / 2; ++p) {
                                        a0[p] = make_float2(0.f, 0.f); a1[p] = make_float2(0.f, 0.f);
                                    }
                                    if (valid)
                                        fwd_row_dot<TJ, false>(m.g01 + (size_t)r * m.nw_pitch + cc + c0, c1 - c0, l4,
                                                               sE + c0 * TJ, a0, a1);
#pragma unroll
                                    for (int p = 0; p < TJ / 2; ++p) {
                                        acc0[2 * p] = a0[p].x; acc0[2 * p + 1] = a0[p].y;
                                        acc1[2 * p] = a1[p].x; acc1[2 * p + 1] = a1[p].y;
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
                                for (int ph = 0; ph < (split ? 2 : 1); ++ph) {
                                    if (ph == 1) __syncthreads();  // first half's columns added first
                                    if (valid && l4 == 0 && half == ph) {
#pragma unroll
                                        for (int j = 0; j < TJ; ++j) {
                                            float2 *dv = reinterpret_cast<float2 *>(sD + (j * NP + r) * 2);
                                            float2 d = *dv;
                                            d.x += acc0[j];
                                            d.y += acc1[j];
                                            *dv = d;
                                        }
                                    }
                                }
                            }
                        }
                    }  // column chunks
                    __syncthreads();

                    // ---- 3. epilogue per (observation, sample) pair; adjoint scatter
#pragma unroll
                    for (int jj = 0; jj < SPW; ++jj) {
                        const int j = (warp / WPS) * SPW + jj, sub = warp % WPS;
                        if (j < nj) {
                            const bool okj = sPj[PJ_OK * TJ + j] != 0.f;
                            const float a = sPj[PJ_A * TJ + j], x0 = sPj[PJ_X0 * TJ + j];
                            const float x1 = sPj[PJ_X1 * TJ + j];
                            const float4 pm = sPm[j];
                            float *yw = sYw + (warp * SPW + jj) * NP;
                            // observations in pairs (il, il + 32) through the packed FP32 forms; each
                            // lane takes il's terms, then il + 32's (the order of the one-at-a-time loop)
                            for (int base = sub * 64; base < nb_obs; base += 64 * WPS) {
                                const int ila = base + lane, ilb = ila + 32;
                                const bool acta = ila < nb_obs, actb = ilb < nb_obs;
                                const int ia = ob0s + (acta ? ila : 0), ib = ob0s + (actb ? ilb : 0);
                                bool oka = false, okb = false;
                                int iva = 0, ivb = 0;
                                float2 t = f2(0.f), iwp = f2(0.f), p = f2(0.f);
                                if (okj && acta) phase_find2(m, sMjd[ia], sMjd[ib], pm, oka, okb, iva, ivb, t, iwp, p);
                                oka = oka && acta;
                                okb = okb && actb;
                                t = make_float2(oka ? t.x : 0.f, okb ? t.y : 0.f);  // finite weights off the axis
                                int fa, fb;
                                float2 w[4], dw[4];
                                axis_taps_from2<GRAD>(iva, ivb, t, NP, iwp, fa, fb, w, dw);
                                if (!oka) fa = -1;
                                if (!okb) fb = -1;
                                float2 Bs = f2(0.f), Bp = f2(0.f), B1 = f2(0.f);
                                const float *dj = sD + j * NP * 2;
#pragma unroll
                                for (int mm = 0; mm < 4; ++mm) {
                                    const float2 da = oka ? *reinterpret_cast<const float2 *>(dj + (fa + mm) * 2) : f2(0.f);
                                    const float2 db = okb ? *reinterpret_cast<const float2 *>(dj + (fb + mm) * 2) : f2(0.f);
                                    const float2 dy = make_float2(da.y, db.y);
                                    const float2 h = __ffma2_rn(f2(x1), dy, make_float2(da.x, db.x));
                                    Bs = __ffma2_rn(w[mm], h, Bs);
                                    if (GRAD) {
                                        Bp = __ffma2_rn(dw[mm], h, Bp);
                                        B1 = __ffma2_rn(w[mm], dy, B1);
                                    }
                                }
                                float2 coef = f2(0.f);
                                if (acta) {
                                    const float2 zpf = make_float2(sZpf[ia], sZpf[ib]);
                                    const float2 pre = __fmul2_rn(f2(x0 * a), zpf);
                                    const float2 B = __fmul2_rn(pre, Bs);
                                    if (!isfinite(B.x) || (actb && !isfinite(B.y))) atomicOr(o.err, ERRBIT_RANGE);
                                    if (MODE == MODE_BANDFLUX) {
                                        float *bo = o.bandflux + wi.bf0 + (int64_t)(wi.jloc0 + tperm[j]) * nobs + oc;
                                        bo[sOrd[ia]] = B.x;
                                        if (actb) bo[sOrd[ib]] = B.y;
                                    } else {
                                        const float2 isig = make_float2(sSig[ia], sSig[ib]);
                                        const float2 r = __fmul2_rn(fsub2(make_float2(sFlux[ia], sFlux[ib]), B), isig);
                                        chi_acc[jj] = fma((double)r.x, (double)r.x, chi_acc[jj]);
                                        if (actb) chi_acc[jj] = fma((double)r.y, (double)r.y, chi_acc[jj]);
                                        if (GRAD) {
                                            const float2 g = __fmul2_rn(__fmul2_rn(f2(-2.0f), r), isig);
                                            // terms of dchi2/dz (prefactor and phase), dt0, dx0, dx1
                                            const float2 T0 = fsub2(__fmul2_rn(f2(-a), B),
                                                                    __fmul2_rn(__fmul2_rn(__fmul2_rn(pre, f2(a)), p), Bp));
                                            const float2 T1 = __fmul2_rn(__fmul2_rn(pre, Bp), f2(-a));
                                            const float2 T2 = __fmul2_rn(__fmul2_rn(f2(a), zpf), Bs);
                                            const float2 T3 = __fmul2_rn(pre, B1);
                                            gacc[jj][0] = fmaf(g.x, T0.x, gacc[jj][0]);
                                            gacc[jj][1] = fmaf(g.x, T1.x, gacc[jj][1]);
                                            gacc[jj][2] = fmaf(g.x, T2.x, gacc[jj][2]);
                                            gacc[jj][3] = fmaf(g.x, T3.x, gacc[jj][3]);
                                            if (actb) {
                                                gacc[jj][0] = fmaf(g.y, T0.y, gacc[jj][0]);
                                                gacc[jj][1] = fmaf(g.y, T1.y, gacc[jj][1]);
                                                gacc[jj][2] = fmaf(g.y, T2.y, gacc[jj][2]);
                                                gacc[jj][3] = fmaf(g.y, T3.y, gacc[jj][3]);
                                            }
                                            coef = __fmul2_rn(g, pre);
                                        }
                                    }
                                }
                                if (GRAD) {
                                    y_scatter(yw, yval, lane, fa,
                                              make_float4(coef.x * w[0].x, coef.x * w[1].x, coef.x * w[2].x, coef.x * w[3].x));
                                    if (base + 32 < nb_obs)  // (warp-uniform: some lane has an observation il + 32)
                                        y_scatter(yw, yval, lane, fb,
                                                  make_float4(coef.y * w[0].y, coef.y * w[1].y, coef.y * w[2].y,
                                                              coef.y * w[3].y));
                                }
                            }
                        }
                    }
                    // ---- 4. reverse: Q_j[col] = sum_r Y[r][j] H_j[r][col], then per band sample adjoints
                    if (GRAD) {
                        __syncthreads();
                        // combine the per-warp adjoint rows into Y[r][j] (in warp order)
                        float *sY = sD;  // D is no longer needed: reuse it as Y[n_phase][TJ]
                        for (int q = tid; q < nrows * TJ; q += THREADS) {
                            const int rr = q / TJ, j = q - rr * TJ;
                            const int r = sRows[rr];
                            float y = 0.f;
#pragma unroll
                            for (int sb = 0; sb < WPS; ++sb) y += sYw[(j * WPS + sb) * NP + r];
                            sY[r * TJ + j] = y;
                        }
                        for (int ch = 0; ch < n_cchunks; ++ch) {
                            const int cc = C_lo + ch * WMAX;
                            const int W = min(WMAX, C_hi - cc + 1);
                            __syncthreads();
                            // partial Q per (row subset, column): threads = column + row split
                            // (W threads per row subset, so nearly all threads have a column)
                            // row subsets: the fewest that keep the fewest passes of the
                            // 8-row unrolled loop (fewer busy warps, the same latency)
                            const int Wp = W;
                            const int nrs_max = THREADS / Wp;
                            const int passes = max(1, ((nrows + nrs_max - 1) / nrs_max + 7) / 8);
                            const int nrs = max(1, min(nrs_max, (nrows + 8 * passes - 1) / (8 * passes)));
                            {
                                const int col = tid % Wp, rs = tid / Wp;
                                if constexpr (TJ == 1) {
                                    float q0 = 0.f, q1 = 0.f;
                                    if (col < W && rs < nrs)
                                        rev_col_dot1<false>(m.g01 + cc + col, (size_t)m.nw_pitch, sRows, rs, nrs,
                                                            nrows, sY, q0, q1);
                                    sQ[tid] = fmaf(sPj[PJ_X1], q1, q0);
                                } else {
                                    float2 q0[TJ / 2], q1[TJ / 2];
#pragma unroll
                                    for (int p = 0; p < TJ / 2; ++p) {
                                        q0[p] = make_float2(0.f, 0.f); q1[p] = make_float2(0.f, 0.f);
                                    }
                                    if (col < W && rs < nrs)
                                        rev_col_dot<TJ, false>(m.g01 + cc + col, (size_t)m.nw_pitch, sRows, rs, nrs,
                                                               nrows, sY, q0, q1);
                                    const float2 *x1p = reinterpret_cast<const float2 *>(sPj + PJ_X1 * TJ);
                                    float2 *qo = reinterpret_cast<float2 *>(sQ) + tid;
#pragma unroll
                                    for (int p = 0; p < TJ / 2; ++p) qo[p * THREADS] = __ffma2_rn(x1p[p], q1[p], q0[p]);
                                }
                            }
                            __syncthreads();
                            // Q_j[col] = sum over row subsets in order, sample-major with row
                            // stride ES (into the E buffer, free now): warps take sample pairs,
                            // lanes consecutive columns
                            float *sQf = sE;
                            if constexpr (TJ == 1) {
                                for (int col = tid; col < W; col += THREADS) {
                                    float qv = 0.f;
                                    for (int rs = 0; rs < nrs; ++rs) qv += sQ[rs * Wp + col];
                                    sQf[col] = qv;
                                }
                            } else {
                                constexpr int NPAIR = TJ / 2, WPP = WARPS / NPAIR;  // warps per sample pair
                                const float2 *qp = reinterpret_cast<const float2 *>(sQ) + (warp / WPP) * THREADS;
                                float *q0 = sQf + (2 * (warp / WPP)) * ES;
                                for (int col = (warp % WPP) * 32 + lane; col < W; col += 32 * WPP) {
                                    float2 qv = make_float2(0.f, 0.f);
                                    for (int rs = 0; rs < nrs; ++rs) {
                                        const float2 v = qp[rs * Wp + col];
                                        qv.x += v.x;
                                        qv.y += v.y;
                                    }
                                    q0[col] = qv.x;
                                    q0[ES + col] = qv.y;
                                }
                            }
                            __syncthreads();
                            // adjoint of the column response per band sample: dchi2/dc and the
                            // rest-wavelength part of dchi2/dz (warp -> sample, band samples split by sub)
#pragma unroll
                            for (int jj = 0; jj < SPW; ++jj) {
                                const int j = (warp / WPS) * SPW + jj, sub = warp % WPS;
                                if (j < nj && sPj[PJ_OK * TJ + j] != 0.f) {
                                    const int kf = __float_as_int(sPj[PJ_KF * TJ + j]);
                                    const int kl = __float_as_int(sPj[PJ_KL * TJ + j]);
                                    const float a = sPj[PJ_A * TJ + j], c = sPj[PJ_C * TJ + j];
                                    if (n_cchunks == 1)
                                        eadjoint_pair<true>(m, lam, wk, kl, kf + 64 * sub, 64 * WPS, a, c, cc, W, lane,
                                                            sQf + j * ES, 1, gacc[jj][4], gacc[jj][5]);
                                    else
                                        eadjoint_pair<false>(m, lam, wk, kl, kf + 64 * sub, 64 * WPS, a, c, cc, W, lane,
                                                             sQf + j * ES, 1, gacc[jj][4], gacc[jj][5]);
                                }
                            }
                        }
                    }
                }  // bands
            }  // observation chunks

            // ---- per-sample reductions in a fixed order, outputs
            if (MODE != MODE_BANDFLUX) {
                __syncthreads();
#pragma unroll
                for (int jj = 0; jj < SPW; ++jj) {
                    const double x2w = warp_sum_d(chi_acc[jj]);
                    float gr[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) gr[q] = GRAD ? warp_sum(gacc[jj][q]) : 0.f;
                    if (lane == 0) {
                        double *rd = sRed + (warp * SPW + jj) * 8;
                        rd[0] = x2w;
#pragma unroll
                        for (int q = 0; q < 6; ++q) rd[1 + q] = gr[q];
                    }
                }
                __syncthreads();
                if (tid < nj) {
                    const int j = tid;
                    double x2 = 0.0;
                    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    for (int sb = 0; sb < WPS; ++sb) {
                        const int w = j * WPS + sb;
                        x2 += sRed[w * 8 + 0];
#pragma unroll
                        for (int q = 0; q < 6; ++q) g[q] += (float)sRed[w * 8 + 1 + q];
                    }
                    const bool bad = sPj[PJ_OK * TJ + j] == 0.f || sMisc[2] != 0;
                    const int64_t pj = wi.par0 + tperm[j];
                    o.chi2[pj] = bad ? __longlong_as_double(0x7ff8000000000000ll) : x2;
                    if (GRAD) {
                        const float gout[5] = {g[0] + g[5], g[1], g[2], g[3], g[4]};
#pragma unroll
                        for (int q = 0; q < 5; ++q) o.grad[5 * pj + q] = bad ? qnanf() : gout[q];
                    }
                }
            } else {
                __syncthreads();
                // invalid supernova or sample: overwrite its bandfluxes with NaN
                for (int j = 0; j < nj; ++j) {
                    const bool bad = sPj[PJ_OK * TJ + j] == 0.f || sMisc[2] != 0;
                    if (bad)
                        for (int64_t i = tid; i < nobs; i += THREADS)
                            o.bandflux[wi.bf0 + (int64_t)(wi.jloc0 + tperm[j]) * nobs + i] = qnanf();
                }
            }
        }  // tiles
    }
}

}  // namespace fk

int factorised_smem_bytes(int tile, int mode) {
    return (int)fk::Lay(tile, mode == MODE_GRAD, fk::NPH_MAX).total;
}

int factorised_max_tile() { return 16; }

template <int TJ, int MODE>
static cudaError_t launch_fk(const salt_ctx *ctx, const WorkItem *items_d, int n_items, int *counter_d,
                             const BatchDev &b, const OutDev &o, cudaStream_t st) {
    const size_t smem = fk::Lay(TJ, MODE == MODE_GRAD, ctx->mp.n_phase).total;
    // once per (device, instantiation): opt in to the dynamic shared memory size
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
        case 8: return launch_fk_mode<8>(ctx, items_d, n_items, counter_d, b, o, mode, st);
        default: return launch_fk_mode<16>(ctx, items_d, n_items, counter_d, b, o, mode, st);
    }
}

}  // namespace salt
