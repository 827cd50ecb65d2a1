// Warp-scheduled factorised kernel: every warp independently pulls
// (supernova, band, group of TS samples) units from a global counter and runs
// the whole factorised pipeline for its unit (column response, row dots over
// the touched phase rows, per-observation epilogue) without any block-level
// barrier. The gradient is forward mode: the column responses E_c = dE/dc and
// E_z = dE/dz (through lambda') are built beside E, their row dots come from
// the same grid loads, and the epilogue finishes every derivative, so a unit
// makes a single pass over its grid window. A unit leaves its (sample, band) partials
// (chi^2 and gradient terms) in a scratch buffer; the warp that completes a
// supernova's last band (arrival counter per item) sums the partials in band
// order and writes the outputs, so results are bitwise reproducible whatever
// the arrival order. Suited to batches with few samples per supernova, where
// whole-supernova items leave warps idle behind block barriers.
#include "fact_common.cuh"

namespace salt {
namespace uk {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int OBS_W = 64;   // observations of the unit's band cached per pass
constexpr int WMAXW = 160;  // window columns per chunk
constexpr int NPHW = 128;   // phase nodes supported by this kernel
constexpr int NSLOT = 8;    // doubles per (sample, band) partial: chi2, g[6], invalid flag

using fk::al16;

struct Lay {
    // No block-level staging: the band tables are read through L1. With the D
    // rows sized by the model's phase nodes a block takes ~44 KB (71 nodes, one
    // sample, gradient); registers hold the kernel at three blocks per SM, and
    // the rest of the SM's 256 KB of L1/shared memory serves as L1 for the grid.
    size_t warp0, warp_bytes, total;
    __host__ __device__ Lay(int ts, bool grad, int np) {
        const int nd = grad ? 4 : 1;
        size_t o = 0;
        warp0 = o;
        // per warp: obs cache (index, mjd, flux, sig, zpf), column responses
        // [WMAXW][ts][E (, E_c, E_z, pad)], row dots D [np][ts][nd], row list [np]
        // (np = the model's phase nodes, at most NPHW)
        warp_bytes = al16(4 * OBS_W) + al16(8 * OBS_W) + 3 * al16(4 * OBS_W) +
                     al16(4 * (size_t)WMAXW * ts * (grad ? 4 : 1)) + al16(4 * (size_t)np * ts * nd) +
                     al16(4 * (size_t)np);
        o += WARPS * warp_bytes;
        total = o;
    }
};

struct UnitScratch {
    double *partial;  // [n_items][ts][n_bands][NSLOT]
    int *arrive;      // [n_items] bands finished (reset by the combining warp)
};

// Sums of 8 per-lane values over the warp by reduce-scatter (9 shuffles instead
// of 40): lane L returns the total of value (L >> 2) & 7. Fixed order.
__device__ __forceinline__ float warp_sum8_scatter(const float (&v)[8], int lane) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float k4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float r = __shfl_xor_sync(0xffffffffu, h16 ? v[j] : v[j + 4], 16);
        k4[j] = (h16 ? v[j + 4] : v[j]) + r;
    }
    float k2[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float r = __shfl_xor_sync(0xffffffffu, h8 ? k4[j] : k4[j + 2], 8);
        k2[j] = (h8 ? k4[j + 2] : k4[j]) + r;
    }
    float k1 = (h4 ? k2[1] : k2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? k2[0] : k2[1], 4);
    k1 += __shfl_xor_sync(0xffffffffu, k1, 2);
    k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
    return k1;
}

// L2 prefetch of everything a launch reads (inputs, work list, grid, band
// tables), cut into 32 KB pieces dealt round-robin over the CTAs; one thread per
// CTA issues its pieces. Skipped when the total would take a large share of L2.
__device__ __forceinline__ void prefetch_launch_l2(const ModelParams &m, const BatchDev &b,
                                                   const WorkItem *items, int n_items) {
    const void *ptr[14];
    size_t len[14];
    int n = 0;
    auto add = [&](const void *p, size_t l) {
        if (p && l) { ptr[n] = p; len[n] = l; ++n; }
    };
    add(b.mjd, 8 * (size_t)b.n_obs);
    add(b.band, 4 * (size_t)b.n_obs);
    add(b.flux, 4 * (size_t)b.n_obs);
    add(b.fluxerr, 4 * (size_t)b.n_obs);
    add(b.zp, 4 * (size_t)b.n_obs);
    add(b.t0, 8 * (size_t)b.n_par);
    add(b.z, 4 * (size_t)b.n_par);
    add(b.x0, 4 * (size_t)b.n_par);
    add(b.x1, 4 * (size_t)b.n_par);
    add(b.c, 4 * (size_t)b.n_par);
    add(items, sizeof(WorkItem) * (size_t)n_items);
    add(m.g01, sizeof(float2) * (size_t)m.n_phase * m.nw_pitch);
    add(m.band_lam, 4 * (size_t)m.bands.k_total);
    add(m.band_w, 4 * (size_t)m.bands.k_total);
    size_t total = 0;
    for (int r = 0; r < n; ++r) total += len[r];
    if (total > ((size_t)48 << 20)) return;
    constexpr size_t PIECE = 32768;
    const size_t G = gridDim.x, bid = blockIdx.x;
    size_t base = 0;  // global index of the range's first piece
    for (int r = 0; r < n; ++r) {
        const size_t np = (len[r] + PIECE - 1) / PIECE;
        for (size_t p = base + (bid + G - base % G) % G; p < base + np; p += G) {
            const size_t off = (p - base) * PIECE;
            prefetch_l2((const char *)ptr[r] + off, min(PIECE, len[r] - off));
        }
        base += np;
    }
}

template <int TS, int MODE>
__global__ void __launch_bounds__(THREADS, 3)
k_unit(ModelParams m, BatchDev b, OutDev o, const WorkItem *__restrict__ items, int n_items, int *counter,
       UnitScratch scr, const int *n_items_dev) {
    constexpr bool GRAD = MODE == MODE_GRAD;
    // row dots per (row, sample), with H = M0 + x1 M1 formed per grid value:
    // H.E (, M1.E, H.E_c, H.E_z)
    constexpr int ND = GRAD ? 4 : 1;
    constexpr int NEP = GRAD ? 4 : 1; // column-response slots per (column, sample)
    extern __shared__ __align__(16) unsigned char smem[];
    const Lay L(TS, GRAD, m.n_phase);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NB = m.bands.n_bands, NW = m.n_wave, NP = m.n_phase;
    unsigned char *wb = smem + L.warp0 + (size_t)warp * L.warp_bytes;
    int *oIdx = (int *)wb;                                     wb += al16(4 * OBS_W);
    float2 *oMjd = (float2 *)wb;                               wb += al16(8 * OBS_W);
    float *oFlux = (float *)wb;                                wb += al16(4 * OBS_W);
    float *oSig = (float *)wb;                                 wb += al16(4 * OBS_W);
    float *oZpf = (float *)wb;                                 wb += al16(4 * OBS_W);
    float *E = (float *)wb;                                    wb += al16(4 * (size_t)WMAXW * TS * NEP);
    float *D = (float *)wb;                                    wb += al16(4 * (size_t)NP * TS * ND);
    int *rowl = (int *)wb;

    if (tid == 0) prefetch_launch_l2(m, b, items, n_items);
    // with n_items_dev the list's length is read on the device (at most n_items)
    const int n_units = (n_items_dev ? min(*n_items_dev, n_items) : n_items) * NB;
    for (;;) {
        // claim one unit at a time: with few units per warp, claiming ahead
        // would fix the assignment and undo the dynamic balancing
        int u = 0;
        if (lane == 0) u = atomicAdd(counter, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        const int item = u / NB, bd = u - item * NB;
        const WorkItem wi = items[item];
        const int64_t ob0 = wi.obs0;
        const int nobs = wi.nobs;
        const int ns = wi.nj;  // <= TS

        // per-sample parameters (uniform across the warp)
        float pa[TS], px0[TS], px1[TS], pc[TS];
        float4 ppm[TS];  // phase maps
        bool pok[TS];
#pragma unroll
        for (int s = 0; s < TS; ++s) {
            pa[s] = 1.f; px0[s] = 0.f; px1[s] = 0.f; pc[s] = 0.f; ppm[s] = make_float4(0.f, 0.f, 0.f, 0.f); pok[s] = false;
            if (s < ns) {
                const int64_t g = wi.par0 + s;
                const float z = b.z[g], x0 = b.x0[g], x1 = b.x1[g], c = b.c[g];
                const double t0 = b.t0[g];
                pok[s] = isfinite(z) && z > -1.f && isfinite(x0) && isfinite(x1) && isfinite(c) && isfinite(t0);
                if (pok[s]) { ppm[s] = phase_map(m, z, t0, pa[s]); px0[s] = x0; px1[s] = x1; pc[s] = c; }
                else if (lane == 0 && bd == 0) atomicOr(o.err, ERRBIT_PARAM);
            }
        }
        const int K = m.bands.n[bd], koff = m.bands.off[bd];
        const float *lam = m.band_lam + koff;
        const float *wk = m.band_w + koff;

        // in-grid band-sample range per sample (contiguous in k) and the union window
        int kf[TS], kl[TS];
        int clo = 0x7fffffff, chi = -1;
#pragma unroll
        for (int s = 0; s < TS; ++s) {
            kf[s] = K; kl[s] = -1;
            if (pok[s] && K > 0 && lam[0] * pa[s] >= m.wave0 && lam[K - 1] * pa[s] <= m.wave_max) {
                kf[s] = 0;  // lambda ascending: both ends inside means every sample is
                kl[s] = K - 1;
            } else if (pok[s]) {
                for (int k0 = 0; k0 < K; k0 += 32) {
                    const int k = k0 + lane;
                    bool in = false;
                    if (k < K) {
                        const float lr = lam[k] * pa[s];
                        in = lr >= m.wave0 && lr <= m.wave_max;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, in);
                    if (bal) {
                        if (kf[s] == K) kf[s] = k0 + __ffs(bal) - 1;
                        kl[s] = k0 + 31 - __clz(bal);
                    }
                }
            }
            if (kf[s] <= kl[s]) {
                int iv; float t;
                { float iw_; wave_find(m, lam[kf[s]] * pa[s], iv, t, iw_); }
                clo = min(clo, fk::first_tap(iv, NW));
                { float iw_; wave_find(m, lam[kl[s]] * pa[s], iv, t, iw_); }
                chi = max(chi, fk::first_tap(iv, NW) + 3);
            }
        }
        const int nch = (chi >= clo) ? (chi - clo + WMAXW) / WMAXW : 0;

        double chi_acc[TS];
        float g[TS][6];
#pragma unroll
        for (int s = 0; s < TS; ++s) {
            chi_acc[s] = 0.0;
#pragma unroll
            for (int q = 0; q < 6; ++q) g[s][q] = 0.f;
        }
        bool bad_obs = false;

        // observation passes: gather this band's observations (in input order)
        int scan = 0;
        while (scan < nobs) {
            int nb_obs = 0;
            // band ids and errors of the next PRE chunks of 32, loaded together so
            // that their latencies overlap
            constexpr int PRE = 4;
            int pb[PRE];
            float pe[PRE];
            const int base0 = scan;
#pragma unroll
            for (int j = 0; j < PRE; ++j) {
                const int i = base0 + 32 * j + lane;
                pb[j] = i < nobs ? __ldg(b.band + ob0 + i) : -1;
                pe[j] = i < nobs ? __ldg(b.fluxerr + ob0 + i) : 1.f;
            }
            while (scan < nobs && nb_obs < OBS_W) {
                const int i = scan + lane;
                int bi = -1;
                float e = 1.f;
                if (i < nobs) {
                    const int off = scan - base0;  // warp-uniform
                    if ((off & 31) == 0 && off < 32 * PRE) {
#pragma unroll
                        for (int j = 0; j < PRE; ++j)
                            if (off == 32 * j) { bi = pb[j]; e = pe[j]; }
                    } else {
                        bi = b.band[ob0 + i];
                        e = b.fluxerr[ob0 + i];
                    }
                    if (bd == 0 && (bi < 0 || bi >= NB || !(e > 0.f))) {
                        bad_obs = true;
                        atomicOr(o.err, (bi < 0 || bi >= NB) ? ERRBIT_BAND : ERRBIT_SIGMA);
                        if (MODE == MODE_BANDFLUX)
                            for (int s = 0; s < ns; ++s)
                                o.bandflux[wi.bf0 + (int64_t)(wi.jloc0 + s) * nobs + i] = fk::qnanf();
                    }
                }
                const bool mine = i < nobs && bi == bd && e > 0.f;
                const unsigned bal = __ballot_sync(0xffffffffu, mine);
                const int room = OBS_W - nb_obs;
                const int cnt = __popc(bal);
                const int rank = __popc(bal & ((1u << lane) - 1u));
                if (mine && rank < room) {
                    const int slot = nb_obs + rank;
                    oIdx[slot] = i;
                    oSig[slot] = e;
                }
                if (cnt <= room) {
                    nb_obs += cnt;
                    scan += 32;
                } else {
                    // cache full: resume right after the last observation taken
                    nb_obs += room;
                    scan += (int)__fns(bal, 0, room) + 1;
                    break;
                }
            }
            bad_obs = __any_sync(0xffffffffu, bad_obs);
            __syncwarp();
            if (nb_obs == 0) continue;
            // the rest of the pass's observations, loaded together (independent loads)
            for (int q = lane; q < nb_obs; q += 32) {
                const int64_t gi = ob0 + oIdx[q];
                oMjd[q] = split_f2(b.mjd[gi]);
                oFlux[q] = b.flux[gi];
                oZpf[q] = zp_scale(b.zp[gi]);
            }
            __syncwarp();

            // touched phase rows of this pass, compacted into rowl
            unsigned msk[NPHW / 32] = {0u, 0u, 0u, 0u};
            for (int base = 0; base < nb_obs; base += 32) {
                const int il = base + lane;
                if (il < nb_obs) {
#pragma unroll
                    for (int s = 0; s < TS; ++s) {
                        if (!pok[s]) continue;
                        int iv; float t, iwp, p;
                        if (phase_find(m, oMjd[il], ppm[s], iv, t, iwp, p)) {
                            const int first = fk::first_tap(iv, NP);
                            const int w0 = first >> 5, sh = first & 31;
                            const unsigned lo = 0xfu << sh;                       // rows in word w0
                            const unsigned hi = sh > 28 ? 0xfu >> (32 - sh) : 0u;  // rows in word w0 + 1
#pragma unroll
                            for (int w = 0; w < NPHW / 32; ++w) {  // registers only: no dynamic index
                                if (w == w0) msk[w] |= lo;
                                if (w == w0 + 1) msk[w] |= hi;
                            }
                        }
                    }
                }
            }
            int nrows = 0;
#pragma unroll
            for (int w = 0; w < NPHW / 32; ++w) {
                const unsigned word = __reduce_or_sync(0xffffffffu, msk[w]);
                const bool on = (word >> lane) & 1u;
                if (on) rowl[nrows + __popc(word & ((1u << lane) - 1u))] = w * 32 + lane;
                nrows += __popc(word);
            }
            __syncwarp();
            for (int q = lane; q < nrows * TS * ND; q += 32) {
                const int rr = q / (TS * ND);
                D[rowl[rr] * TS * ND + (q - rr * TS * ND)] = 0.f;
            }
            __syncwarp();

            // column response and forward row dots, per column chunk
            for (int ch = 0; ch < nch; ++ch) {
                const int cc = clo + ch * WMAXW;
                const int W = min(WMAXW, chi - cc + 1);
                for (int q = lane; q < W * TS * NEP; q += 32) E[q] = 0.f;
                __syncwarp();
#pragma unroll
                for (int s = 0; s < TS; ++s) {
                    if (kf[s] > kl[s]) continue;
                    if (GRAD)
                        fk::ebuild3(m, lam, wk, kl[s], kf[s], 32, pa[s], pc[s], cc, W, lane, E + 4 * s,
                                    E + 4 * s + 1, E + 4 * s + 2, 4 * TS);
                    else
                        fk::ebuild(m, lam, wk, kl[s], kf[s], 32, pa[s], pc[s], cc, W, lane, E + s, TS);
                }
                __syncwarp();
                const int l4 = lane & 3;
                for (int rb = 0; rb < nrows; rb += 8) {
                    const int rr = rb + (lane >> 2);
                    const bool valid = rr < nrows;
                    const int r = valid ? rowl[rr] : 0;
                    float acc[TS][ND];
#pragma unroll
                    for (int s = 0; s < TS; ++s)
#pragma unroll
                        for (int d = 0; d < ND; ++d) acc[s][d] = 0.f;
                    if (valid) {
                        const float2 *grow = m.g01 + (size_t)r * m.nw_pitch + cc;
                        constexpr int UF = 8;
                        for (int col0 = l4; col0 < W; col0 += 4 * UF) {
                            float2 gv[UF];
#pragma unroll
                            for (int uu = 0; uu < UF; ++uu) {
                                const int col = col0 + 4 * uu;
                                gv[uu] = col < W ? __ldg(grow + col) : make_float2(0.f, 0.f);
                            }
#pragma unroll
                            for (int uu = 0; uu < UF; ++uu) {
                                const int col = min(col0 + 4 * uu, W - 1);
#pragma unroll
                                for (int s = 0; s < TS; ++s) {
                                    const float h = fmaf(px1[s], gv[uu].y, gv[uu].x);  // M0 + x1 M1
                                    if constexpr (GRAD) {
                                        const float4 ev = *reinterpret_cast<const float4 *>(E + (col * TS + s) * 4);
                                        acc[s][0] = fmaf(h, ev.x, acc[s][0]);
                                        acc[s][1] = fmaf(gv[uu].y, ev.x, acc[s][1]);
                                        acc[s][2] = fmaf(h, ev.y, acc[s][2]);
                                        acc[s][3] = fmaf(h, ev.z, acc[s][3]);
                                    } else {
                                        acc[s][0] = fmaf(h, E[col * TS + s], acc[s][0]);
                                    }
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int s = 0; s < TS; ++s)
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            acc[s][d] += __shfl_xor_sync(0xffffffffu, acc[s][d], 1);
                            acc[s][d] += __shfl_xor_sync(0xffffffffu, acc[s][d], 2);
                        }
                    if (valid && l4 == 0) {
#pragma unroll
                        for (int s = 0; s < TS; ++s)
#pragma unroll
                            for (int d = 0; d < ND; ++d) D[(r * TS + s) * ND + d] += acc[s][d];
                    }
                }
                __syncwarp();
            }

            // epilogue per (observation, sample): bandflux, residual, chi^2, gradient terms, adjoint rows
            for (int base = 0; base < nb_obs; base += 32) {
                const int il = base + lane;
                const bool act = il < nb_obs;
                const float2 mj = act ? oMjd[il] : make_float2(0.f, 0.f);
                const float zpf = act ? oZpf[il] : 0.f;
                const float fl = act ? oFlux[il] : 0.f;
                const float sig = act ? oSig[il] : 1.f;
#pragma unroll
                for (int s = 0; s < TS; ++s) {
                    Taps4 tp;
                    float Bs = 0.f, Bp = 0.f, B1 = 0.f, Bc = 0.f, Bz = 0.f;
                    if (act && s < ns) {
                        const float a = pa[s];
                        int iv; float t, iwp, p = 0.f;
                        if (pok[s] && phase_find(m, mj, ppm[s], iv, t, iwp, p)) {
                            axis_taps_from<GRAD>(iv, t, NP, iwp, tp);
#pragma unroll
                            for (int mm = 0; mm < 4; ++mm) {
                                const float *dv = D + ((tp.first + mm) * TS + s) * ND;
                                Bs = fmaf(tp.w[mm], dv[0], Bs);
                                if (GRAD) {
                                    Bp = fmaf(tp.dw[mm], dv[0], Bp);
                                    B1 = fmaf(tp.w[mm], dv[1], B1);
                                    Bc = fmaf(tp.w[mm], dv[2], Bc);
                                    Bz = fmaf(tp.w[mm], dv[3], Bz);
                                }
                            }
                        }
                        const float pre = px0[s] * a * zpf;
                        const float B = pre * Bs;
                        if (pok[s] && !isfinite(B)) atomicOr(o.err, ERRBIT_RANGE);
                        if (MODE == MODE_BANDFLUX) {
                            o.bandflux[wi.bf0 + (int64_t)(wi.jloc0 + s) * nobs + oIdx[il]] = pok[s] ? B : fk::qnanf();
                        } else {
                            const float r = (fl - B) / sig;
                            chi_acc[s] = fma((double)r, (double)r, chi_acc[s]);
                            if (GRAD) {
                                const float gg = -2.0f * r / sig;
                                g[s][0] += gg * (-a * B - pre * a * p * Bp);
                                g[s][1] += gg * pre * Bp * (-a);
                                g[s][2] += gg * a * zpf * Bs;
                                g[s][3] += gg * pre * B1;
                                g[s][4] += gg * pre * Bc;
                                g[s][5] += gg * pre * Bz;
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }  // observation passes

        if (MODE == MODE_BANDFLUX) continue;  // bandfluxes are written by the epilogue

        // unit partials -> scratch; the last band of the item combines in band order
        double *pbase = scr.partial + (size_t)item * TS * NB * NSLOT;
#pragma unroll
        for (int s = 0; s < TS; ++s) {
            const double x2 = warp_sum_d(chi_acc[s]);
            double *sl = pbase + ((size_t)s * NB + bd) * NSLOT;
            if (lane == 0) {
                sl[0] = x2;
                sl[7] = bad_obs ? 1.0 : 0.0;
            }
            if (GRAD) {
                float v[8] = {g[s][0], g[s][1], g[s][2], g[s][3], g[s][4], g[s][5], 0.f, 0.f};
                const float gsum = warp_sum8_scatter(v, lane);
                const int q = (lane >> 2) & 7;
                if ((lane & 3) == 0 && q < 6) sl[1 + q] = gsum;
            }
        }
        int last = 0;
        __syncwarp();  // every lane's partial stores precede lane 0's fence
        if (lane == 0) {
            __threadfence();
            last = atomicAdd(scr.arrive + item, 1) == NB - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) continue;
        __threadfence();
        if (lane < ns) {
            const int s = lane;
            double x2 = 0.0;
            float gg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool badv = false;
            for (int bb = 0; bb < NB; ++bb) {
                const double *sl = pbase + ((size_t)s * NB + bb) * NSLOT;
                x2 += __ldcg(sl);
                if (GRAD)
#pragma unroll
                    for (int q = 0; q < 6; ++q) gg[q] += (float)__ldcg(sl + 1 + q);
                badv |= __ldcg(sl + 7) != 0.0;
            }
            const bool bad = badv || !pok[min(s, TS - 1)];
            const int64_t gj = wi.par0 + s;
            o.chi2[gj] = bad ? __longlong_as_double(0x7ff8000000000000ll) : x2;
            if (GRAD) {
                const float gout[5] = {gg[0] + gg[5], gg[1], gg[2], gg[3], gg[4]};
#pragma unroll
                for (int q = 0; q < 5; ++q) o.grad[5 * gj + q] = bad ? fk::qnanf() : gout[q];
            }
        }
        if (lane == 0) scr.arrive[item] = 0;  // ready for the next launch
    }
}

}  // namespace uk

int unit_item_samples() { return 2; }
int unit_max_phase() { return uk::NPHW; }
size_t unit_scratch_bytes(int n_items, int ts, int n_bands) {
    return (size_t)n_items * ts * (n_bands > 0 ? n_bands : 1) * uk::NSLOT * sizeof(double) +
           (size_t)n_items * sizeof(int) + 256;
}

template <int TS, int MODE>
static cudaError_t launch_uk(const salt_ctx *ctx, const WorkItem *items_d, int n_items, int *counter_d,
                             void *scratch, const BatchDev &b, const OutDev &o, cudaStream_t st,
                             const int *n_items_dev) {
    const size_t smem = uk::Lay(TS, MODE == MODE_GRAD, ctx->mp.n_phase).total;
    // once per (device, instantiation): opt in at the size of the largest model
    // the kernel takes (NPHW phase nodes), so that contexts with more phase
    // nodes than the first one launched stay within the opted-in limit
    static std::atomic<int> attr_done[64];
    cudaError_t e;
    const int dv = ctx->device & 63;
    if (!attr_done[dv].load()) {
        e = cudaFuncSetAttribute(uk::k_unit<TS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)uk::Lay(TS, MODE == MODE_GRAD, uk::NPHW).total);
        if (e != cudaSuccess) return e;
        attr_done[dv].store(1);
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, uk::k_unit<TS, MODE>, uk::THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int nb = ctx->mp.bands.n_bands > 0 ? ctx->mp.bands.n_bands : 1;
    const int64_t units = (int64_t)n_items * nb;
    int grid = ctx->num_sms * per_sm;
    if ((int64_t)grid * uk::WARPS > units) grid = (int)((units + uk::WARPS - 1) / uk::WARPS);
    if (grid < 1) return cudaSuccess;
    uk::UnitScratch scr;
    scr.partial = (double *)scratch;
    scr.arrive = (int *)((unsigned char *)scratch + (size_t)n_items * TS * nb * uk::NSLOT * sizeof(double));
    e = cudaMemsetAsync(counter_d, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    uk::k_unit<TS, MODE><<<grid, uk::THREADS, smem, st>>>(ctx->mp, b, o, items_d, n_items, counter_d, scr,
                                                          n_items_dev);
    return cudaGetLastError();
}

cudaError_t launch_unit_items(const salt_ctx *ctx, int ts, const WorkItem *items_d, int n_items, int *counter_d,
                              void *scratch, const BatchDev &b, const OutDev &o, int mode, cudaStream_t st,
                              const int *n_items_dev) {
    if (n_items <= 0) return cudaSuccess;
    if (ts == 2) {
        switch (mode) {
            case MODE_BANDFLUX: return launch_uk<2, MODE_BANDFLUX>(ctx, items_d, n_items, counter_d, scratch, b, o, st, n_items_dev);
            case MODE_CHI2: return launch_uk<2, MODE_CHI2>(ctx, items_d, n_items, counter_d, scratch, b, o, st, n_items_dev);
            default: return launch_uk<2, MODE_GRAD>(ctx, items_d, n_items, counter_d, scratch, b, o, st, n_items_dev);
        }
    }
    switch (mode) {
        case MODE_BANDFLUX: return launch_uk<1, MODE_BANDFLUX>(ctx, items_d, n_items, counter_d, scratch, b, o, st, n_items_dev);
        case MODE_CHI2: return launch_uk<1, MODE_CHI2>(ctx, items_d, n_items, counter_d, scratch, b, o, st, n_items_dev);
        default: return launch_uk<1, MODE_GRAD>(ctx, items_d, n_items, counter_d, scratch, b, o, st, n_items_dev);
    }
}

}  // namespace salt
