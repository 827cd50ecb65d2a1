// Band-parallel factorised kernel: the same factorisation as k_fact (column
// response E, row dots D = G E over touched phase rows, per-pair epilogue,
// reverse-mode adjoint), but each warp owns one (band, group of TS samples)
// unit and runs it warp-synchronously. A CTA takes one (supernova,
// sample-range) item, spreads its units over 8 warps, and after a single
// barrier reduces the per-(sample, band) partials in band order, so results
// are bitwise reproducible for a given TS. Suited to items with few samples
// (batched one-vector fits, small serving requests), where band-serial phases
// separated by CTA barriers would leave most warps idle.
#include "fact_common.cuh"

namespace salt {
namespace bw {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int OBS_MAX = 512;   // observations of one supernova staged per pass
constexpr int WMAXW = 192;     // window columns per chunk (per warp)
constexpr int NPHW = 128;      // phase nodes supported by this kernel
constexpr int NJ_MAX = 16;     // samples per item
constexpr int NSLOT = 8;       // doubles per (sample, band) partial: chi2, g[6]
constexpr int KTOT = 2048;     // band samples (all bands) staged in shared memory per CTA

using fk::al16;

struct Lay {
    size_t ord, zpf, band, mjd, flux, sig, bst, pj, pm, slots, misc, lam, wk, warp0, warp_bytes, total;
    __host__ __device__ Lay(int ts, bool grad, int nb) {
        size_t o = 0;
        ord = o;   o = al16(o + 4 * OBS_MAX);
        zpf = o;   o = al16(o + 4 * OBS_MAX);
        band = o;  o = al16(o + 4 * OBS_MAX);
        mjd = o;   o = al16(o + 8 * OBS_MAX);
        flux = o;  o = al16(o + 4 * OBS_MAX);
        sig = o;   o = al16(o + 4 * OBS_MAX);
        bst = o;   o = al16(o + 4 * (2 * SALT_MAX_BANDS + 2));
        pj = o;    o = al16(o + 4 * 8 * NJ_MAX);
        pm = o;    o = al16(o + 16 * NJ_MAX);
        slots = o; o = al16(o + 8 * (size_t)NSLOT * NJ_MAX * (nb > 0 ? nb : 1));
        misc = o;  o = al16(o + 4 * (16 + SALT_MAX_BANDS));
        lam = o;   o = al16(o + 4 * KTOT);
        wk = o;    o = al16(o + 4 * KTOT);
        warp0 = o;
        // per warp: E [ne][WMAXW][ts], D [NPHW][ts][2], Y [NPHW][ts], rows [NPHW], yval[32]
        warp_bytes = al16(4 * (size_t)WMAXW * ts) + al16(4 * (size_t)NPHW * ts * 2) +
                     al16(grad ? 4 * (size_t)NPHW * ts : 0) + al16(4 * NPHW) + al16(4 * 32);
        o += WARPS * warp_bytes;
        total = o;
    }
};

enum { PJ_A = 0, PJ_X0, PJ_X1, PJ_C, PJ_OK };

template <int TS, int MODE>
__global__ void __launch_bounds__(THREADS, 2)
k_bandwarp(ModelParams m, BatchDev b, OutDev o, const WorkItem *__restrict__ items, int n_items,
           int *counter) {
    constexpr bool GRAD = MODE == MODE_GRAD;
    extern __shared__ __align__(16) unsigned char smem[];
    const int NB = m.bands.n_bands;
    const Lay L(TS, GRAD, NB);
    int *sOrd = (int *)(smem + L.ord);
    float *sZpf = (float *)(smem + L.zpf);
    int *sBand = (int *)(smem + L.band);
    float2 *sMjd = (float2 *)(smem + L.mjd);  // observation times as float pairs
    float *sFlux = (float *)(smem + L.flux);
    float *sSig = (float *)(smem + L.sig);
    int *sBst = (int *)(smem + L.bst);
    float *sPj = (float *)(smem + L.pj);  // [5][NJ_MAX]
    float4 *sPm = (float4 *)(smem + L.pm);    // [NJ_MAX] phase maps
    double *sSlot = (double *)(smem + L.slots);  // [NJ_MAX][NB][NSLOT]
    int *sMisc = (int *)(smem + L.misc);
    int *sPresent = sMisc + 16;  // present band ids, in band order

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NW = m.n_wave, NP = m.n_phase;

    unsigned char *wbase = smem + L.warp0 + (size_t)warp * L.warp_bytes;
    float *E = (float *)wbase;  // [WMAXW][TS] column responses, then Q
    float *D = (float *)(wbase + al16(4 * (size_t)WMAXW * TS));  // [NPHW][TS][2]
    float *Y = (float *)((unsigned char *)D + al16(4 * (size_t)NPHW * TS * 2));  // [NPHW][TS]
    int *rowl = (int *)((unsigned char *)Y + al16(GRAD ? 4 * (size_t)NPHW * TS : 0));
    float *yval = (float *)((unsigned char *)rowl + al16(4 * NPHW));
    float *sLam = (float *)(smem + L.lam);
    float *sWk = (float *)(smem + L.wk);
    const bool bands_staged = m.bands.k_total <= KTOT;
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
        const int nj = wi.nj;  // <= NJ_MAX

        if (tid < NJ_MAX) {
            const int j = tid;
            float z = 0.f, x0 = 0.f, x1 = 0.f, c = 0.f;
            double t0 = 0.0;
            int ok = 0;
            if (j < nj) {
                const int64_t g = wi.par0 + j;
                z = b.z[g]; x0 = b.x0[g]; x1 = b.x1[g]; c = b.c[g]; t0 = b.t0[g];
                ok = isfinite(z) && z > -1.f && isfinite(x0) && isfinite(x1) && isfinite(c) && isfinite(t0);
                if (!ok) atomicOr(o.err, ERRBIT_PARAM);
            }
            if (!ok) { z = 0.f; x0 = 0.f; x1 = 0.f; c = 0.f; t0 = 0.0; }
            float a;
            sPm[j] = phase_map(m, z, t0, a);
            sPj[PJ_A * NJ_MAX + j] = a;
            sPj[PJ_X0 * NJ_MAX + j] = x0;
            sPj[PJ_X1 * NJ_MAX + j] = x1;
            sPj[PJ_C * NJ_MAX + j] = c;
            sPj[PJ_OK * NJ_MAX + j] = (j < nj && ok) ? 1.f : 0.f;
        }
        if (tid == 0) sMisc[2] = 0;
        for (int q = tid; q < NSLOT * NJ_MAX * NB; q += THREADS) sSlot[q] = 0.0;

        for (int64_t oc = 0; oc < nobs; oc += OBS_MAX) {
            const int nc = (int)min((int64_t)OBS_MAX, nobs - oc);
            const int64_t obase = ob0 + oc;
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
                sBand[i] = (okb && e > 0.f) ? bd : -1;
                sMjd[i] = split_f2(b.mjd[obase + i]);
                sFlux[i] = b.flux[obase + i];
                sSig[i] = e;
            }
            __syncthreads();
            if (warp == 0) {
                int *cnt = sBst + 1;
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
                    int acc = 0, np = 0;
                    for (int q = 0; q <= NB; ++q) {
                        const int v = (q < NB) ? sBst[q + 1] : 0;
                        sBst[q] = acc;
                        sBst[NB + 1 + q] = acc;
                        if (q < NB && v > 0) sPresent[np++] = q;
                        acc += v;
                    }
                    sMisc[3] = np;
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
                    if (bd >= 0) sOrd[pos[bd] + rank] = i;
                    __syncwarp();
                    if (bd >= 0 && lane == __ffs(mm) - 1) pos[bd] += __popc(mm);
                    __syncwarp();
                }
            }
            __syncthreads();

            // ---- units: (present band, group of TS samples), round-robin over warps
            const int npres = sMisc[3];
            const int ngroups = (nj + TS - 1) / TS;
            const int nunits = npres * ngroups;
            for (int u = warp; u < nunits; u += WARPS) {
                const int bi = u / ngroups, grp = u - bi * ngroups;
                const int bd = sPresent[bi];
                const int j0 = grp * TS;
                const int ns = min(TS, nj - j0);
                const int nb_obs = sBst[bd + 1] - sBst[bd];
                const int *ordb = sOrd + sBst[bd];
                const int K = m.bands.n[bd], koff = m.bands.off[bd];
                const float *lam = (bands_staged ? sLam : m.band_lam) + koff;
                const float *wk = (bands_staged ? sWk : m.band_w) + koff;

                // 1. in-grid band-sample range per sample (contiguous in k) and union window
                int kf[TS], kl[TS];
                int clo = 0x7fffffff, chi = -1;
#pragma unroll
                for (int s = 0; s < TS; ++s) {
                    kf[s] = K; kl[s] = -1;
                    if (s < ns && sPj[PJ_OK * NJ_MAX + j0 + s] != 0.f) {
                        const float a = sPj[PJ_A * NJ_MAX + j0 + s];
                        for (int k0 = 0; k0 < K; k0 += 32) {
                            const int k = k0 + lane;
                            bool in = false;
                            if (k < K) {
                                const float lr = lam[k] * a;
                                in = lr >= m.wave0 && lr <= m.wave_max;
                            }
                            const unsigned bal = __ballot_sync(0xffffffffu, in);
                            if (bal) {
                                if (kf[s] == K) kf[s] = k0 + __ffs(bal) - 1;
                                kl[s] = k0 + 31 - __clz(bal);
                            }
                        }
                        if (kf[s] <= kl[s]) {
                            int iv; float t;
                            { float iw_; wave_find(m, lam[kf[s]] * a, iv, t, iw_); }
                            clo = min(clo, fk::first_tap(iv, NW));
                            { float iw_; wave_find(m, lam[kl[s]] * a, iv, t, iw_); }
                            chi = max(chi, fk::first_tap(iv, NW) + 3);
                        }
                    }
                }
                // 2. touched phase rows (OR over lanes), compacted into rowl
                unsigned msk[NPHW / 32] = {0u, 0u, 0u, 0u};
                for (int base = 0; base < nb_obs; base += 32) {
                    const int il = base + lane;
                    if (il < nb_obs) {
                        const int i = ordb[il];
                        const float2 mj = sMjd[i];
#pragma unroll
                        for (int s = 0; s < TS; ++s) {
                            if (s >= ns || sPj[PJ_OK * NJ_MAX + j0 + s] == 0.f) continue;
                            int iv; float t, iwp, p;
                            if (phase_find(m, mj, sPm[j0 + s], iv, t, iwp, p)) {
                                const int first = fk::first_tap(iv, NP);
#pragma unroll
                                for (int q = 0; q < 4; ++q) msk[(first + q) >> 5] |= 1u << ((first + q) & 31);
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
                for (int q = lane; q < nrows * TS * 2; q += 32) {
                    const int rr = q / (TS * 2);
                    D[rowl[rr] * TS * 2 + (q - rr * TS * 2)] = 0.f;
                }
                if (GRAD)
                    for (int q = lane; q < nrows * TS; q += 32) Y[rowl[q / TS] * TS + (q % TS)] = 0.f;
                __syncwarp();
                const int nch = (chi >= clo) ? (chi - clo + WMAXW) / WMAXW : 0;

                // 3. column response and forward row dots, per column chunk
                for (int ch = 0; ch < nch; ++ch) {
                    const int cc = clo + ch * WMAXW;
                    const int W = min(WMAXW, chi - cc + 1);
                    for (int q = lane; q < W * TS; q += 32) E[q] = 0.f;
                    __syncwarp();
#pragma unroll
                    for (int s = 0; s < TS; ++s) {
                        if (s >= ns || kf[s] > kl[s]) continue;
                        const float a = sPj[PJ_A * NJ_MAX + j0 + s], c = sPj[PJ_C * NJ_MAX + j0 + s];
                        fk::ebuild(m, lam, wk, kl[s], kf[s], 32, a, c, cc, W, lane, E + s, TS);
                    }
                    __syncwarp();
                    // 4 lanes per row, 8 rows per pass, 4 columns in flight per lane
                    const int l4 = lane & 3;
                    for (int rb = 0; rb < nrows; rb += 8) {
                        const int rr = rb + (lane >> 2);
                        const bool valid = rr < nrows;
                        const int r = valid ? rowl[rr] : 0;
                        float a0[TS], a1[TS];
#pragma unroll
                        for (int s = 0; s < TS; ++s) { a0[s] = 0.f; a1[s] = 0.f; }
                        if (valid) {
                            const float2 *grow = m.g01 + (size_t)r * m.nw_pitch + cc;
                            // UF columns per lane in flight: few dependent L2 round trips per row
                            constexpr int UF = 16;
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
                                        const float e = E[col * TS + s];
                                        a0[s] = fmaf(gv[uu].x, e, a0[s]);
                                        a1[s] = fmaf(gv[uu].y, e, a1[s]);
                                    }
                                }
                            }
                        }
#pragma unroll
                        for (int s = 0; s < TS; ++s) {
                            a0[s] += __shfl_xor_sync(0xffffffffu, a0[s], 1);
                            a1[s] += __shfl_xor_sync(0xffffffffu, a1[s], 1);
                            a0[s] += __shfl_xor_sync(0xffffffffu, a0[s], 2);
                            a1[s] += __shfl_xor_sync(0xffffffffu, a1[s], 2);
                        }
                        if (valid && l4 == 0) {
#pragma unroll
                            for (int s = 0; s < TS; ++s) {
                                D[(r * TS + s) * 2] += a0[s];
                                D[(r * TS + s) * 2 + 1] += a1[s];
                            }
                        }
                    }
                    __syncwarp();
                }

                // 4. epilogue per (observation, sample): bandflux, residual, chi^2, gradient terms, adjoint rows
                double chi_acc[TS];
                float g[TS][6];
#pragma unroll
                for (int s = 0; s < TS; ++s) {
                    chi_acc[s] = 0.0;
#pragma unroll
                    for (int q = 0; q < 6; ++q) g[s][q] = 0.f;
                }
                for (int base = 0; base < nb_obs; base += 32) {
                    const int il = base + lane;
                    const bool act = il < nb_obs;
                    const int i = act ? ordb[il] : 0;
                    const float2 mj = act ? sMjd[i] : make_float2(0.f, 0.f);
                    const float zpf = act ? sZpf[i] : 0.f;
                    const float fl = (act && MODE != MODE_BANDFLUX) ? sFlux[i] : 0.f;
                    const float sig = (act && MODE != MODE_BANDFLUX) ? sSig[i] : 1.f;
#pragma unroll
                    for (int s = 0; s < TS; ++s) {
                        const int j = j0 + s;
                        Taps4 tp;
                        tp.first = -1;
                        float Bs = 0.f, Bp = 0.f, B1 = 0.f, coef = 0.f;
                        const bool okj = s < ns && sPj[PJ_OK * NJ_MAX + j] != 0.f;
                        if (act && s < ns) {
                            const float a = sPj[PJ_A * NJ_MAX + j], x0 = sPj[PJ_X0 * NJ_MAX + j];
                            const float x1 = sPj[PJ_X1 * NJ_MAX + j];
                            int iv; float t, iwp, p = 0.f;
                            if (okj && phase_find(m, mj, sPm[j], iv, t, iwp, p)) {
                                axis_taps_from<GRAD>(iv, t, NP, iwp, tp);
#pragma unroll
                                for (int mm = 0; mm < 4; ++mm) {
                                    const float2 dv = *reinterpret_cast<const float2 *>(D + ((tp.first + mm) * TS + s) * 2);
                                    const float h = fmaf(x1, dv.y, dv.x);
                                    Bs = fmaf(tp.w[mm], h, Bs);
                                    if (GRAD) {
                                        Bp = fmaf(tp.dw[mm], h, Bp);
                                        B1 = fmaf(tp.w[mm], dv.y, B1);
                                    }
                                }
                            } else {
                                tp.first = -1;
                            }
                            const float pre = x0 * a * zpf;
                            const float B = pre * Bs;
                            if (!isfinite(B)) atomicOr(o.err, ERRBIT_RANGE);
                            if (MODE == MODE_BANDFLUX) {
                                o.bandflux[wi.bf0 + (int64_t)(wi.jloc0 + j) * nobs + (oc + i)] = B;
                            } else {
                                const float r = (fl - B) / sig;
                                chi_acc[s] = fma((double)r, (double)r, chi_acc[s]);
                                if (GRAD) {
                                    const float gg = -2.0f * r / sig;
                                    g[s][0] += gg * (-a * B - pre * a * p * Bp);
                                    g[s][1] += gg * pre * Bp * (-a);
                                    g[s][2] += gg * a * zpf * Bs;
                                    g[s][3] += gg * pre * B1;
                                    coef = gg * pre;
                                }
                            }
                        }
                        if (GRAD) {
#pragma unroll
                            for (int mm = 0; mm < 4; ++mm) {
                                const bool has = tp.first >= 0;
                                const int key = has ? tp.first + mm : -1 - lane;
                                yval[lane] = has ? coef * tp.w[mm] : 0.f;
                                __syncwarp();
                                const unsigned grp = __match_any_sync(0xffffffffu, key);
                                if (has && lane == __ffs(grp) - 1) {
                                    float sum = 0.f;
                                    unsigned g2 = grp;
                                    while (g2) {
                                        sum += yval[__ffs(g2) - 1];
                                        g2 &= g2 - 1;
                                    }
                                    Y[key * TS + s] += sum;
                                }
                                __syncwarp();
                            }
                        }
                    }
                }

                // 5. reverse: Q_s[col] = sum_r Y[r][s] H_s[r][col], then per band sample adjoints
                if (GRAD) {
                    for (int ch = 0; ch < nch; ++ch) {
                        const int cc = clo + ch * WMAXW;
                        const int W = min(WMAXW, chi - cc + 1);
                        __syncwarp();
                        for (int col = lane; col < W; col += 32) {
                            float q0[TS], q1[TS];
#pragma unroll
                            for (int s = 0; s < TS; ++s) { q0[s] = 0.f; q1[s] = 0.f; }
                            const float2 *gcol = m.g01 + cc + col;
                            constexpr int UR = 16;  // rows in flight per lane
                            for (int rr0 = 0; rr0 < nrows; rr0 += UR) {
                                float2 gv[UR];
                                int rv[UR];
#pragma unroll
                                for (int uu = 0; uu < UR; ++uu) {
                                    rv[uu] = rr0 + uu < nrows ? rowl[rr0 + uu] : -1;
                                    gv[uu] = rv[uu] >= 0 ? __ldg(gcol + (size_t)rv[uu] * m.nw_pitch) : make_float2(0.f, 0.f);
                                }
#pragma unroll
                                for (int uu = 0; uu < UR; ++uu) {
                                    if (rv[uu] < 0) continue;
#pragma unroll
                                    for (int s = 0; s < TS; ++s) {
                                        const float y = Y[rv[uu] * TS + s];
                                        q0[s] = fmaf(y, gv[uu].x, q0[s]);
                                        q1[s] = fmaf(y, gv[uu].y, q1[s]);
                                    }
                                }
                            }
#pragma unroll
                            for (int s = 0; s < TS; ++s)
                                E[col * TS + s] = fmaf(sPj[PJ_X1 * NJ_MAX + j0 + min(s, ns - 1)], q1[s], q0[s]);
                        }
                        __syncwarp();
                        // adjoint of the column response per band sample (E now holds Q)
#pragma unroll
                        for (int s = 0; s < TS; ++s) {
                            if (s >= ns || kf[s] > kl[s]) continue;
                            const float a = sPj[PJ_A * NJ_MAX + j0 + s], c = sPj[PJ_C * NJ_MAX + j0 + s];
                            fk::eadjoint(m, lam, wk, kl[s], kf[s], 32, a, c, cc, W, lane, E + s, TS, g[s][4], g[s][5]);
                        }
                        __syncwarp();
                    }
                }

                // 6. unit partials -> slot[sample][band index]
                if (MODE != MODE_BANDFLUX) {
#pragma unroll
                    for (int s = 0; s < TS; ++s) {
                        const double x2 = warp_sum_d(chi_acc[s]);
                        float gs[6];
#pragma unroll
                        for (int q = 0; q < 6; ++q) gs[q] = GRAD ? warp_sum(g[s][q]) : 0.f;
                        if (lane == 0 && s < ns) {
                            double *sl = sSlot + ((size_t)(j0 + s) * NB + bd) * NSLOT;
                            sl[0] += x2;
#pragma unroll
                            for (int q = 0; q < 6; ++q) sl[1 + q] += gs[q];
                        }
                    }
                }
                __syncwarp();
            }  // units
        }  // observation chunks

        __syncthreads();
        if (MODE != MODE_BANDFLUX) {
            if (tid < nj) {
                const int j = tid;
                double x2 = 0.0;
                float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int bd = 0; bd < NB; ++bd) {  // band order, absent bands hold zeros
                    const double *sl = sSlot + ((size_t)j * NB + bd) * NSLOT;
                    x2 += sl[0];
#pragma unroll
                    for (int q = 0; q < 6; ++q) g[q] += (float)sl[1 + q];
                }
                const bool bad = sPj[PJ_OK * NJ_MAX + j] == 0.f || sMisc[2] != 0;
                const int64_t gj = wi.par0 + j;
                o.chi2[gj] = bad ? __longlong_as_double(0x7ff8000000000000ll) : x2;
                if (GRAD) {
                    const float gout[5] = {g[0] + g[5], g[1], g[2], g[3], g[4]};
#pragma unroll
                    for (int q = 0; q < 5; ++q) o.grad[5 * gj + q] = bad ? fk::qnanf() : gout[q];
                }
            }
        } else {
            for (int j = 0; j < nj; ++j) {
                const bool bad = sPj[PJ_OK * NJ_MAX + j] == 0.f || sMisc[2] != 0;
                if (bad)
                    for (int64_t i = tid; i < nobs; i += THREADS)
                        o.bandflux[wi.bf0 + (int64_t)(wi.jloc0 + j) * nobs + i] = fk::qnanf();
            }
        }
    }
}

}  // namespace bw

int bandwarp_item_samples() { return bw::NJ_MAX; }
int bandwarp_max_phase() { return bw::NPHW; }

template <int TS, int MODE>
static cudaError_t launch_bw(const salt_ctx *ctx, const WorkItem *items_d, int n_items, int *counter_d,
                             const BatchDev &b, const OutDev &o, cudaStream_t st) {
    const int nb = ctx->mp.bands.n_bands;
    const size_t smem = bw::Lay(TS, MODE == MODE_GRAD, nb).total;
    static std::atomic<int> attr_done[64];
    cudaError_t e;
    const int dv = ctx->device & 63;
    if (!attr_done[dv].load()) {
        e = cudaFuncSetAttribute(bw::k_bandwarp<TS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bw::Lay(TS, MODE == MODE_GRAD, SALT_MAX_BANDS).total);
        if (e != cudaSuccess) return e;
        attr_done[dv].store(1);
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bw::k_bandwarp<TS, MODE>, bw::THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = ctx->num_sms * per_sm;
    if (grid > n_items) grid = n_items;
    if (grid < 1) return cudaSuccess;
    e = cudaMemsetAsync(counter_d, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    bw::k_bandwarp<TS, MODE><<<grid, bw::THREADS, smem, st>>>(ctx->mp, b, o, items_d, n_items, counter_d);
    return cudaGetLastError();
}

cudaError_t launch_bandwarp_items(const salt_ctx *ctx, int ts, const WorkItem *items_d, int n_items,
                                  int *counter_d, const BatchDev &b, const OutDev &o, int mode,
                                  cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (ts == 2) {
        switch (mode) {
            case MODE_BANDFLUX: return launch_bw<2, MODE_BANDFLUX>(ctx, items_d, n_items, counter_d, b, o, st);
            case MODE_CHI2: return launch_bw<2, MODE_CHI2>(ctx, items_d, n_items, counter_d, b, o, st);
            default: return launch_bw<2, MODE_GRAD>(ctx, items_d, n_items, counter_d, b, o, st);
        }
    }
    switch (mode) {
        case MODE_BANDFLUX: return launch_bw<1, MODE_BANDFLUX>(ctx, items_d, n_items, counter_d, b, o, st);
        case MODE_CHI2: return launch_bw<1, MODE_CHI2>(ctx, items_d, n_items, counter_d, b, o, st);
        default: return launch_bw<1, MODE_GRAD>(ctx, items_d, n_items, counter_d, b, o, st);
    }
}

}  // namespace salt
