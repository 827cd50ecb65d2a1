// Internal types shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "salt.h"

namespace salt {

// Error bits a kernel records in the context's device error word.
// Sticky error word bits set by the kernels (read and cleared by salt_check).
// RANGE: a bandflux came out non-finite from finite parameters (FP32 overflow of
// the colour factor or the surfaces, or a non-finite zero point).
enum : int { ERRBIT_BAND = 1, ERRBIT_SIGMA = 2, ERRBIT_PARAM = 4, ERRBIT_RANGE = 8 };

// Band table passed by value to every kernel (fits the kernel parameter space).
struct BandTable {
    int n_bands;
    int k_total;  // length of the flat arrays: every band's samples, each band padded to an even length
    int off[SALT_MAX_BANDS];  // first sample of band b in the flat arrays (even)
    int n[SALT_MAX_BANDS];    // samples in band b
    float lam_lo[SALT_MAX_BANDS], lam_hi[SALT_MAX_BANDS];  // first / last observer wavelength
};

// Model constants in the form the kernels use (FP32, derived on the host in FP64).
struct ModelParams {
    int n_phase, n_wave;
    int nw_pitch;  // row pitch of g01 in float2 (n_wave rounded up to even: 16-byte aligned rows)
    float phase0, inv_dphase, phase_max;
    float dphase;                   // uniform phase step (for the phase itself, gradient terms)
    double phase0_d, inv_dphase_d;  // the same in FP64 (per-sample phase maps)
    float wave0, inv_dwave, wave_max, dwave;
    // colour law: P(x) = sum_{m=1..5} p[m-1] x^m, x = (lambda - lamB) * inv_span
    float cl_p[5];
    float cl_lamB, cl_inv_span, cl_lo, cl_hi;
    float cl_xlo, cl_Plo, cl_dPlo, cl_xhi, cl_Phi, cl_dPhi;
    const float2 *__restrict__ g01;      // [n_phase][nw_pitch] interleaved (M0, M1)
    const float *__restrict__ band_lam;  // flat band wavelengths (observer frame)
    const float *__restrict__ band_w;    // flat weights lambda T Delta / (h c Z_b)
    // non-uniform axes (NULL = uniform): node positions and 1/(node[i+1] - node[i])
    const float *__restrict__ pnode;
    const float *__restrict__ pinv;
    const float *__restrict__ pnode_lo;  // node - (float)node: phase nodes as float pairs
    const float *__restrict__ wnode;
    const float *__restrict__ winv;
    BandTable bands;
};

// Device view of a batch (all pointers device-resident).
struct BatchDev {
    int64_t n_sn, n_obs, n_par;
    const int64_t *__restrict__ obs_off;
    const int64_t *__restrict__ par_off;
    const double *__restrict__ mjd;
    const int32_t *__restrict__ band;
    const float *__restrict__ flux;
    const float *__restrict__ fluxerr;
    const float *__restrict__ zp;
    const double *__restrict__ t0;
    const float *__restrict__ z;
    const float *__restrict__ x0;
    const float *__restrict__ x1;
    const float *__restrict__ c;
};

enum Mode : int { MODE_BANDFLUX = 0, MODE_CHI2 = 1, MODE_GRAD = 2 };

struct OutDev {
    float *bandflux;                // [bf_off[n_sn]]
    const int64_t *bf_off;          // [n_sn + 1]
    double *chi2;                   // [n_par]
    float *grad;                    // [n_par][5]
    int *err;                       // sticky error word
};

// One unit of work for the fused factorised kernel: one supernova's
// observations [obs0, obs0 + nobs) against parameter samples
// [par0, par0 + nj); jloc0 is the local index of sample par0 within its
// supernova and bf0 the supernova's first bandflux slot (bandflux mode).
struct WorkItem {
    int64_t obs0, par0, bf0;
    int32_t nobs, nj, jloc0, pad;
};

// Launch configurations of the factorised path: kernel family and tile.
enum Family : int { FAM_CTA = 0, FAM_WARP = 1, FAM_UNIT = 2 };
inline int cfg_key(int family, int tile) { return family * 32 + tile; }  // tile <= 16
inline int cfg_family(int key) { return key / 32; }
inline int cfg_tile(int key) { return key % 32; }

}  // namespace salt

struct salt_plan {
    salt_ctx *ctx = nullptr;  // identity check only; never dereferenced after creation
    int device = 0;
    int64_t n_sn = 0, n_obs = 0, n_par = 0, n_bandflux = 0;
    std::vector<int64_t> obs_off_h, par_off_h, bf_off_h;
    int64_t *obs_off_d = nullptr, *par_off_d = nullptr, *bf_off_d = nullptr;
    // work lists, one per launch configuration (family, tile), built on demand
    struct ItemList {
        salt::WorkItem *d = nullptr;
        int n = 0;
        void *scratch = nullptr;  // per-item partials + arrival counters (warp-unit family)
    };
    std::map<int, ItemList> lists;
    int choice[3] = {-1, -1, -1};  // tuned configuration key per mode (-1 = not tuned yet)
    int band_gen = 0;               // the context's band generation the work state was built for
    int *counter_d = nullptr;      // dynamic work counter of the persistent kernels
    bool temporary = false;
    // Captured CUDA graphs per (mode, launch configuration), for up to kGraphSlots
    // sets of batch and output pointers (a caller alternating buffers keeps
    // every set): a set's first call launches directly and records its pointers,
    // the graph is captured when the same pointers come back, and the least
    // recently used set makes room for a new one.
    static constexpr int kGraphSlots = 4;
    struct GraphEntry {
        salt::BatchDev b{};
        salt::OutDev o{};
        bool seen = false;     // b/o hold a call's pointers
        uint64_t used = 0;     // last use (set tick)
        cudaGraphExec_t exec = nullptr;
    };
    struct GraphSet {
        GraphEntry e[kGraphSlots];
        bool failed = false;   // a capture failed once: launch directly from then on
        uint64_t tick = 0;
    };
    std::map<int, GraphSet> graphs;
};

namespace salt {
struct ServeEngine;
}

struct salt_ctx {
    int device = 0;
    int num_sms = 0;
    salt::ModelParams mp{};
    float2 *g01_d = nullptr;
    float *band_lam_d = nullptr, *band_w_d = nullptr;
    float *nodes_d = nullptr;  // non-uniform axes: phase nodes, inverse widths, wave nodes, inverse widths
    int *err_d = nullptr;
    std::string last_error;
    int kernel = SALT_KERNEL_AUTO;
    int tile_samples = 0;  // 0 = autotuned
    int use_graphs = 1;
    int serve_chunk = 8;  // samples per serving work item (latency: one 8-sample tile per item)
    int last_kernel = 0;   // SALT_KERNEL_* x 32 + tile of the last batch launch (0 = none yet)
    cudaStream_t capture_stream = nullptr;  // private stream for graph capture (created on first use)
    std::vector<double> host_cl;  // colour-law coefficients (for serving validation)
    std::vector<float> host_lam, host_w;  // band tables as uploaded (for registering bands)
    int band_gen = 0;             // bumped by every band registration
    salt::ServeEngine *serve = nullptr;
    size_t serve_mem = 0;
    std::mutex mu;  // guards last_error for serve_* callers
};

namespace salt {

// Launchers (kernels.cu).
cudaError_t launch_direct(const salt_ctx *ctx, const BatchDev &b, const OutDev &o, int mode,
                          cudaStream_t st);

cudaError_t launch_factorised_items(const salt_ctx *ctx, int tile, const WorkItem *items_d, int n_items,
                                    int *counter_d, const BatchDev &b, const OutDev &o, int mode,
                                    cudaStream_t st);
cudaError_t launch_bandwarp_items(const salt_ctx *ctx, int ts, const WorkItem *items_d, int n_items,
                                  int *counter_d, const BatchDev &b, const OutDev &o, int mode,
                                  cudaStream_t st);
int bandwarp_item_samples();
int bandwarp_max_phase();
// n_items_dev (optional): device int read by the kernel as the list's length
// (clamped to n_items, which sizes the grid and the scratch).
cudaError_t launch_unit_items(const salt_ctx *ctx, int ts, const WorkItem *items_d, int n_items, int *counter_d,
                              void *scratch, const BatchDev &b, const OutDev &o, int mode, cudaStream_t st,
                              const int *n_items_dev = nullptr);
int unit_max_phase();
size_t unit_scratch_bytes(int n_items, int ts, int n_bands);
cudaError_t launch_validate(const salt_ctx *ctx, const BatchDev &b, int *flag, cudaStream_t st);
int factorised_smem_bytes(int tile, int mode);
int factorised_max_tile();

// Serving engine (serve.cu).
ServeEngine *serve_create(salt_ctx *ctx, size_t mem_limit);
void serve_destroy(ServeEngine *e);
int serve_submit(ServeEngine *e, const salt_request *req, uint64_t *ticket);
int serve_poll(ServeEngine *e, uint64_t ticket, int32_t wait_ms, double *chi2, float *grad);
int serve_cancel(ServeEngine *e, uint64_t ticket);
int serve_stats(ServeEngine *e, salt_serve_stats *out);

// Host helpers (api.cu).
int plan_build(salt_ctx *ctx, int64_t n_sn, const int64_t *obs_off, const int64_t *par_off,
               int tile, salt_plan *p, cudaStream_t st, bool async_alloc);
void plan_free(salt_plan *p, cudaStream_t st);
int run_batch(salt_ctx *ctx, const BatchDev &b, const salt_plan *plan, const OutDev &o, int mode,
              cudaStream_t st);
// The plan with one fixed configuration (no autotuning, no graph replay).
int run_batch_fixed(salt_ctx *ctx, const BatchDev &b, salt_plan *p, const OutDev &o, int mode, cudaStream_t st,
                    int family, int tile);

}  // namespace salt
