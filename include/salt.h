/*
 * salt.h - C ABI of the B300 (sm_103a) batched SALT synthetic-photometry library.
 *
 * What is computed (JAX-bandflux, arXiv:2504.08081, Implementation section):
 *   SALT model form, Eq. 1:
 *       F(p, lambda) = x0 [M0(p, lambda) + x1 M1(p, lambda)] * 10^(-0.4 c CL(lambda))
 *     (the paper's exp[c CL] with its CL = -0.4 ln10 times this CL), where the
 *     free parameters are x0, x1, t0 and c; p = (t - t0)/(1 + z) is the
 *     rest-frame phase and lambda = lambda_obs/(1 + z) the rest wavelength; the
 *     observer-frame flux density is F/(1 + z).
 *   Bandflux, Eq. 2:  integral F(lambda) T(lambda) lambda/(h c) dlambda, taken
 *     with the trapezoidal rule on the band's own samples (paragraph after
 *     Eq. 2), scaled to the observation's AB zero point by 10^(0.4 zp) / Z_b
 *     where Z_b is the same integral of the 3631 Jy AB spectrum.
 *   chi^2 = sum_i ((flux_i - bandflux_i) / fluxerr_i)^2 per parameter sample,
 *     and its gradient with respect to (z, t0, x0, x1, c) (the paper's claim
 *     of gradient propagation through the whole pipeline, Implementation,
 *     last paragraph).
 *   M0/M1 are interpolated with tensor-product Keys cubic convolution
 *   (a = -1/2; linear on the first and last interval of each axis; zero
 *   outside the grid): the paper's "dedicated interpolation routines". The
 *   colour law is the SALT2 polynomial with linear extrapolation outside
 *   [cl_lo, cl_hi].
 *
 * Conventions for every call:
 *   - Status codes are returned; no C++ exception crosses this boundary. The
 *     text of the last error on a context is available from salt_last_error.
 *   - Batch calls are asynchronous on the caller's CUDA stream (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - The caller owns every batch array and every output buffer. The library
 *     owns everything reachable from a salt_ctx or a salt_plan.
 *   - Precision: FP32 arithmetic, except the epoch difference t - t0 (FP64,
 *     MJD values) and the chi^2 accumulation (FP64).
 *   - Thread safety: batch calls on one context from one thread at a time;
 *     salt_serve_* calls are safe from any thread.
 */
#ifndef SALT_H
#define SALT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SALT_ABI_VERSION 1
#define SALT_MAX_BANDS 64

typedef enum {
    SALT_OK = 0,
    SALT_PENDING = 1,          /* serving: request not finished yet */
    SALT_ERR_INVALID = -1,     /* argument or data failed validation */
    SALT_ERR_OOM = -2,         /* device or host allocation failed, or can never fit */
    SALT_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    SALT_ERR_TIMEOUT = -4,     /* serving: wait_ms elapsed */
    SALT_ERR_NOT_FOUND = -5,   /* serving: unknown or already collected ticket */
    SALT_ERR_CANCELLED = -6,   /* serving: request was cancelled */
    SALT_ERR_DATA = -7         /* a kernel met invalid batch data (see salt_check) */
} salt_status;

typedef struct salt_ctx salt_ctx;
typedef struct salt_plan salt_plan;

/* ---------------------------------------------------------------- model --- */

/* Model grid (Eq. 1 surfaces). HOST pointers, copied.
 *   phase axis: phase0 + r*dphase, r < n_phase (days); wave axis: wave0 +
 *   j*dwave, j < n_wave (Angstrom). n_phase, n_wave >= 4.
 *   m0, m1: row-major [n_phase][n_wave] float32.
 *   cl: n_cl == 4 colour-law coefficients a1..a4 of
 *       P(x) = (1 - sum a) x + a1 x^2 + a2 x^3 + a3 x^4 + a4 x^5,
 *       x = (lambda - 4302.57)/(5428.55 - 4302.57), CL = -P on [cl_lo, cl_hi],
 *       linear continuation outside.
 *   phase_nodes [n_phase], wave_nodes [n_wave]: optional non-uniform axes
 *       (SALT3-NIR-style grids; the paper's "dedicated interpolation
 *       routines", Implementation, last but one paragraph): strictly
 *       ascending finite node positions; when given, phase0/dphase (or
 *       wave0/dwave) are ignored. A coordinate is located by binary search
 *       and the Keys weights apply to its fraction of the local interval
 *       (index space); derivatives carry 1/(local interval width). NULL =
 *       the uniform axis. */
typedef struct {
    int32_t n_phase, n_wave;
    double phase0, dphase, wave0, dwave;
    const float *m0, *m1;
    int32_t n_cl;
    const double *cl;
    double cl_lo, cl_hi;
    const double *phase_nodes, *wave_nodes;
} salt_model_desc;

/* A bandpass (paper: Bandpass / register_bandpass): n >= 2 samples of
 * strictly ascending wavelength (Angstrom) and transmission. HOST, copied. */
typedef struct {
    int32_t n;
    const double *wave, *trans;
} salt_band_desc;

/* Create a context on CUDA device `device`: uploads the grids, registers the
 * bands (band id = index in `bands`, n_bands <= SALT_MAX_BANDS), precomputes
 * the trapezoid weights lambda T Delta/(h c Z_b) in FP64 on the host and
 * rounds them to float32. serve_mem_bytes bounds the device memory the serving
 * engine may hold for admitted requests (0 = no serving engine).
 * Returns SALT_ERR_INVALID for a non-finite grid, axes with n < 4 or a
 * non-positive step, bands with n < 2 or non-ascending wavelengths;
 * SALT_ERR_CUDA / SALT_ERR_OOM on device failures. *out is NULL on error. */
int salt_init_model(const salt_model_desc *model, const salt_band_desc *bands, int32_t n_bands,
                    int32_t device, size_t serve_mem_bytes, salt_ctx **out);

/* Stop the serving engine (pending requests are cancelled), free everything. */
void salt_destroy(salt_ctx *ctx);

/* Register one more bandpass on a live context (the paper's
 * register_bandpass, Implementation, paragraph on bandpasses.py). Same rules
 * and weights as a band passed to salt_init_model; *band_id = its id (the
 * previous band count). Not concurrently with other calls on the context;
 * waits for device work that may read the old band tables. Plans made before
 * drop their work lists, scratch, tuned choices and captured graphs on their
 * next use (which then must not be inside a stream capture).
 * SALT_ERR_INVALID for a bad band or a full registry (SALT_MAX_BANDS). */
int salt_register_band(salt_ctx *ctx, const salt_band_desc *band, int32_t *band_id);

/* Read a bandpass from a text file (the paper's load_bandpass_from_file).
 * One sample per line: wavelength and transmission separated by blanks, tabs
 * or a comma (further columns ignored); '#' starts a comment; blank lines are
 * skipped. Wavelengths are multiplied by wave_scale (1 for Angstrom, 10 for
 * nm) and must be finite, positive and strictly ascending; at least 2 samples.
 * step > 0 resamples the curve, taken as piecewise linear between its samples,
 * at the multiples of step inside [first, last wavelength]; step = 0 keeps
 * the file's samples. Host only (no device work).
 *   wave, trans: HOST float64 [capacity] out; *n: the number of samples.
 *   wave = trans = NULL with capacity = 0 only sets *n (size query).
 *   ctx: optional, receives the error text for salt_last_error.
 * SALT_ERR_INVALID for an unreadable or malformed file, bad arguments, or a
 * capacity below *n. */
int salt_band_load(salt_ctx *ctx, const char *path, double wave_scale, double step, double *wave,
                   double *trans, int32_t capacity, int32_t *n);

/* ---------------------------------------------------------------- batches - */

/* A ragged batch (the paper's vmap over data instances, Implementation,
 * paragraph after Eq. 2). Supernova s owns observations [obs_off[s],
 * obs_off[s+1]) and parameter samples [par_off[s], par_off[s+1]).
 *   obs_off, par_off: HOST int64 [n_sn + 1], nondecreasing, starting at 0.
 *   mjd[n_obs] (FP64), band[n_obs] (band id), flux, fluxerr (> 0), zp (AB):
 *     DEVICE arrays.
 *   t0[n_par] (FP64, MJD), z (> -1), x0, x1, c [n_par]: DEVICE arrays.
 *   plan: optional, from salt_plan_create with the same offsets (saves the
 *     host-side planning and the offset upload on every call); NULL = plan
 *     on the fly.
 *   validate: nonzero = check band ids, fluxerr > 0 and finite parameters on
 *     the device first and return SALT_ERR_INVALID (outputs untouched) if any
 *     fails; this synchronises the stream. With validate = 0 the kernels still
 *     never read out of bounds: an observation with a bad band id or
 *     fluxerr <= 0 makes its sample's outputs NaN and records SALT_ERR_DATA,
 *     reported by salt_check. */
typedef struct {
    int64_t n_sn;
    const int64_t *obs_off;
    const int64_t *par_off;
    const double *mjd;
    const int32_t *band;
    const float *flux, *fluxerr, *zp;
    const double *t0;
    const float *z, *x0, *x1, *c;
    const salt_plan *plan;
    int32_t validate;
} salt_batch;

/* Precompute the launch plan for a batch layout (host CSR offsets): device
 * copies of the offsets and, on first use, the cost-sorted work lists of
 * (supernova, sample-range) items. Reusable for every batch with the same
 * offsets (parameters and observation values may change between calls).
 * With SALT_KERNEL_AUTO the first batch call of each mode on a plan
 * autotunes: it times every candidate kernel family / tile on that batch,
 * synchronising the stream, and keeps the fastest (cached per layout for the
 * process, and appended to the file named by SALT_TUNE_CACHE if set). A plan
 * must not be used from two threads at once. */
int salt_plan_create(salt_ctx *ctx, int64_t n_sn, const int64_t *obs_off, const int64_t *par_off,
                     salt_plan **out);
void salt_plan_destroy(salt_plan *plan);

/* Offsets of the bandflux output: bf_off[s] = sum_{s'<s} n_obs(s') n_par(s'),
 * bf_off[n_sn] = total. HOST in, HOST out ([n_sn + 1]). */
int salt_bandflux_offsets(int64_t n_sn, const int64_t *obs_off, const int64_t *par_off,
                          int64_t *bf_off);

/* Bandflux (Eq. 2, zero-point scaled) of every (sample, observation) pair of
 * every supernova: out[bf_off[s] + j*n_obs(s) + i] for local sample j and
 * local observation i. out: DEVICE float32 [bf_off[n_sn]] (may be NULL when
 * bf_off[n_sn] = 0). */
int salt_bandflux(salt_ctx *ctx, const salt_batch *batch, float *out, void *cuda_stream);

/* chi^2 of every parameter sample against its supernova's observations.
 * chi2: DEVICE float64 [n_par]. */
int salt_chi2(salt_ctx *ctx, const salt_batch *batch, double *chi2, void *cuda_stream);

/* chi^2 and its gradient d chi^2 / d(z, t0, x0, x1, c) (hand-written adjoint).
 * chi2: DEVICE float64 [n_par]; grad: DEVICE float32 [n_par][5]. A gradient
 * component beyond the float32 range (|d chi^2/d x0| ~ chi^2 / x0 passes 3.4e38
 * once chi^2 ~ 1e36 at x0 ~ 1e-5) comes out as +-inf with a finite chi^2;
 * salt_check does not report it. */
int salt_chi2_grad(salt_ctx *ctx, const salt_batch *batch, double *chi2, float *grad,
                   void *cuda_stream);

/* Synchronise `cuda_stream` and report SALT_ERR_DATA if any kernel since the
 * last salt_check met invalid batch data or produced a non-finite bandflux
 * from finite parameters (FP32 overflow: a colour factor 10^(-0.4 c CL) or
 * surface values beyond ~3e38; salt_last_error says which), the sticky flag
 * then being cleared; SALT_ERR_CUDA on an asynchronous CUDA error; else
 * SALT_OK. */
int salt_check(salt_ctx *ctx, void *cuda_stream);

/* ---------------------------------------------------------------- options - */

typedef enum {
    SALT_OPT_KERNEL = 1,       /* SALT_KERNEL_* : which kernel family batch calls use */
    SALT_OPT_TILE_SAMPLES = 2, /* samples per tile for the forced kernel families: 1, 2, 4, 8, 16
                                  (CTA family; the warp families take 1 or 2) or 0 = default */
    SALT_OPT_GRAPHS = 3,       /* 1 (default) = a plan call repeated with the same batch and output
                                  pointers, mode and kernel is captured into a CUDA graph once and
                                  replayed on later such calls (up to four pointer sets per plan,
                                  mode and kernel are remembered, so alternating buffers replay
                                  too); 0 = always launch directly */
    SALT_OPT_SERVE_CHUNK = 4,  /* serving: samples per work item (default 8; larger chunks
                                  cut per-item overhead but lengthen each item's latency) */
    SALT_OPT_LAST_KERNEL = 5   /* read-only: SALT_KERNEL_* x 32 + samples per tile of the kernel
                                  the last batch call on this context launched (0 = none yet) */
} salt_option;

typedef enum {
    SALT_KERNEL_AUTO = 0,        /* factorised path; family and tile autotuned per plan and mode */
    SALT_KERNEL_DIRECT = 1,      /* per-band-sample evaluation straight from Eq. 1-2 */
    SALT_KERNEL_FACTORISED = 2,  /* factorised, CTA-cooperative per (sample tile, band) */
    SALT_KERNEL_BANDWARP = 3,    /* factorised, one warp per (band, 1-2 samples); <= 128 phase nodes */
    SALT_KERNEL_UNIT = 4         /* factorised, warps pull (supernova, band, 1-2 samples) units from a
                                    global counter; per-band partials combined in band order through
                                    plan-owned scratch memory; <= 128 phase nodes */
} salt_kernel;

int salt_set_option(salt_ctx *ctx, int32_t option, int64_t value);
int salt_get_option(const salt_ctx *ctx, int32_t option, int64_t *value);

/* ---------------------------------------------------------------- serving - */

/* One serving request: one supernova, its observations and n_par parameter
 * samples. HOST pointers; the library copies them at submit. */
typedef struct {
    int32_t n_obs, n_par, want_grad;
    const double *mjd;
    const int32_t *band;
    const float *flux, *fluxerr, *zp;
    const double *t0;
    const float *z, *x0, *x1, *c;
} salt_request;

/* Queue a request for continuous batching. Returns SALT_ERR_INVALID for bad
 * data (validated on the host), SALT_ERR_OOM if it can never fit in the
 * serving memory budget. *ticket identifies it for poll/cancel. */
int salt_serve_submit(salt_ctx *ctx, const salt_request *req, uint64_t *ticket);

/* Wait up to wait_ms (0 = do not wait, < 0 = forever) for a request.
 * SALT_OK: results copied to chi2 (HOST float64 [n_par]) and, if requested,
 * grad (HOST float32 [n_par][5]); the ticket is then released.
 * SALT_PENDING / SALT_ERR_TIMEOUT: not finished. SALT_ERR_CANCELLED,
 * SALT_ERR_NOT_FOUND, SALT_ERR_CUDA otherwise. */
int salt_serve_poll(salt_ctx *ctx, uint64_t ticket, int32_t wait_ms, double *chi2, float *grad);

/* Cancel a queued or running request; its memory is released when any
 * in-flight work on it completes. */
int salt_serve_cancel(salt_ctx *ctx, uint64_t ticket);

typedef struct {
    uint64_t submitted, completed, cancelled, rejected;
    uint64_t launches;            /* fused kernel launches issued by the engine */
    uint64_t queued, active;      /* current queue depth and admitted requests */
    size_t mem_in_use, mem_limit; /* admitted device bytes and the budget */
    double p50_ms, p99_ms;        /* submit -> result-ready latency over completed requests */
} salt_serve_stats;

int salt_serve_stats_get(salt_ctx *ctx, salt_serve_stats *out);

/* ---------------------------------------------------------------- fitting - */

/* Parameters a fit may move (bit i = gradient component i). */
#define SALT_FIT_Z 1
#define SALT_FIT_T0 2
#define SALT_FIT_X0 4
#define SALT_FIT_X1 8
#define SALT_FIT_C 16
#define SALT_FIT_DEFAULT_MASK (SALT_FIT_T0 | SALT_FIT_X0 | SALT_FIT_X1 | SALT_FIT_C)

/* Per-supernova fit outcome. status[s] >= 0: converged after that many
 * accepted steps, either with the projected scaled gradient's inf-norm pg
 * <= gtol, or with chi^2 flat (an accepted step lowering it by <= ftol
 * relative, or eight in a row lowering it together by no more than its FP32
 * resolution, 2e-6 relative) while pg <= 100 gtol. A flat chi^2 with a larger
 * pg drops the L-BFGS curvature pairs and goes on along steepest descent; the
 * fourth such flat stretch ends the fit with SALT_FIT_FLAT. */
#define SALT_FIT_MAXITER (-1)    /* max_iter steps or max_evals evaluations used */
#define SALT_FIT_LINESEARCH (-2) /* no step lowers chi^2 any more (at the precision floor) */
#define SALT_FIT_INVALID (-3)    /* non-finite chi^2 at the start, or an empty box */
#define SALT_FIT_FLAT (-4)       /* chi^2 flat after three steepest-descent restarts while
                                    pg stayed above 100 gtol: stopped, not converged */

/* Options of salt_fit; zero fields take the defaults. */
typedef struct {
    int32_t max_iter;   /* accepted steps per fit (default 300) */
    int32_t max_evals;  /* chi^2 evaluations per fit (default 2 x max_iter + 20) */
    int32_t history;    /* L-BFGS memory, 1..8 pairs (default 6) */
    int32_t free_mask;  /* SALT_FIT_* bits of the fitted parameters (default t0, x0, x1, c) */
    double gtol;        /* stop when the inf-norm of the projected gradient in scaled
                           variables is <= gtol (default 1e-3) */
    double ftol;        /* an accepted step lowering chi^2 by <= ftol relative counts as
                           a flat chi^2 (default 1e-10): the fit ends there only if
                           pg <= 100 gtol (see the statuses above) */
} salt_fit_opts;

/* Fit the SALT parameters of every supernova of a batch independently by
 * minimising its chi^2 (the paper's L-BFGS-B optimisation of x0, x1, t0 and c,
 * Implementation, first paragraph), all supernovae in lockstep on the device.
 * Method: bound-constrained limited-memory BFGS in scaled variables
 * (z/0.01, t0/1 d, x0/|x0 start|, x1, c/0.1): two-loop direction over the
 * variables not pinned at a bound, steps capped at the box, a strong Wolfe
 * line search (c1 = 1e-4, c2 = 0.9; bracketing and cubic zoom); each
 * evaluation is one batched salt_chi2_grad-equivalent pass over every
 * supernova's trial point.
 *   batch: exactly one parameter sample per supernova (par_off[s] = s); the
 *     parameter arrays hold the starting point; validate is ignored.
 *   lower, upper: DEVICE float64 [n_sn][5] (z, t0, x0, x1, c) box, or NULL for
 *     unbounded; parameters outside free_mask stay at their start values; a
 *     free z is kept >= -0.99.
 *   theta: DEVICE float64 [n_sn][5] out, the best point found (FP32-rounded
 *     values for z, x0, x1, c: the values the chi^2 was evaluated at);
 *   chi2: DEVICE float64 [n_sn] out, chi^2 at theta; status: DEVICE int32
 *     [n_sn] out (>= 0 or SALT_FIT_*).
 * Synchronises cuda_stream (the host checks progress every 8 iterations).
 * Allocates its scratch (about 1.2 KB per supernova) for the call.
 * Returns SALT_ERR_INVALID for bad arguments, SALT_ERR_CUDA/OOM on device
 * failures. */
int salt_fit(salt_ctx *ctx, const salt_batch *batch, const double *lower, const double *upper,
             const salt_fit_opts *opts, double *theta, double *chi2, int32_t *status,
             void *cuda_stream);

/* ------------------------------------------------------- nested sampling - */

/* Options of salt_nested; zero fields take the defaults. */
typedef struct {
    int32_t n_live;     /* live points per supernova (default 256; 2..1024) */
    int32_t n_batch;    /* live points replaced per iteration (default n_live / 4; < n_live) */
    int32_t n_steps;    /* random-walk steps per replacement (default 20) */
    int32_t max_iter;   /* iterations (default 2000) */
    int32_t free_mask;  /* SALT_FIT_* bits of the sampled parameters (default t0, x0, x1, c) */
    int32_t reserved;   /* 0 */
    uint64_t seed;      /* Philox4x32-10 key */
    double dlogz;       /* stop when the live points could add < dlogz to log Z (default 0.1) */
} salt_nested_opts;

/* Nested sampling of every supernova's posterior and evidence (the paper's
 * nested-sampling example, Implementation, first paragraph), all supernovae
 * in lockstep on the device. Likelihood L = exp(-chi^2/2) (the library's
 * chi^2), prior uniform in the box [lower, upper] of the sampled parameters.
 * Per iteration the n_batch lowest live points are removed (the j-th removal
 * with N - j points live shrinks log X by 1/(N - j)) and replaced by the end
 * points of n_batch random-walk chains (n_steps steps each, started at
 * survivors picked uniformly; step = f * survivors' standard deviation *
 * standard normal; accepted inside the box above the last removed log L;
 * f *= exp(acceptance - 1/2) per iteration, clipped to [1e-3, 10]). Random
 * numbers: Philox4x32-10 with the seed as key (Salmon et al., SC'11), so a
 * seed reproduces a run; every chi^2 evaluation uses the CTA-factorised
 * kernel at a fixed tile.
 *   batch: one sample per supernova (par_off[s] = s) holding the values of
 *     the parameters that are not sampled (z, usually); validate ignored.
 *   lower, upper: DEVICE float64 [n_sn][5] prior box (finite for sampled
 *     parameters).
 *   logz, logz_err (sqrt(H / n_live)): DEVICE float64 [n_sn] out; mean, std:
 *     DEVICE float64 [n_sn][5] out (posterior moments); status: DEVICE int32
 *     [n_sn] out (iterations used, SALT_FIT_MAXITER, or SALT_FIT_INVALID for
 *     an empty or non-finite box).
 * Synchronises cuda_stream; allocates its scratch (about 60 x n_live bytes
 * per supernova plus the chains) for the call. */
int salt_nested(salt_ctx *ctx, const salt_batch *batch, const double *lower, const double *upper,
                const salt_nested_opts *opts, double *logz, double *logz_err, double *mean, double *std,
                int32_t *status, void *cuda_stream);

/* ------------------------------------------------- no-allocation variant - */

/* Bytes of device scratch available to salt_chi2_grad_noalloc: one fixed
 * array inside the library per device (held from module load on). */
#define SALT_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* salt_chi2_grad without any device-memory allocation during the call. The
 * paper has no counterpart: it is a service for callers that cannot allocate,
 * e.g. a process whose device memory is all reserved by another allocator's
 * pool (a caching allocator that has taken the free HBM), or a fitting loop
 * that cannot afford the stalls of allocation (cudaFree synchronises the
 * device). Same arguments, outputs (chi2: DEVICE float64 [n_par]; grad:
 * DEVICE float32 [n_par][5]) and data errors as salt_chi2_grad; it always
 * runs the warp-unit kernel with one sample per unit (SALT_KERNEL_UNIT,
 * tile 1) and ignores batch->plan and the kernel options.
 * Scratch: the offset copies, the work list, the unit counter and the
 * per-band partials come from the library's fixed array; the call needs
 * 256 + 2 x round256(8 (n_sn + 1)) + round256(40 n_par)
 *   + 64 n_bands n_par + 4 n_par + 256 bytes
 * (about 39,000 samples with 6 bands) and returns SALT_ERR_INVALID, touching
 * nothing, if that exceeds SALT_NOALLOC_SCRATCH_BYTES or if the model has more
 * than 128 phase nodes; salt_last_error gives the bytes needed. Each call
 * copies the HOST offsets (pageable memory, cudaMemcpyAsync) into the array
 * and clears the counters that must start at zero, on cuda_stream. With
 * batch->validate set it synchronises cuda_stream to read the verdict.
 * The first call on each device looks the array's address up
 * (cudaGetSymbolAddress).
 * The array is shared by every call on that device in the process: two calls
 * whose executions overlap (different streams, threads or contexts on the same
 * device) race on it and give wrong results, so serialise them. */
int salt_chi2_grad_noalloc(salt_ctx *ctx, const salt_batch *batch, double *chi2, float *grad,
                           void *cuda_stream);

/* ------------------------------------------------- device peaks ---------- */

/* Microbenchmarks of the context's device (the paper has no counterpart: they
 * are the measured side of the roofline the photometry kernels are reported
 * against). */
typedef struct {
    double fp32_tflops;      /* FMA throughput, 2 FLOP per FMA: 8 independent FMA chains per
                                thread, 8 blocks of 256 threads per SM, best of 3 launches */
    double l2_read_gbs;      /* 200 passes of 16-byte L2-only loads (ld.global.cg) over a 32 MiB
                                buffer (L2-resident) */
    double smem_read_gbs;    /* conflict-free 16-byte shared-memory loads, all SMs */
    double sm_clock_max_mhz; /* the device's maximum SM clock (cudaDevAttrClockRate) */
    int32_t num_sms;
} salt_peaks;

/* Runs the three microbenchmarks on a private stream (synchronous, ~50 ms;
 * allocates and frees 32 MiB plus a small sink) and fills *out.
 * SALT_ERR_INVALID for NULL arguments, SALT_ERR_OOM / SALT_ERR_CUDA with
 * salt_last_error set otherwise. */
int salt_measure_peaks(salt_ctx *ctx, salt_peaks *out);

/* ---------------------------------------------------------------- misc ---- */

const char *salt_status_str(int status);
const char *salt_last_error(const salt_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SALT_H */
