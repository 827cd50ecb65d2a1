// Batched per-supernova fitting of the free SALT parameters by bound-constrained
// limited-memory quasi-Newton iterations (the paper optimises x0, x1, t0 and c
// with L-BFGS-B, Implementation, first paragraph).
//
// Every supernova is an independent problem over the parameters selected by a
// mask (default t0, x0, x1, c with z fixed). All problems advance in lockstep:
// one iteration of the driver is one batched chi^2 + gradient evaluation of
// every supernova's trial point by the library's factorised kernels, followed
// by one update kernel with a thread per supernova holding its FP64 state:
//   - variables are scaled, v = x / s with s = (0.01, 1 day, |x0 at start|, 1, 0.1)
//     for (z, t0, x0, x1, c);
//   - the search direction is the two-loop L-BFGS product over the free
//     variables (those not pinned at a bound by a gradient pointing outward),
//     with H0 = (s.y / y.y) I from the newest pair;
//   - a free variable at a bound is not pushed outward by d, and the step is
//     capped at the distance to the box along d (so the path stays straight);
//   - the step length satisfies the strong Wolfe conditions (sufficient
//     decrease with c1 = 1e-4, |g(alpha).d| <= 0.9 |g(0).d|) by bracketing
//     (alpha x4 while the slope stays steep) and zooming with safeguarded
//     cubic interpolation, or stops at the box. chi^2 from FP32 photometry
//     resolves differences only down to eps = 2e-6 chi^2, while the gradient
//     stays accurate; so, in the manner of approximate Wolfe conditions, a
//     step that meets the curvature condition is also taken when chi^2 rose
//     by at most eps, the bracket is steered by the slope's sign wherever
//     chi^2 differences are within eps;
//   - a fit stops when the projected scaled gradient's inf-norm pg is <= gtol,
//     at max_iter iterations, or when the line search cannot lower chi^2 any
//     more (after one retry along steepest descent with the curvature pairs
//     dropped). When chi^2 stops falling measurably (an accepted step lowers it
//     by <= ftol relative, or eight in a row together by no more than eps) the
//     fit has converged to chi^2's resolution if pg <= 100 gtol; with a larger
//     (accurate) gradient the curvature pairs are dropped instead and the fit
//     goes on along steepest descent, at most three times; a fit still flat
//     with pg > 100 gtol after that ends with SALT_FIT_FLAT, not as converged.
// Unlike L-BFGS-B proper there is no generalised Cauchy point or subspace
// minimisation: bounds enter through the active set and the projection.
// Blocks of iterations are captured once as a CUDA graph and replayed.
#include <cmath>
#include <cstring>
#include <string>

#include "salt_internal.cuh"

namespace salt {
namespace fit {

constexpr int NP = 5;    // z, t0, x0, x1, c (the gradient's order)
constexpr int MMAX = 8;  // largest L-BFGS memory

enum Stage { ST_START = 0, ST_SEARCH = 1, ST_DONE = 2 };
constexpr double C1 = 1e-4, C2 = 0.9;  // Wolfe constants
constexpr double NOISE = 2e-6;         // relative chi^2 resolution of the FP32 photometry
constexpr int QUIET = 8;               // accepted steps without a decrease beyond the noise
constexpr int RESTARTS = 3;            // flat stretches that restart along steepest descent
constexpr double FLAT_G = 100.0;       // a flat chi^2 counts as converged when pg <= FLAT_G gtol
constexpr int LS_MAX = 30;             // evaluations per line search

struct State {
    double x[NP], g[NP];    // accepted point and its gradient (natural units)
    double f;               // chi^2 there
    double xt[NP];          // trial point being evaluated
    double d[NP];           // search direction (scaled units)
    double sc[NP];          // variable scales
    double lo[NP], hi[NP];  // box (natural units)
    double S[MMAX][NP], Y[MMAX][NP], rho[MMAX];
    double alpha, gd;       // trial step and directional derivative g(0).d (scaled)
    double amax;            // step to the box along d
    // line search: previous bracketing trial, zoom interval ends, best sufficient-decrease point
    double a_prev, f_prev, g_prev;
    double lo_a, lo_f, lo_g, hi_a, hi_f, hi_g;
    double xb[NP], gb[NP], fb;
    int head, count;        // ring buffer of (s, y) pairs
    int iter, nls, evals, stage, status, zoom, has_best;
    int quiet;      // accepted steps since chi^2 last fell by more than the noise
    double f_quiet; // chi^2 when that window began
    int restarts;   // flat stretches answered by dropping the curvature pairs
};

struct Opts {
    double gtol, ftol;
    int max_iter, max_evals, m, mask;
    // list of the fits still running, rebuilt by every update: the next
    // evaluation covers only these supernovae (NULL: evaluate all)
    WorkItem *act;
    const int64_t *obs_off;
};

// Count supernova j as running and append its one-sample work item.
__device__ __forceinline__ void mark_active(const Opts &op, int *n_active, int j) {
    const int k = atomicAdd(n_active, 1);
    if (op.act) {
        WorkItem w;
        w.obs0 = op.obs_off[j];
        w.par0 = j;
        w.bf0 = 0;
        w.nobs = (int32_t)(op.obs_off[j + 1] - op.obs_off[j]);
        w.nj = 1;
        w.jloc0 = 0;
        w.pad = 0;
        op.act[k] = w;
    }
}

struct Trial {
    double *t0;
    float *z, *x0, *x1, *c;
};

__device__ __forceinline__ double clampd(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }

// Round a trial point to what the chi^2 kernels read (t0 FP64, the rest FP32),
// keep it inside the box, and publish it.
__device__ void publish(State &st, const Trial &tr, int j) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        double v = clampd(st.xt[i], st.lo[i], st.hi[i]);
        if (i != 1) {
            float fv = (float)v;
            if ((double)fv < st.lo[i]) fv = nextafterf(fv, INFINITY);
            if ((double)fv > st.hi[i]) fv = nextafterf(fv, -INFINITY);
            v = (double)fv;
        }
        st.xt[i] = v;
    }
    tr.z[j] = (float)st.xt[0];
    tr.t0[j] = st.xt[1];
    tr.x0[j] = (float)st.xt[2];
    tr.x1[j] = (float)st.xt[3];
    tr.c[j] = (float)st.xt[4];
}

__device__ __forceinline__ bool in_mask(int mask, int i) { return (mask >> i) & 1; }

// A variable counts as sitting on a bound within a few FP32 ulps of the bound
// (plus 1e-7 of its scale): publish() may round an FP32 parameter one ulp
// inside a bound it cannot represent exactly. t0 is FP64: 1e-9 day.
__device__ __forceinline__ double bound_tol(const State &st, int i, double b) {
    return i == 1 ? 1e-9 * st.sc[i] : 1e-7 * st.sc[i] + 4.8e-7 * fabs(b);
}
__device__ __forceinline__ bool at_lo(const State &st, int i) {
    return isfinite(st.lo[i]) && st.x[i] <= st.lo[i] + bound_tol(st, i, st.lo[i]);
}
__device__ __forceinline__ bool at_hi(const State &st, int i) {
    return isfinite(st.hi[i]) && st.x[i] >= st.hi[i] - bound_tol(st, i, st.hi[i]);
}

// Scaled gradient component i, projected for the bound it sits on.
__device__ __forceinline__ double proj_grad(const State &st, int mask, int i) {
    if (!in_mask(mask, i)) return 0.0;
    const double gs = st.g[i] * st.sc[i];
    if (at_lo(st, i)) return fmin(gs, 0.0);
    if (at_hi(st, i)) return fmax(gs, 0.0);
    return gs;
}

// New search direction from the accepted point and the first trial along it.
__device__ void new_direction(State &st, const Opts &op, const Trial &tr, int j) {
    double q[NP];
    bool fr[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const double gs = st.g[i] * st.sc[i];
        fr[i] = in_mask(op.mask, i) && !((at_lo(st, i) && gs > 0.0) || (at_hi(st, i) && gs < 0.0));
        q[i] = fr[i] ? gs : 0.0;
    }
    double a[MMAX];
    // first loop: newest to oldest
    for (int k = 0; k < st.count; ++k) {
        const int p = (st.head - 1 - k + op.m) % op.m;
        double sq = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) sq += fr[i] ? st.S[p][i] * q[i] : 0.0;
        a[k] = st.rho[p] * sq;
#pragma unroll
        for (int i = 0; i < NP; ++i) if (fr[i]) q[i] -= a[k] * st.Y[p][i];
    }
    if (st.count > 0) {
        const int p = (st.head - 1 + op.m) % op.m;
        double sy = 0.0, yy = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i)
            if (fr[i]) { sy += st.S[p][i] * st.Y[p][i]; yy += st.Y[p][i] * st.Y[p][i]; }
        const double gamma = (sy > 0.0 && yy > 0.0) ? sy / yy : 1.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) q[i] *= gamma;
    }
    // second loop: oldest to newest
    for (int k = st.count - 1; k >= 0; --k) {
        const int p = (st.head - 1 - k + op.m) % op.m;
        double yq = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) yq += fr[i] ? st.Y[p][i] * q[i] : 0.0;
        const double b = st.rho[p] * yq;
#pragma unroll
        for (int i = 0; i < NP; ++i) if (fr[i]) q[i] += (a[k] - b) * st.S[p][i];
    }
    double gd = 0.0, gn = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        double di = fr[i] ? -q[i] : 0.0;
        if ((at_lo(st, i) && di < 0.0) || (at_hi(st, i) && di > 0.0)) di = 0.0;
        st.d[i] = di;
        const double gs = fr[i] ? st.g[i] * st.sc[i] : 0.0;
        gd += gs * di;
        gn += gs * gs;
    }
    if (!(gd < 0.0)) {  // not a descent direction: restart from (projected) steepest descent
        st.count = 0;
        gd = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const double gs = fr[i] ? st.g[i] * st.sc[i] : 0.0;
            double di = -gs;
            if ((at_lo(st, i) && di < 0.0) || (at_hi(st, i) && di > 0.0)) di = 0.0;
            st.d[i] = di;
            gd += gs * di;
        }
    }
    double amax = 1e20;  // largest step inside the box along d
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const double step = st.d[i] * st.sc[i];
        if (step > 0.0 && isfinite(st.hi[i])) amax = fmin(amax, (st.hi[i] - st.x[i]) / step);
        if (step < 0.0 && isfinite(st.lo[i])) amax = fmin(amax, (st.lo[i] - st.x[i]) / step);
    }
    st.gd = gd;
    st.amax = amax;
    st.alpha = fmin(st.count > 0 ? 1.0 : fmin(1.0, 1.0 / fmax(sqrt(gn), 1e-300)), amax);
    st.nls = 0;
    st.zoom = 0;
    st.has_best = 0;
    st.a_prev = 0.0;
    st.f_prev = st.f;
    st.g_prev = gd;
#pragma unroll
    for (int i = 0; i < NP; ++i) st.xt[i] = st.x[i] + st.alpha * st.d[i] * st.sc[i];
    publish(st, tr, j);
}

// Minimiser of the cubic through (a0, f0, g0) and (a1, f1, g1), kept 10 % away
// from both ends; bisection when the data are not finite or the cubic has no
// minimiser.
__device__ double cubic_step(double a0, double f0, double g0, double a1, double f1, double g1) {
    const double lo = fmin(a0, a1), hi = fmax(a0, a1);
    if (isfinite(f0) && isfinite(g0) && isfinite(f1) && isfinite(g1) && a0 != a1) {
        const double d1 = g0 + g1 - 3.0 * (f0 - f1) / (a0 - a1);
        const double disc = d1 * d1 - g0 * g1;
        if (disc >= 0.0) {
            const double d2 = copysign(sqrt(disc), a1 - a0);
            const double den = g1 - g0 + 2.0 * d2;
            if (den != 0.0) {
                const double a = a1 - (a1 - a0) * (g1 + d2 - d1) / den;
                if (isfinite(a)) return fmin(fmax(a, lo + 0.1 * (hi - lo)), hi - 0.1 * (hi - lo));
            }
        }
    }
    return 0.5 * (lo + hi);
}

__global__ void k_fit_init(int n, const double *t0, const float *z, const float *x0, const float *x1,
                           const float *c, const double *lower, const double *upper, int mask, State *S,
                           Trial tr, Opts op, int *n_active) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    State st;
    const double init[NP] = {(double)z[j], t0[j], (double)x0[j], (double)x1[j], (double)c[j]};
    const double sc[NP] = {0.01, 1.0, fabs((double)x0[j]) > 0.0 ? fabs((double)x0[j]) : 1e-5, 1.0, 0.1};
    bool ok = true;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        double lo = lower ? lower[NP * j + i] : -INFINITY;
        double hi = upper ? upper[NP * j + i] : INFINITY;
        if (!in_mask(mask, i)) lo = hi = init[i];  // fixed parameter
        if (i == 0 && in_mask(mask, i)) lo = fmax(lo, -0.99);  // a free z stays > -1
        if (!(lo <= hi) || !isfinite(init[i])) ok = false;
        st.lo[i] = lo;
        st.hi[i] = hi;
        st.sc[i] = sc[i];
        st.xt[i] = init[i];
        st.x[i] = init[i];
        st.g[i] = 0.0;
        st.d[i] = 0.0;
    }
    st.f = INFINITY;
    st.alpha = 0.0;
    st.gd = 0.0;
    st.head = st.count = 0;
    st.iter = st.nls = st.evals = 0;
    st.quiet = 0;
    st.f_quiet = INFINITY;
    st.restarts = 0;
    st.stage = ok ? ST_START : ST_DONE;
    st.status = ok ? 0 : SALT_FIT_INVALID;
    publish(st, tr, j);
    S[j] = st;
    if (ok) mark_active(op, n_active, j);
}

// Take the step to st.xt (chi^2 ft, gradient gt): curvature pair, convergence
// tests, next direction.
__device__ void accept_step(State &st, const Opts &op, const Trial &tr, int j, double ft, const double *gt,
                            int *n_active) {
    double s[NP], y[NP], sy = 0.0, yy = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        s[i] = (st.xt[i] - st.x[i]) / st.sc[i];
        y[i] = (gt[i] - st.g[i]) * st.sc[i];
        sy += s[i] * y[i];
        yy += y[i] * y[i];
    }
    if (sy > 1e-10 * yy && op.m > 0) {
        const int p = st.head;
#pragma unroll
        for (int i = 0; i < NP; ++i) { st.S[p][i] = s[i]; st.Y[p][i] = y[i]; }
        st.rho[p] = 1.0 / sy;
        st.head = (st.head + 1) % op.m;
        st.count = min(st.count + 1, op.m);
    }
    const double fprev = st.f;
#pragma unroll
    for (int i = 0; i < NP; ++i) { st.x[i] = st.xt[i]; st.g[i] = gt[i]; }
    st.f = ft;
    ++st.iter;
    double pg = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) pg = fmax(pg, fabs(proj_grad(st, op.mask, i)));
    const double rel = (fprev - ft) / fmax(fmax(fabs(fprev), fabs(ft)), 1.0);
    if (!(st.f_quiet - ft <= NOISE * fabs(st.f_quiet))) {  // real progress: restart the window
        st.f_quiet = ft;
        st.quiet = 0;
    } else {
        ++st.quiet;
    }
    if (pg <= op.gtol) {
        st.stage = ST_DONE;
        st.status = st.iter;
        return;
    }
    if ((rel >= 0.0 && rel <= op.ftol) || st.quiet >= QUIET) {
        // chi^2 has stopped falling measurably (a step within ftol, or eight
        // within the noise). That is convergence to its resolution when the
        // accurate gradient is small too. A large one means the curvature pairs
        // have gone stale in a curved valley (tiny steps, a tiny inverse-Hessian
        // scale): drop them and go on along steepest descent, a bounded number
        // of times.
        if (pg <= FLAT_G * op.gtol || st.restarts >= RESTARTS) {
            // restarts used up with the gradient still large: stopped, not converged
            st.stage = ST_DONE;
            st.status = pg <= FLAT_G * op.gtol ? st.iter : SALT_FIT_FLAT;
            return;
        }
        ++st.restarts;
        st.quiet = 0;
        st.f_quiet = st.f;
        st.count = 0;
        st.head = 0;
    }
    if (st.iter >= op.max_iter || st.evals >= op.max_evals) {
        st.stage = ST_DONE;
        st.status = SALT_FIT_MAXITER;
    } else {
        new_direction(st, op, tr, j);
        mark_active(op, n_active, j);
    }
}

__global__ void k_fit_update(int n, State *S, const double *chi2, const float *grad, Trial tr, Opts op,
                             int *n_active) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    State &st = S[j];
    if (st.stage == ST_DONE) return;
    const double ft = chi2[j];
    double gt[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) gt[i] = (double)grad[NP * j + i];
    bool ok_t = isfinite(ft);
#pragma unroll
    for (int i = 0; i < NP; ++i) ok_t = ok_t && isfinite(gt[i]);
    ++st.evals;

    if (st.stage == ST_START) {
        if (!ok_t) {
            st.stage = ST_DONE;
            st.status = SALT_FIT_INVALID;
            return;
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) { st.x[i] = st.xt[i]; st.g[i] = gt[i]; }
        st.f = ft;
        st.f_quiet = ft;
        double pg = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) pg = fmax(pg, fabs(proj_grad(st, op.mask, i)));
        if (pg <= op.gtol) {
            st.stage = ST_DONE;
            st.status = 0;
            return;
        }
        st.stage = ST_SEARCH;
        new_direction(st, op, tr, j);
        mark_active(op, n_active, j);
        return;
    }

    // ST_SEARCH: strong Wolfe line search along d (bracketing, then zoom)
    double gdt = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) gdt += gt[i] * st.sc[i] * st.d[i];
    const double a = st.alpha;
    const double eps = NOISE * fabs(st.f) + 1e-12;
    const bool armijo = ok_t && ft <= st.f + C1 * a * st.gd;
    const bool within = ok_t && ft <= st.f + C1 * a * st.gd + eps;  // not worse beyond the noise
    const bool curv = ok_t && fabs(gdt) <= -C2 * st.gd;
    ++st.nls;
    bool accept = false;
    auto keep_best = [&]() {
        if (!armijo) return;  // only true sufficient-decrease points are kept as fallbacks
#pragma unroll
        for (int i = 0; i < NP; ++i) { st.xb[i] = st.xt[i]; st.gb[i] = gt[i]; }
        st.fb = ft;
        st.has_best = 1;
    };
    if (!st.zoom) {
        if (!within || (st.nls > 1 && ft > st.f_prev + eps)) {
            st.zoom = 1;
            st.lo_a = st.a_prev; st.lo_f = st.f_prev; st.lo_g = st.g_prev;
            st.hi_a = a; st.hi_f = ft; st.hi_g = gdt;
        } else if (curv || a >= st.amax) {
            accept = true;
        } else if (gdt >= 0.0) {
            keep_best();
            st.zoom = 1;
            st.lo_a = a; st.lo_f = ft; st.lo_g = gdt;
            st.hi_a = st.a_prev; st.hi_f = st.f_prev; st.hi_g = st.g_prev;
        } else {  // not worse and still steep: lengthen the step
            keep_best();
            st.a_prev = a; st.f_prev = ft; st.g_prev = gdt;
            if (st.nls < LS_MAX && st.evals < op.max_evals) {
                st.alpha = fmin(4.0 * a, st.amax);
#pragma unroll
                for (int i = 0; i < NP; ++i) st.xt[i] = st.x[i] + st.alpha * st.d[i] * st.sc[i];
                publish(st, tr, j);
                mark_active(op, n_active, j);
                return;
            }
        }
    } else {
        if (!within || ft > st.lo_f + eps) {
            st.hi_a = a; st.hi_f = ft; st.hi_g = gdt;
        } else if (curv) {
            accept = true;
        } else {
            keep_best();
            // the slope's sign says on which side the minimum along d lies
            if (gdt * (st.hi_a - st.lo_a) >= 0.0) { st.hi_a = st.lo_a; st.hi_f = st.lo_f; st.hi_g = st.lo_g; }
            st.lo_a = a; st.lo_f = ft; st.lo_g = gdt;
        }
    }
    if (!accept) {
        if (st.nls >= LS_MAX || st.evals >= op.max_evals || !st.zoom) {
            if (!st.has_best) {  // nothing lowers chi^2 along d
                if (st.count > 0 && st.evals < op.max_evals) {
                    // drop the curvature pairs and retry once along steepest descent
                    st.count = 0;
                    st.head = 0;
                    new_direction(st, op, tr, j);
                    mark_active(op, n_active, j);
                    return;
                }
                st.stage = ST_DONE;
                st.status = st.evals >= op.max_evals ? SALT_FIT_MAXITER : SALT_FIT_LINESEARCH;
                return;
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) { st.xt[i] = st.xb[i]; gt[i] = st.gb[i]; }
            // accept the best sufficient-decrease point found
            const double fbest = st.fb;
            return accept_step(st, op, tr, j, fbest, gt, n_active);
        }
        st.alpha = cubic_step(st.lo_a, st.lo_f, st.lo_g, st.hi_a, st.hi_f, st.hi_g);
#pragma unroll
        for (int i = 0; i < NP; ++i) st.xt[i] = st.x[i] + st.alpha * st.d[i] * st.sc[i];
        publish(st, tr, j);
        mark_active(op, n_active, j);
        return;
    }
    accept_step(st, op, tr, j, ft, gt, n_active);
}

// Fold the fit's own error word into the context's, without the FP32-range bit:
// a trial point far out along a search direction may overflow the colour factor,
// which the line search already treats as "too far".
__global__ void k_fold_errors(const int *src, int *dst, int mask) {
    const int v = *src & mask;
    if (v) atomicOr(dst, v);
}

__global__ void k_fit_finish(int n, const State *S, Trial tr, double *theta, double *chi2, int *status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const State &st = S[j];
#pragma unroll
    for (int i = 0; i < NP; ++i) theta[NP * j + i] = st.x[i];
    chi2[j] = st.f;
    status[j] = st.stage == ST_DONE ? st.status : SALT_FIT_MAXITER;
}

}  // namespace fit

namespace {

int fit_fail(salt_ctx *ctx, int code, const std::string &msg) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_error = msg;
    return code;
}

int fit_cuda(salt_ctx *ctx, cudaError_t e, const char *what) {
    (void)cudaGetLastError();
    return fit_fail(ctx, e == cudaErrorMemoryAllocation ? SALT_ERR_OOM : SALT_ERR_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

// One batched chi^2 + gradient evaluation at the trial points, then the update.
// One evaluation of the running fits' trial points, then the update (which
// also lists the fits still running for the next evaluation). With a list
// (op.act) the warp-unit kernel reads its length on the device, so finished
// fits cost nothing; without one, the whole batch goes through the plan.
static int fit_step(salt_ctx *ctx, salt_plan *plan, const BatchDev &b, const OutDev &o, fit::State *S,
                    const fit::Trial &tr, const fit::Opts &op, int *n_active, int n, int *counter,
                    void *scratch, cudaStream_t st) {
    cudaError_t e;
    if (op.act) {
        e = launch_unit_items(ctx, 1, op.act, n, counter, scratch, b, o, MODE_GRAD, st, n_active);
        if (e != cudaSuccess) return fit_cuda(ctx, e, "fit evaluation");
    } else {
        const int rc = run_batch(ctx, b, plan, o, MODE_GRAD, st);
        if (rc != SALT_OK) return rc;
    }
    e = cudaMemsetAsync(n_active, 0, sizeof(int), st);
    if (e != cudaSuccess) return fit_cuda(ctx, e, "fit counter");
    fit::k_fit_update<<<(n + 127) / 128, 128, 0, st>>>(n, S, o.chi2, o.grad, tr, op, n_active);
    e = cudaGetLastError();
    return e == cudaSuccess ? SALT_OK : fit_cuda(ctx, e, "fit update");
}

}  // namespace salt

using namespace salt;

extern "C" int salt_fit(salt_ctx *ctx, const salt_batch *bt, const double *lower, const double *upper,
                        const salt_fit_opts *opts, double *theta, double *chi2_out, int32_t *status,
                        void *cuda_stream) {
    if (!ctx || !bt) return SALT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    salt_fit_opts o = opts ? *opts : salt_fit_opts{0, 0, 0, 0, 0.0, 0.0};
    if (o.max_iter <= 0) o.max_iter = 300;
    if (o.history <= 0) o.history = 6;
    if (o.free_mask == 0) o.free_mask = SALT_FIT_DEFAULT_MASK;
    if (o.gtol <= 0.0) o.gtol = 1e-3;
    if (o.ftol <= 0.0) o.ftol = 1e-10;
    if (o.max_evals <= 0) o.max_evals = 2 * o.max_iter + 20;
    if (o.history > fit::MMAX || (o.free_mask & ~0x1f) != 0)
        return fit_fail(ctx, SALT_ERR_INVALID, "fit: history must be <= 8 and free_mask within 5 bits");
    if (bt->n_sn < 0 || !bt->obs_off || !bt->par_off) return fit_fail(ctx, SALT_ERR_INVALID, "missing offsets");
    const int64_t n_sn = bt->n_sn;
    for (int64_t s = 0; s <= n_sn; ++s)
        if (bt->par_off[s] != s)
            return fit_fail(ctx, SALT_ERR_INVALID, "fit: one parameter sample (the starting point) per supernova");
    if (n_sn > INT32_MAX / 2) return fit_fail(ctx, SALT_ERR_INVALID, "fit: too many supernovae");
    if (n_sn == 0) return SALT_OK;
    if (!theta || !chi2_out || !status) return fit_fail(ctx, SALT_ERR_INVALID, "fit: missing output");
    if (!bt->t0 || !bt->z || !bt->x0 || !bt->x1 || !bt->c)
        return fit_fail(ctx, SALT_ERR_INVALID, "missing parameter arrays");
    const int64_t n_obs = bt->obs_off[n_sn];
    if (n_obs > 0 && (!bt->mjd || !bt->band || !bt->flux || !bt->fluxerr || !bt->zp))
        return fit_fail(ctx, SALT_ERR_INVALID, "missing observation arrays");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fit_cuda(ctx, e, "cudaSetDevice");
    const int n = (int)n_sn;

    salt_plan plan;  // reused by every evaluation of this call (tuned once, graph-captured)
    int rc = plan_build(ctx, n_sn, bt->obs_off, bt->par_off, 0, &plan, st, false);
    if (rc != SALT_OK) {
        plan_free(&plan, st);
        return rc;
    }
    // device scratch: states, trial parameters, chi^2 / gradient of the trials, active count
    fit::State *S = nullptr;
    double *t0t = nullptr, *chi2 = nullptr;
    float *zt = nullptr, *x0t = nullptr, *x1t = nullptr, *ct = nullptr, *grad = nullptr;
    int *n_active = nullptr, *counter = nullptr, *err_fit = nullptr;
    WorkItem *act = nullptr;  // running fits' work items (warp-unit path)
    void *uscr = nullptr;     // warp-unit kernel scratch
    const bool compact = ctx->mp.n_phase <= unit_max_phase() && ctx->mp.bands.n_bands >= 1;
    const size_t uscr_bytes = compact ? unit_scratch_bytes(n, 1, ctx->mp.bands.n_bands) : 0;
    const size_t fb = (size_t)n * sizeof(float);
    e = cudaMalloc((void **)&S, (size_t)n * sizeof(fit::State));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t0t, (size_t)n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&chi2, (size_t)n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&zt, fb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&x0t, fb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&x1t, fb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ct, fb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&grad, 5 * fb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&n_active, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&counter, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&err_fit, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err_fit, 0, sizeof(int), st);
    if (e == cudaSuccess && compact) e = cudaMalloc((void **)&act, (size_t)n * sizeof(WorkItem));
    if (e == cudaSuccess && compact) e = cudaMalloc(&uscr, uscr_bytes);
    if (e == cudaSuccess && compact) e = cudaMemsetAsync(uscr, 0, uscr_bytes, st);  // arrival counters
    if (e == cudaSuccess) e = cudaMemsetAsync(n_active, 0, sizeof(int), st);
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        void *ptrs[] = {S, t0t, chi2, zt, x0t, x1t, ct, grad, n_active, counter, err_fit, act, uscr};
        cudaStreamSynchronize(st);
        for (void *q : ptrs)
            if (q) cudaFree(q);
        plan_free(&plan, st);
    };
    if (e != cudaSuccess) {
        rc = fit_cuda(ctx, e, "fit scratch");
        cleanup();
        return rc;
    }
    const fit::Trial tr{t0t, zt, x0t, x1t, ct};
    const fit::Opts op{o.gtol, o.ftol, o.max_iter, o.max_evals, o.history, o.free_mask, act, plan.obs_off_d};
    BatchDev b{};
    b.n_sn = n_sn;
    b.n_obs = n_obs;
    b.n_par = n_sn;
    b.obs_off = plan.obs_off_d;
    b.par_off = plan.par_off_d;
    b.mjd = bt->mjd; b.band = bt->band; b.flux = bt->flux; b.fluxerr = bt->fluxerr; b.zp = bt->zp;
    b.t0 = t0t; b.z = zt; b.x0 = x0t; b.x1 = x1t; b.c = ct;
    const OutDev od{nullptr, plan.bf_off_d, chi2, grad, err_fit};

    fit::k_fit_init<<<(n + 127) / 128, 128, 0, st>>>(n, bt->t0, bt->z, bt->x0, bt->x1, bt->c, lower, upper,
                                                      o.free_mask, S, tr, op, n_active);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        rc = fit_cuda(ctx, e, "fit init");
        cleanup();
        return rc;
    }
    // first evaluation outside capture (on the plan path it tunes the kernel choice)
    rc = fit_step(ctx, &plan, b, od, S, tr, op, n_active, n, counter, uscr, st);
    // then blocks of iterations replayed from one captured graph
    constexpr int BLOCK = 8;
    int evals = 1, active = 1;
    if (rc == SALT_OK) {
        if (!ctx->capture_stream &&
            (e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
            rc = fit_cuda(ctx, e, "fit stream");
    }
    if (rc == SALT_OK) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
        int rc_cap = SALT_OK;
        for (int k = 0; k < BLOCK && e == cudaSuccess && rc_cap == SALT_OK; ++k)
            rc_cap = fit_step(ctx, &plan, b, od, S, tr, op, n_active, n, counter, uscr, ctx->capture_stream);
        const cudaError_t e_end = cudaStreamEndCapture(ctx->capture_stream, &g);
        if (e == cudaSuccess) e = e_end;
        if (e == cudaSuccess && rc_cap == SALT_OK) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || rc_cap != SALT_OK) {
            (void)cudaGetLastError();
            exec = nullptr;  // capture unavailable: iterate with direct launches
        }
    }
    while (rc == SALT_OK && active > 0 && evals < o.max_evals + 1) {
        if (exec) {
            e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) { rc = fit_cuda(ctx, e, "fit graph"); break; }
        } else {
            for (int k = 0; k < BLOCK && rc == SALT_OK; ++k)
                rc = fit_step(ctx, &plan, b, od, S, tr, op, n_active, n, counter, uscr, st);
            if (rc != SALT_OK) break;
        }
        evals += BLOCK;
        e = cudaMemcpyAsync(&active, n_active, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = fit_cuda(ctx, e, "fit progress"); break; }
    }
    if (rc == SALT_OK) {
        fit::k_fit_finish<<<(n + 127) / 128, 128, 0, st>>>(n, S, tr, theta, chi2_out, status);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            fit::k_fold_errors<<<1, 1, 0, st>>>(err_fit, ctx->err_d, ~(int)ERRBIT_RANGE);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) rc = fit_cuda(ctx, e, "fit finish");
    }
    cleanup();
    return rc;
}
