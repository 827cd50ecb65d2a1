/*
 * FP64 CPU oracle for batched SALT synthetic photometry.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the GPU path must compute. Only the tests, the smoke check
 * and the bench's CPU-baseline leg load it. It shares no code, header, table
 * or helper with the CUDA library, and the library never calls it.
 *
 * Everything is evaluated straight from the definitions, per band sample, in
 * double precision with the host libm:
 *
 *   SALT model form (paper, Implementation, Eq. 1):
 *       F(p, lambda) = x0 [M0(p, lambda) + x1 M1(p, lambda)] 10^(-0.4 c CL(lambda))
 *     (the paper writes the colour term as exp[c CL]; that is the same
 *     function with its CL equal to -0.4 ln10 times the CL used here),
 *     with p = (t - t0) / (1 + z) and lambda the rest-frame wavelength
 *     lambda_obs / (1 + z); the observer-frame flux density carries the
 *     factor 1 / (1 + z).
 *   Bandflux (paper, Implementation, Eq. 2):
 *       bandflux = integral F(lambda) T(lambda) lambda / (h c) dlambda,
 *     integrated with the trapezoidal rule on the band's own samples
 *     (paper, Implementation, the paragraph after Eq. 2), then scaled to the
 *     observation's AB zero point: 10^(0.4 zp) / (the same integral of the
 *     AB reference spectrum f_AB = 3631 Jy, as f_lambda).
 *   chi^2 = sum_i ((f_i - bandflux_i) / sigma_i)^2 (diagonal Gaussian).
 *
 * Readings where the paper is silent (stated once here, used everywhere):
 *   - surface interpolation: tensor-product Keys cubic convolution, a = -1/2,
 *     linear on the first and last interval of each axis, zero outside the grid;
 *   - colour law: SALT2 polynomial form with linear extrapolation outside
 *     [cl_lo, cl_hi] using the value and slope at the nearer end;
 *   - gradient: analytic forward mode over (z, t0, x0, x1, c).
 *
 * Pins (tests/test_oracle_*.py): node reproduction, partition of unity,
 * quadratic/linear reproduction, colour-law anchors and continuity,
 * closed-form top-hat integrals, the trapezoid's exact quadratic error, the
 * AB zero point, linearity in x0, z = 0, epoch-shift invariance, chi^2 = 0 and
 * zero gradient at a noiseless truth, the least-squares x0, FP64 central
 * differences, and a 50-digit mpmath evaluation of a tiny case.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CGS constants: Planck (exact SI definition), speed of light in A/s (exact),
 * AB reference 3631 Jy = 3631e-23 erg s^-1 cm^-2 Hz^-1. */
static const double OM_H_ERG_S = 6.62607015e-27;
static const double OM_C_AA_S = 2.99792458e18;
static const double OM_AB_FNU = 3631e-23;
/* SALT2 colour-law reference wavelengths (B and V), in A. */
static const double OM_LAMBDA_B = 4302.57;
static const double OM_LAMBDA_V = 5428.55;

typedef struct {
    int32_t n_phase, n_wave;
    double phase0, dphase, wave0, dwave;
    const double *m0, *m1; /* row-major [n_phase][n_wave] */
    double cl[4];
    double cl_lo, cl_hi;
    /* non-uniform axes: ascending node positions [n_phase] / [n_wave]; NULL =
     * the uniform axis phase0 + r dphase / wave0 + j dwave */
    const double *pnode, *wnode;
} om_model;

typedef struct {
    int32_t n;
    const double *wave, *trans; /* ascending wavelength, transmission */
} om_band;

/* ------------------------------------------------------------------------ */
/* Keys (1981) cubic convolution kernel with a = -1/2, and its derivative.   */

static double keys_kernel(double s)
{
    const double a = -0.5;
    double u = fabs(s);
    if (u <= 1.0) return (a + 2.0) * u * u * u - (a + 3.0) * u * u + 1.0;
    if (u < 2.0) return a * u * u * u - 5.0 * a * u * u + 8.0 * a * u - 4.0 * a;
    return 0.0;
}

static double keys_kernel_deriv(double s)
{
    const double a = -0.5;
    double u = fabs(s), sg = (s < 0.0) ? -1.0 : 1.0;
    if (u <= 1.0) return sg * (3.0 * (a + 2.0) * u * u - 2.0 * (a + 3.0) * u);
    if (u < 2.0) return sg * (3.0 * a * u * u - 10.0 * a * u + 8.0 * a);
    return 0.0;
}

/* One axis of the interpolation: the nodes that carry weight at x, their
 * weights, and the weights' derivatives with respect to x. Returns the number
 * of nodes (4 on an interior interval, 2 on an edge interval, 0 outside). */
int om_axis_taps(double x, double x0, double dx, int32_t n, int32_t *first,
                 double w[4], double dw[4])
{
    double xmax = x0 + (double)(n - 1) * dx;
    if (n < 2 || !(x >= x0 && x <= xmax)) return 0;
    double u = (x - x0) / dx;
    int32_t i = (int32_t)floor(u);
    if (i > n - 2) i = n - 2;
    if (i < 0) i = 0;
    double t = u - (double)i;
    if (i == 0 || i == n - 2) {
        *first = i;
        w[0] = 1.0 - t;  dw[0] = -1.0 / dx;
        w[1] = t;        dw[1] = 1.0 / dx;
        return 2;
    }
    *first = i - 1;
    for (int m = 0; m < 4; ++m) {
        double s = u - (double)(i - 1 + m); /* signed distance to node i-1+m */
        w[m] = keys_kernel(s);
        dw[m] = keys_kernel_deriv(s) / dx;
    }
    return 4;
}

/* The same on an axis with ascending, possibly non-uniform nodes (the SALT3 /
 * SALT3-NIR "dedicated interpolation routines", Implementation, last but one
 * paragraph; reading: the interval i is found by search, the coordinate is
 * mapped to index space u = i + (x - x_i)/(x_{i+1} - x_i), and the Keys kernel
 * applies in u, so a uniform axis gives exactly the taps above). */
int om_axis_taps_nodes(double x, const double *node, int32_t n, int32_t *first,
                       double w[4], double dw[4])
{
    if (n < 2 || !(x >= node[0] && x <= node[n - 1])) return 0;
    int32_t lo = 0, hi = n - 1; /* node[lo] <= x, and x <= node[hi] */
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) / 2;
        if (node[mid] <= x) lo = mid; else hi = mid;
    }
    int32_t i = lo;
    double h = node[i + 1] - node[i];
    double t = (x - node[i]) / h;
    if (i == 0 || i == n - 2) {
        *first = i;
        w[0] = 1.0 - t;  dw[0] = -1.0 / h;
        w[1] = t;        dw[1] = 1.0 / h;
        return 2;
    }
    *first = i - 1;
    for (int m = 0; m < 4; ++m) {
        double s = t + 1.0 - (double)m; /* signed index-space distance to node i-1+m */
        w[m] = keys_kernel(s);
        dw[m] = keys_kernel_deriv(s) / h;
    }
    return 4;
}

/* Surface value at (phase p, rest wavelength lam), with d/dp and d/dlam.
 * Zero (with zero derivatives) outside the grid. */
double om_surface(const om_model *m, const double *G, double p, double lam,
                  double *d_p, double *d_lam)
{
    int32_t fp = 0, fl = 0;
    double wp[4], dwp[4], wl[4], dwl[4];
    int np = m->pnode ? om_axis_taps_nodes(p, m->pnode, m->n_phase, &fp, wp, dwp)
                      : om_axis_taps(p, m->phase0, m->dphase, m->n_phase, &fp, wp, dwp);
    int nl = m->wnode ? om_axis_taps_nodes(lam, m->wnode, m->n_wave, &fl, wl, dwl)
                      : om_axis_taps(lam, m->wave0, m->dwave, m->n_wave, &fl, wl, dwl);
    double v = 0.0, vp = 0.0, vl = 0.0;
    for (int a = 0; a < np; ++a)
        for (int b = 0; b < nl; ++b) {
            double g = G[(size_t)(fp + a) * (size_t)m->n_wave + (size_t)(fl + b)];
            v += wp[a] * wl[b] * g;
            vp += dwp[a] * wl[b] * g;
            vl += wp[a] * dwl[b] * g;
        }
    if (d_p) *d_p = vp;
    if (d_lam) *d_lam = vl;
    return v;
}

/* ------------------------------------------------------------------------ */
/* Colour law (SALT2 form). With x = (lam - lambda_B)/(lambda_V - lambda_B):
 *   P(x) = (1 - a1 - a2 - a3 - a4) x + a1 x^2 + a2 x^3 + a3 x^4 + a4 x^5,
 *   CL(lam) = -P(x) on [cl_lo, cl_hi]; outside, P is continued linearly with
 *   its value and slope at the nearer end. Returns CL and dCL/dlam.        */

static double cl_P(const double a[4], double x)
{
    double lin = 1.0 - a[0] - a[1] - a[2] - a[3];
    return lin * x + a[0] * pow(x, 2) + a[1] * pow(x, 3) + a[2] * pow(x, 4) + a[3] * pow(x, 5);
}

static double cl_dP(const double a[4], double x)
{
    double lin = 1.0 - a[0] - a[1] - a[2] - a[3];
    return lin + 2.0 * a[0] * x + 3.0 * a[1] * pow(x, 2) + 4.0 * a[2] * pow(x, 3) +
           5.0 * a[3] * pow(x, 4);
}

double om_colorlaw(const double a[4], double cl_lo, double cl_hi, double lam, double *d_lam)
{
    double span = OM_LAMBDA_V - OM_LAMBDA_B;
    double x = (lam - OM_LAMBDA_B) / span;
    double P, dP;
    if (lam < cl_lo) {
        double xe = (cl_lo - OM_LAMBDA_B) / span;
        dP = cl_dP(a, xe);
        P = cl_P(a, xe) + dP * (x - xe);
    } else if (lam > cl_hi) {
        double xe = (cl_hi - OM_LAMBDA_B) / span;
        dP = cl_dP(a, xe);
        P = cl_P(a, xe) + dP * (x - xe);
    } else {
        P = cl_P(a, x);
        dP = cl_dP(a, x);
    }
    if (d_lam) *d_lam = -dP / span;
    return -P;
}

/* ------------------------------------------------------------------------ */
/* Observer-frame model flux density at observer wavelength lam_obs and epoch
 * mjd for par = (z, t0, x0, x1, c); d (nullable) receives dF/dpar.          */
double om_flux_obs(const om_model *m, double lam_obs, double mjd, const double par[5],
                   double d[5])
{
    double z = par[0], t0 = par[1], x0 = par[2], x1 = par[3], c = par[4];
    double opz = 1.0 + z;
    double p = (mjd - t0) / opz;
    double lr = lam_obs / opz;
    double m0p, m0l, m1p, m1l, dcl;
    double M0 = om_surface(m, m->m0, p, lr, &m0p, &m0l);
    double M1 = om_surface(m, m->m1, p, lr, &m1p, &m1l);
    double CL = om_colorlaw(m->cl, m->cl_lo, m->cl_hi, lr, &dcl);
    double C = pow(10.0, -0.4 * c * CL);
    double S = M0 + x1 * M1;
    double F = x0 * S * C / opz;
    if (d) {
        double ln10 = log(10.0);
        double S_p = m0p + x1 * m1p, S_l = m0l + x1 * m1l;
        double C_l = C * (-0.4 * ln10 * c * dcl);
        double p_z = -p / opz, l_z = -lr / opz;
        d[0] = -F / opz + x0 / opz * ((S_p * p_z + S_l * l_z) * C + S * C_l * l_z);
        d[1] = x0 * C / opz * S_p * (-1.0 / opz);
        d[2] = S * C / opz;
        d[3] = x0 * M1 * C / opz;
        d[4] = F * (-0.4 * ln10 * CL);
    }
    return F;
}

/* Trapezoidal rule on the samples (x_k, y_k). */
double om_trapz(int32_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (int32_t k = 0; k + 1 < n; ++k) s += 0.5 * (x[k + 1] - x[k]) * (y[k] + y[k + 1]);
    return s;
}

/* Photon-count integral of the AB reference spectrum through the band:
 * integral f_AB(lam) T(lam) lam / (h c) dlam, f_AB = 3631 Jy * c / lam^2.  */
double om_band_ab_flux(const om_band *b)
{
    double s = 0.0;
    for (int32_t k = 0; k + 1 < b->n; ++k) {
        double g0 = OM_AB_FNU * OM_C_AA_S / (b->wave[k] * b->wave[k]) * b->trans[k] *
                    b->wave[k] / (OM_H_ERG_S * OM_C_AA_S);
        double g1 = OM_AB_FNU * OM_C_AA_S / (b->wave[k + 1] * b->wave[k + 1]) * b->trans[k + 1] *
                    b->wave[k + 1] / (OM_H_ERG_S * OM_C_AA_S);
        s += 0.5 * (b->wave[k + 1] - b->wave[k]) * (g0 + g1);
    }
    return s;
}

/* Bandflux of one observation (band b, epoch mjd, zero point zp) for one
 * parameter vector, in the zp-scaled AB system; grad (nullable) receives
 * d bandflux / d(z, t0, x0, x1, c). */
double om_bandflux_one(const om_model *m, const om_band *b, double mjd, double zp,
                       const double par[5], double grad[5])
{
    double B = 0.0, dB[5] = {0, 0, 0, 0, 0};
    double hc = OM_H_ERG_S * OM_C_AA_S;
    double g_prev = 0.0, dg_prev[5] = {0, 0, 0, 0, 0};
    for (int32_t k = 0; k < b->n; ++k) {
        double d[5];
        double F = om_flux_obs(m, b->wave[k], mjd, par, grad ? d : NULL);
        double scale = b->trans[k] * b->wave[k] / hc;
        double g = F * scale;
        if (k > 0) {
            double h = b->wave[k] - b->wave[k - 1];
            B += 0.5 * h * (g_prev + g);
            if (grad)
                for (int q = 0; q < 5; ++q) dB[q] += 0.5 * h * (dg_prev[q] + d[q] * scale);
        }
        g_prev = g;
        if (grad)
            for (int q = 0; q < 5; ++q) dg_prev[q] = d[q] * scale;
    }
    double zpscale = pow(10.0, 0.4 * zp) / om_band_ab_flux(b);
    if (grad)
        for (int q = 0; q < 5; ++q) grad[q] = dB[q] * zpscale;
    return B * zpscale;
}

/* ------------------------------------------------------------------------ */
/* Batched forms over the ragged CSR batch. Supernova s owns observations
 * [obs_off[s], obs_off[s+1]) and parameter samples [par_off[s], par_off[s+1]).
 * par_f32 holds (z, x0, x1, c) per sample as 4 separate arrays.            */

typedef struct {
    int64_t n_sn;
    const int64_t *obs_off;
    const double *mjd;
    const int32_t *band;
    const double *flux, *fluxerr, *zp;
    const int64_t *par_off;
    const double *t0, *z, *x0, *x1, *c;
} om_batch;

static int om_threads = 1;

void om_set_threads(int n)
{
    om_threads = n > 0 ? n : 1;
}

int om_get_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* out[bf_off[s] + j * n_s + i] with bf_off[s] = sum_{s' < s} S_{s'} n_{s'}. */
void om_bandflux_batch(const om_model *m, const om_band *bands, const om_batch *bt,
                       const int64_t *bf_off, double *out)
{
#pragma omp parallel for schedule(dynamic, 1) num_threads(om_threads)
    for (int64_t s = 0; s < bt->n_sn; ++s) {
        int64_t o0 = bt->obs_off[s], ns = bt->obs_off[s + 1] - o0;
        for (int64_t j = bt->par_off[s]; j < bt->par_off[s + 1]; ++j) {
            double par[5] = {bt->z[j], bt->t0[j], bt->x0[j], bt->x1[j], bt->c[j]};
            int64_t jj = j - bt->par_off[s];
            for (int64_t i = 0; i < ns; ++i) {
                int64_t o = o0 + i;
                out[bf_off[s] + jj * ns + i] =
                    om_bandflux_one(m, &bands[bt->band[o]], bt->mjd[o], bt->zp[o], par, NULL);
            }
        }
    }
}

/* chi2[j] for every sample j; grad (nullable) is [n_par][5] = d chi2 / d(z, t0, x0, x1, c).
 * Samples are independent: the threads share them out one sample at a time. */
void om_chi2_batch(const om_model *m, const om_band *bands, const om_batch *bt, double *chi2,
                   double *grad)
{
    int64_t n_par = bt->n_sn > 0 ? bt->par_off[bt->n_sn] : 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(om_threads)
    for (int64_t j = 0; j < n_par; ++j) {
        int64_t lo = 0, hi = bt->n_sn; /* supernova s of sample j: par_off[s] <= j < par_off[s+1] */
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (bt->par_off[mid] <= j) lo = mid; else hi = mid;
        }
        int64_t s = lo;
        int64_t o0 = bt->obs_off[s], o1 = bt->obs_off[s + 1];
        double par[5] = {bt->z[j], bt->t0[j], bt->x0[j], bt->x1[j], bt->c[j]};
        double x2 = 0.0, g[5] = {0, 0, 0, 0, 0};
        for (int64_t o = o0; o < o1; ++o) {
            double dB[5];
            double B = om_bandflux_one(m, &bands[bt->band[o]], bt->mjd[o], bt->zp[o], par,
                                       grad ? dB : NULL);
            double r = (bt->flux[o] - B) / bt->fluxerr[o];
            x2 += r * r;
            if (grad)
                for (int q = 0; q < 5; ++q) g[q] += -2.0 * r / bt->fluxerr[o] * dB[q];
        }
        chi2[j] = x2;
        if (grad)
            for (int q = 0; q < 5; ++q) grad[5 * j + q] = g[q];
    }
}
