/*
 * Plain FP64 CPU oracle for the stochastic Richards' equation solve.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).
 *
 * Everything here is written for a reader to check against the paper by eye:
 * straight loops, no blocking, no fusion, no reordering.  Compiled with
 * -O2 -ffp-contract=off so that no multiply-add is contracted.
 *
 * Array layout: row-major [nz][nx], index j*nx + i, cell (i, j) has centre
 * ((i + 1/2) h, (j + 1/2) h), j = 0 is the bottom row, z points up (Eq. Grid_fine).
 * The mesh width is h = 1/nz (unit height; width nx*h).
 *
 * Readings of the paper taken here (each one is listed with its reason in the
 * design notes of the repository):
 *  R1 gravity: q = -K (grad p + e_z) with z the upward elevation (Eq. darcy).
 *  R2 Dirichlet face: distance h/2, conductivity K(p_D) evaluated with the
 *     adjacent cell's Ks and alpha ("modified appropriately", Sec. 4.2).
 *  R3 correction dp = 0 on Dirichlet faces, zero normal flux on the sides
 *     (garbled boundary line of Eq. diffusion_problem).
 *  R6 coarse mass term and coarse Dirichlet coefficients: arithmetic means,
 *     rediscretised with H = 2h, like the face coefficients (Fig. diffUpscale).
 *  R10 MG stop: ||f - A dp||_inf < eps_MG * max(1, ||f||_inf) (Sec. 4.2 states
 *     the absolute form; the factor only matters when ||f||_inf > 1, where the
 *     absolute 1e-10 lies below the FP64 rounding floor on fine grids).
 */
#include "richards_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, as defined by Salmon, Moraes, Dror and Shaw, "Parallel      */
/* random numbers: as easy as 1, 2, 3", SC'11: ten rounds of the Philox      */
/* S-box (two 32x32->64 multiplies) with a Weyl-sequence key schedule.        */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from the top 53 bits of a 64-bit word made of two outputs. */
static double orc_u01(uint32_t hi, uint32_t lo)
{
    uint64_t m = (((uint64_t)hi << 32) | (uint64_t)lo) >> 11;
    return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

/* Standard normal white noise y for one (sample, field) on npts torus points.
 * Key = (low word of seed, high word of seed XOR level); counter =
 * (pair index, field, low word of sample, high word of sample).  Each Philox
 * call gives two uniforms and, by Box-Muller, the normals of points 2q, 2q+1. */
void orc_white_noise(uint64_t seed, uint32_t level, uint64_t sample, uint32_t field,
                     int64_t npts, double* y)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) ^ level };
    for (int64_t q = 0; 2 * q < npts; ++q) {
        uint32_t ctr[4] = { (uint32_t)q, field, (uint32_t)sample, (uint32_t)(sample >> 32) };
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        double u1 = orc_u01(x[0], x[1]);
        double u2 = orc_u01(x[2], x[3]);
        double r = sqrt(-2.0 * log(u1));
        double t = two_pi * u2;
        y[2 * q] = r * cos(t);
        if (2 * q + 1 < npts) y[2 * q + 1] = r * sin(t);
    }
}

/* ------------------------------------------------------------------------- */
/* Radix-2 complex FFT (Cooley-Tukey, bit reversal then butterflies).         */
/* forward: X_k = sum_n x_n exp(-2 pi i k n / N); inverse divides by N.       */
/* ------------------------------------------------------------------------- */
static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static void fft1(double* re, double* im, int n, int inverse)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    const double pi = 3.14159265358979323846264338327950;
    for (int len = 2; len <= n; len <<= 1) {
        double ang = (inverse ? 2.0 : -2.0) * pi / (double)len;
        for (int b = 0; b < n; b += len) {
            for (int k = 0; k < len / 2; ++k) {
                double wr = cos(ang * k), wi = sin(ang * k);
                int a = b + k, c = b + k + len / 2;
                double xr = re[c] * wr - im[c] * wi;
                double xi = re[c] * wi + im[c] * wr;
                re[c] = re[a] - xr; im[c] = im[a] - xi;
                re[a] = re[a] + xr; im[a] = im[a] + xi;
            }
        }
    }
    if (inverse) {
        for (int i = 0; i < n; ++i) { re[i] /= (double)n; im[i] /= (double)n; }
    }
}

int orc_fft2(double* re, double* im, int32_t nx, int32_t nz, int32_t inverse)
{
    if (!is_pow2(nx) || !is_pow2(nz)) return -1;
    int nmax = nx > nz ? nx : nz;
    double* tr = (double*)malloc(sizeof(double) * nmax);
    double* ti = (double*)malloc(sizeof(double) * nmax);
    for (int j = 0; j < nz; ++j) fft1(re + (size_t)j * nx, im + (size_t)j * nx, nx, inverse);
    for (int i = 0; i < nx; ++i) {
        for (int j = 0; j < nz; ++j) { tr[j] = re[(size_t)j * nx + i]; ti[j] = im[(size_t)j * nx + i]; }
        fft1(tr, ti, nz, inverse);
        for (int j = 0; j < nz; ++j) { re[(size_t)j * nx + i] = tr[j]; im[(size_t)j * nx + i] = ti[j]; }
    }
    free(tr); free(ti);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Modified Bessel function of the second kind, x > 0, nu >= 0, from its       */
/* integral representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt    */
/* (DLMF 10.32.9) by the trapezoidal rule: the integrand is analytic and even  */
/* with doubly exponential decay, so the rule converges geometrically          */
/* (Trefethen and Weideman, SIAM Review 56, 2014).  Near t = 0 it behaves like */
/* exp(-x t^2 / 2), so the step is min(1/16, 1/(2 sqrt x)), which keeps the     */
/* aliasing error of that Gaussian below exp(-8 pi^2).  The sum stops once a   */
/* term is below 1e-18 of the sum and past the integrand's maximum.            */
/* ------------------------------------------------------------------------- */
double orc_bessel_k(double nu, double x)
{
    const double tau = x > 64.0 ? 0.5 / sqrt(x) : 1.0 / 16.0;
    double sum = 0.5 * exp(-x);
    for (int k = 1; k < 4096; ++k) {
        double t = k * tau;
        double term = exp(-x * cosh(t)) * cosh(nu * t);
        sum += term;
        if (term <= 1e-18 * sum && x * sinh(t) > nu) break;
    }
    return tau * sum;
}

/* Covariance of the Gaussian fields at offset (dx, dz).  nu > 0: the          */
/* anisotropic Matern function of Eq. nonIsotropic,                            */
/*   sigma2 2^(1-nu)/Gamma(nu) (2 sqrt(nu) r)^nu K_nu(2 sqrt(nu) r),           */
/*   r = sqrt((dx/lx)^2 + (dz/lz)^2)  (value sigma2 at r = 0);                 */
/* nu = 0: the exponential sigma2 exp(-r) (with lz = lx: exp(-|d|/lx)).        */
/* Supported: 0 < nu <= 16 (Gamma(nu) and x^nu stay finite).                   */
/* lz <= 0 means lz = lx (isotropic).                                          */
/* ------------------------------------------------------------------------- */
double orc_covariance(const orc_cov* cv, double dx, double dz)
{
    double lx = cv->corr_len, lz = cv->corr_len_z > 0.0 ? cv->corr_len_z : cv->corr_len;
    double r = (lz == lx) ? sqrt(dx * dx + dz * dz) / lx : sqrt((dx / lx) * (dx / lx) + (dz / lz) * (dz / lz));
    if (!(cv->nu > 0.0)) return cv->sigma2 * exp(-r);
    if (r == 0.0) return cv->sigma2;
    double x = 2.0 * sqrt(cv->nu) * r;
    return cv->sigma2 * pow(2.0, 1.0 - cv->nu) / tgamma(cv->nu) * pow(x, cv->nu) * orc_bessel_k(cv->nu, x);
}

/* ------------------------------------------------------------------------- */
/* FFT-MA (Appendix A).  The covariance is sampled on a px x pz torus with    */
/* periodic distances; its DFT is the spectrum Lambda of the circulant        */
/* covariance; F(s) = sqrt(Lambda) (Eq. product1) and z = F^-1(F(s) . F(y))   */
/* (Eq. product2 and the one after).                                          */
/* ------------------------------------------------------------------------- */
int orc_fftma_spectrum(int32_t px, int32_t pz, double h, const orc_cov* cv,
                       double* sqrt_lambda, double* min_ratio)
{
    size_t n = (size_t)px * pz;
    double* re = (double*)malloc(sizeof(double) * n);
    double* im = (double*)calloc(n, sizeof(double));
    for (int b = 0; b < pz; ++b)
        for (int a = 0; a < px; ++a) {
            int ia = a < px - a ? a : px - a;
            int ib = b < pz - b ? b : pz - b;
            re[(size_t)b * px + a] = orc_covariance(cv, ia * h, ib * h);
        }
    int rc = orc_fft2(re, im, px, pz, 0);
    if (rc) { free(re); free(im); return rc; }
    double lmin = re[0], lmax = re[0];
    for (size_t k = 0; k < n; ++k) { if (re[k] < lmin) lmin = re[k]; if (re[k] > lmax) lmax = re[k]; }
    if (min_ratio) *min_ratio = lmin / lmax;
    for (size_t k = 0; k < n; ++k) sqrt_lambda[k] = re[k] > 0.0 ? sqrt(re[k]) : 0.0;
    free(re); free(im);
    return 0;
}

static int next_pow2(int n) { int p = 1; while (p < n) p <<= 1; return p; }

/* Smallest torus (powers of two, at least twice the grid per side, grown by  */
/* doubling) whose spectrum has no eigenvalue below -1e-12 * max.             */
int orc_torus_size(int32_t nx, int32_t nz, double h, const orc_cov* cv, int32_t* px, int32_t* pz)
{
    int a = next_pow2(2 * nx), b = next_pow2(2 * nz);
    for (int tries = 0; tries < 4; ++tries) {
        double* s = (double*)malloc(sizeof(double) * (size_t)a * b);
        double ratio = 0.0;
        orc_fftma_spectrum(a, b, h, cv, s, &ratio);
        free(s);
        if (ratio >= -1e-12) { *px = a; *pz = b; return 0; }
        a *= 2; b *= 2;
    }
    *px = a / 2; *pz = b / 2;   /* negative eigenvalues are clipped to zero */
    return 1;
}

/* Fields of one draw: field 0 is Gaussian (out = shift0 + z), fields f >= 1
 * are lo[f] + span[f] * Phi(z / sigma) with Phi(x) = erfc(-x / sqrt 2) / 2
 * (the relation Y = F_Y^-1(F_Z(Z)) of Sec. 3.1 for a uniform marginal); all
 * are then 2x2-averaged `coarsen` times.  Field f uses noise stream f. */
#define ORC_MAX_FIELDS 5
typedef struct {
    uint64_t seed; double sigma2; int32_t nf; double shift0;
    double lo[ORC_MAX_FIELDS], span[ORC_MAX_FIELDS]; double* out[ORC_MAX_FIELDS];
    int32_t nx, nz, px, pz; uint32_t level; int64_t first; int32_t ns, coarsen;
    const double* sq; int32_t nthreads, tid;
} orc_field_job;

static void* field_worker(void* arg)
{
    orc_field_job* J = (orc_field_job*)arg;
    size_t n = (size_t)J->px * J->pz;
    int nxo = J->nx >> J->coarsen, nzo = J->nz >> J->coarsen;
    double* re = (double*)malloc(sizeof(double) * n);
    double* im = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * (size_t)J->nx * J->nz);
    double sig = sqrt(J->sigma2);
    for (int k = J->tid; k < J->ns; k += J->nthreads) {
        uint64_t sample = (uint64_t)(J->first + k);
        for (int fld = 0; fld < J->nf; ++fld) {
            orc_white_noise(J->seed, J->level, sample, (uint32_t)fld, (int64_t)n, re);
            memset(im, 0, sizeof(double) * n);
            orc_fft2(re, im, J->px, J->pz, 0);
            for (size_t q = 0; q < n; ++q) { re[q] *= J->sq[q]; im[q] *= J->sq[q]; }
            orc_fft2(re, im, J->px, J->pz, 1);
            for (int j = 0; j < J->nz; ++j)
                for (int i = 0; i < J->nx; ++i) {
                    double v = re[(size_t)j * J->px + i];
                    z[(size_t)j * J->nx + i] = fld == 0 ? J->shift0 + v
                        : J->lo[fld] + J->span[fld] * 0.5 * erfc(-(v / sig) / sqrt(2.0));
                }
            /* 2x2 averaging, coarsen times */
            int cx = J->nx, cz = J->nz;
            for (int c = 0; c < J->coarsen; ++c) {
                int ncx = cx / 2, ncz = cz / 2;
                for (int j = 0; j < ncz; ++j)
                    for (int i = 0; i < ncx; ++i) {
                        double t = z[(size_t)(2 * j) * cx + 2 * i] + z[(size_t)(2 * j) * cx + 2 * i + 1]
                                 + z[(size_t)(2 * j + 1) * cx + 2 * i] + z[(size_t)(2 * j + 1) * cx + 2 * i + 1];
                        z[(size_t)j * ncx + i] = 0.25 * t;
                    }
                cx = ncx; cz = ncz;
            }
            memcpy(J->out[fld] + (size_t)k * nxo * nzo, z, sizeof(double) * (size_t)nxo * nzo);
        }
    }
    free(re); free(im); free(z);
    return NULL;
}

static int sample_n(uint64_t seed, const orc_cov* cv, int nf, double shift0, const double* lo,
                    const double* span, double** out, int32_t nx, int32_t nz, uint32_t level,
                    int64_t first_sample, int32_t nsamples, int32_t coarsen_times, int32_t nthreads)
{
    if (nx < 1 || nz < 1 || nsamples < 0 || coarsen_times < 0) return -1;
    if ((nx % (1 << coarsen_times)) || (nz % (1 << coarsen_times))) return -1;
    double h = 1.0 / nz;
    int32_t px, pz;
    orc_torus_size(nx, nz, h, cv, &px, &pz);
    double* sq = (double*)malloc(sizeof(double) * (size_t)px * pz);
    double ratio;
    orc_fftma_spectrum(px, pz, h, cv, sq, &ratio);
    if (nthreads < 1) nthreads = 1;
    orc_field_job* jobs = (orc_field_job*)malloc(sizeof(orc_field_job) * nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        orc_field_job J;
        memset(&J, 0, sizeof J);
        J.seed = seed; J.sigma2 = cv->sigma2; J.nf = nf; J.shift0 = shift0;
        for (int f = 0; f < nf; ++f) { J.lo[f] = lo[f]; J.span[f] = span[f]; J.out[f] = out[f]; }
        J.nx = nx; J.nz = nz; J.px = px; J.pz = pz; J.level = level; J.first = first_sample;
        J.ns = nsamples; J.coarsen = coarsen_times; J.sq = sq; J.nthreads = nthreads; J.tid = t;
        jobs[t] = J;
        pthread_create(&th[t], NULL, field_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th); free(sq);
    return 0;
}

/* ln Ks = z_0 (Eq. RandK with Ks^(bl) = 1) and alpha = lo + span Phi(z_1 / sigma) */
int orc_sample_fields(uint64_t seed, const orc_cov* cv, double alpha_lo,
                      double alpha_span, int32_t nx, int32_t nz, uint32_t level,
                      int64_t first_sample, int32_t nsamples, int32_t coarsen_times,
                      double* lnKs, double* alpha, int32_t nthreads)
{
    double lo[2] = { 0.0, alpha_lo }, span[2] = { 0.0, alpha_span };
    double* out[2] = { lnKs, alpha };
    return sample_n(seed, cv, 2, 0.0, lo, span, out, nx, nz, level, first_sample, nsamples,
                    coarsen_times, nthreads);
}

/* The five soil fields of Table soilparams: ln Ks (noise stream 0), alpha (1),
 * n (2), theta_s (3), theta_r (4). */
int orc_sample_soil(uint64_t seed, const orc_cov* cv, const orc_soil_model* sm, int32_t nx, int32_t nz,
                    uint32_t level, int64_t first_sample, int32_t nsamples, int32_t coarsen_times,
                    double* lnKs, double* alpha, double* n, double* theta_s, double* theta_r,
                    int32_t nthreads)
{
    double lo[5] = { 0.0, sm->alpha_lo, sm->n_lo, sm->theta_s_lo, sm->theta_r_lo };
    double span[5] = { 0.0, sm->alpha_span, sm->n_span, sm->theta_s_span, sm->theta_r_span };
    double* out[5] = { lnKs, alpha, n, theta_s, theta_r };
    return sample_n(seed, cv, 5, sm->lnks_mean, lo, span, out, nx, nz, level, first_sample, nsamples,
                    coarsen_times, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Covariance upscaling (Appendix A, Eqs. averaging, cov_upscale): white noise */
/* y on the fine torus gives the fine field; the coarse noise                  */
/* y_c(I,J) = (1/2) * (sum of the 2x2 block of y) on the half-size torus gives  */
/* the coarse field through the coarse grid's own spectrum (spacing 2h).       */
/* ------------------------------------------------------------------------- */
static int sample_pair_n(uint64_t seed, const orc_cov* cv, int nf, double shift0, const double* lo,
                         const double* span, double** outf, double** outc, int32_t nx, int32_t nz,
                         uint32_t level, int64_t first_sample, int32_t nsamples)
{
    if (nx < 2 || nz < 2 || nx % 2 || nz % 2 || nsamples < 0) return -1;
    double h = 1.0 / nz;
    int32_t px, pz;
    orc_torus_size(nx, nz, h, cv, &px, &pz);
    int pxc = px / 2, pzc = pz / 2, ncx = nx / 2, ncz = nz / 2;
    size_t nf_ = (size_t)px * pz, nc = (size_t)pxc * pzc;
    double* sqf = (double*)malloc(sizeof(double) * nf_);
    double* sqc = (double*)malloc(sizeof(double) * nc);
    double ratio;
    orc_fftma_spectrum(px, pz, h, cv, sqf, &ratio);
    orc_fftma_spectrum(pxc, pzc, 2.0 * h, cv, sqc, &ratio);
    double* y = (double*)malloc(sizeof(double) * nf_);
    double* re = (double*)malloc(sizeof(double) * nf_);
    double* im = (double*)malloc(sizeof(double) * nf_);
    double sig = sqrt(cv->sigma2);
    for (int k = 0; k < nsamples; ++k) {
        uint64_t sample = (uint64_t)(first_sample + k);
        for (int fld = 0; fld < nf; ++fld) {
            orc_white_noise(seed, level, sample, (uint32_t)fld, (int64_t)nf_, y);
            for (int pass = 0; pass < 2; ++pass) {
                /* pass 0: the fine member from y; pass 1: the coarse member
                 * from y_c(I,J) = (1/2) (sum of the 2x2 block of y) */
                int tx = pass ? pxc : px, tz = pass ? pzc : pz, ox = pass ? ncx : nx, oz = pass ? ncz : nz;
                const double* sq = pass ? sqc : sqf;
                double* out = (pass ? outc[fld] : outf[fld]) + (size_t)k * ox * oz;
                if (pass == 0) {
                    memcpy(re, y, sizeof(double) * nf_);
                } else {
                    for (int J = 0; J < pzc; ++J)
                        for (int I = 0; I < pxc; ++I) {
                            size_t a = (size_t)(2 * J) * px + 2 * I, b = a + px;
                            re[(size_t)J * pxc + I] = 0.5 * (y[a] + y[a + 1] + y[b] + y[b + 1]);
                        }
                }
                memset(im, 0, sizeof(double) * (size_t)tx * tz);
                orc_fft2(re, im, tx, tz, 0);
                for (size_t q = 0; q < (size_t)tx * tz; ++q) { re[q] *= sq[q]; im[q] *= sq[q]; }
                orc_fft2(re, im, tx, tz, 1);
                for (int j = 0; j < oz; ++j)
                    for (int i = 0; i < ox; ++i) {
                        double v = re[(size_t)j * tx + i];
                        out[(size_t)j * ox + i] = fld == 0 ? shift0 + v
                            : lo[fld] + span[fld] * 0.5 * erfc(-(v / sig) / sqrt(2.0));
                    }
            }
        }
    }
    free(sqf); free(sqc); free(y); free(re); free(im);
    return 0;
}

int orc_sample_fields_pair(uint64_t seed, const orc_cov* cv, double alpha_lo,
                           double alpha_span, int32_t nx, int32_t nz, uint32_t level,
                           int64_t first_sample, int32_t nsamples, double* lnKs_f, double* alpha_f,
                           double* lnKs_c, double* alpha_c)
{
    double lo[2] = { 0.0, alpha_lo }, span[2] = { 0.0, alpha_span };
    double* of[2] = { lnKs_f, alpha_f };
    double* oc[2] = { lnKs_c, alpha_c };
    return sample_pair_n(seed, cv, 2, 0.0, lo, span, of, oc, nx, nz, level, first_sample, nsamples);
}

/* The five soil fields as fine / coarse couples by covariance upscaling;
 * outputs [5] arrays each, in the order ln Ks, alpha, n, theta_s, theta_r. */
int orc_sample_soil_pair(uint64_t seed, const orc_cov* cv, const orc_soil_model* sm, int32_t nx, int32_t nz,
                         uint32_t level, int64_t first_sample, int32_t nsamples, double** fine,
                         double** coarse)
{
    double lo[5] = { 0.0, sm->alpha_lo, sm->n_lo, sm->theta_s_lo, sm->theta_r_lo };
    double span[5] = { 0.0, sm->alpha_span, sm->n_span, sm->theta_s_span, sm->theta_r_span };
    return sample_pair_n(seed, cv, 5, sm->lnks_mean, lo, span, fine, coarse, nx, nz, level, first_sample,
                         nsamples);
}

/* ------------------------------------------------------------------------- */
/* Closures.  K, theta and C = d theta / d p at head p for one cell.          */
/* Gardner exponential model (kind 0):                                        */
/*   p < 0 : E = exp(a p), K = Ks E, theta = theta_r + (theta_s - theta_r) E, */
/*           C = (theta_s - theta_r) a E                                      */
/* van Genuchten-Mualem (kind 1; Eqs. Sw, sc_van, Krw), m = 1 - 1/n:          */
/*   p < 0 : an = (a |p|)^n, S = (1 + an)^-m, theta = theta_r + (theta_s -    */
/*           theta_r) S, C = (theta_s - theta_r) a m n (1 + an)^-(m+1)        */
/*           (a |p|)^(n-1), K = Ks S^(1/2) (1 - (1 - S^(1/m))^m)^2 with the   */
/*           exact identity 1 - S^(1/m) = an / (1 + an) (no cancellation as   */
/*           S -> 1)                                                          */
/* Both: p >= 0 gives K = Ks, theta = theta_s, C = 0 (saturated branch).      */
/* ------------------------------------------------------------------------- */
typedef struct { double Ks, a, n, tr, ts; } cellp;

static void closure(int kind, const cellp* c, double p, double* K, double* theta, double* C)
{
    if (!(p < 0.0)) {
        *K = c->Ks;
        *theta = c->ts;
        *C = 0.0;
    } else if (kind == 0) {
        double E = exp(c->a * p);
        *K = c->Ks * E;
        *theta = c->tr + (c->ts - c->tr) * E;
        *C = (c->ts - c->tr) * c->a * E;
    } else {
        double m = 1.0 - 1.0 / c->n;
        double ap = c->a * fabs(p);
        double an = pow(ap, c->n);
        double S = pow(1.0 + an, -m);
        double b = 1.0 - pow(an / (1.0 + an), m);
        *K = c->Ks * sqrt(S) * b * b;
        *theta = c->tr + (c->ts - c->tr) * S;
        *C = (c->ts - c->tr) * c->a * m * c->n * pow(1.0 + an, -(m + 1.0)) * pow(ap, c->n - 1.0);
    }
}

int orc_closure(int32_t kind, double Ks, double a, double n, double theta_r, double theta_s,
                double p, double* K, double* theta, double* C)
{
    if (kind != 0 && kind != 1) return -1;
    cellp c = { Ks, a, n, theta_r, theta_s };
    closure(kind, &c, p, K, theta, C);
    return 0;
}

/* parameters of cell q of one sample (soil pointers already offset) */
static cellp cell_at(const orc_problem* pb, const orc_soil* so, size_t q)
{
    cellp c;
    c.Ks = exp(so->lnKs[q]);
    c.a = so->alpha[q] * so->alpha_scale + so->alpha_shift;
    c.n = so->n ? so->n[q] + so->n_shift : 0.0;
    c.tr = (pb->closure == 1 && so->theta_r) ? so->theta_r[q] : pb->theta_r;
    c.ts = (pb->closure == 1 && so->theta_s) ? so->theta_s[q] : pb->theta_s;
    return c;
}

/* Conductivity on a Dirichlet face (reading R2): the closure's K at the
 * boundary head with the adjacent cell's parameters. */
static double k_dirichlet(int kind, const cellp* c, double pD)
{
    double K, th, C;
    closure(kind, c, pD, &K, &th, &C);
    return K;
}

/* ------------------------------------------------------------------------- */
/* Picard system (Eqs. Mixed_based_3, diffusion_problem, five_stencil).       */
/* Transmissibilities per unit cell area:                                     */
/*   interior face  T = (2/h^2) K_P K_N / (K_P + K_N)   (harmonic mean / h^2) */
/*   Dirichlet face T_b = 2 K_b / h^2                    (distance h/2)       */
/* Outward flux per unit area of cell P through each face (Eq. darcy, R1):   */
/*   east/west  -T (p_nb - p_P)                                               */
/*   north      -T (p_N - p_P) - T h        south  -T (p_S - p_P) + T h       */
/*   top        -Tb (p_top - p_P) - Tb h/2  bottom  Tb (p_P - p_bot) + Tb h/2 */
/* Residual R_P = (theta_P - theta_P^old)/dt + sum(out-fluxes) - src_P, and   */
/* the Picard system is  (C/dt) dp + L(T) dp = f := -R.                       */
/* ------------------------------------------------------------------------- */
static void picard_system(const orc_problem* pb, int32_t nx, int32_t nz, const orc_soil* so,
                          const double* p, const double* p_old, double* Tx, double* Tz,
                          double* Tbt, double* Tbb, double* Cdt, double* f)
{
    const double h = 1.0 / nz, h2 = h * h;
    const size_t n = (size_t)nx * nz;
    const int kind = pb->closure;
    double* K = (double*)malloc(sizeof(double) * n);
    double* th = (double*)malloc(sizeof(double) * n);
    double* C = (double*)malloc(sizeof(double) * n);
    for (size_t q = 0; q < n; ++q) {
        cellp c = cell_at(pb, so, q);
        closure(kind, &c, p[q], &K[q], &th[q], &C[q]);
    }
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t P = (size_t)j * nx + i;
            Tx[P] = (i < nx - 1) ? (2.0 / h2) * K[P] * K[P + 1] / (K[P] + K[P + 1]) : 0.0;
            Tz[P] = (j < nz - 1) ? (2.0 / h2) * K[P] * K[P + nx] / (K[P] + K[P + nx]) : 0.0;
        }
    for (int i = 0; i < nx; ++i) {
        cellp ct = cell_at(pb, so, (size_t)(nz - 1) * nx + i), cb = cell_at(pb, so, (size_t)i);
        Tbt[i] = (2.0 / h2) * k_dirichlet(kind, &ct, pb->p_top);
        Tbb[i] = (2.0 / h2) * k_dirichlet(kind, &cb, pb->p_bottom);
    }
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t P = (size_t)j * nx + i;
            double Kd, thold, Cd;
            cellp c = cell_at(pb, so, P);
            closure(kind, &c, p_old[P], &Kd, &thold, &Cd);
            double R = (th[P] - thold) / pb->dt;
            if (i < nx - 1) R += -Tx[P] * (p[P + 1] - p[P]);
            if (i > 0)      R += -Tx[P - 1] * (p[P - 1] - p[P]);
            if (j < nz - 1) R += -Tz[P] * (p[P + nx] - p[P]) - Tz[P] * h;
            else            R += -Tbt[i] * (pb->p_top - p[P]) - Tbt[i] * h / 2.0;
            if (j > 0)      R += -Tz[P - nx] * (p[P - nx] - p[P]) + Tz[P - nx] * h;
            else            R += Tbb[i] * (p[P] - pb->p_bottom) + Tbb[i] * h / 2.0;
            f[P] = -R;
            Cdt[P] = C[P] / pb->dt;
        }
    free(K); free(th); free(C);
}

int orc_picard_system(const orc_problem* pb, int32_t nx, int32_t nz, const double* lnKs,
                      const double* alpha, double alpha_scale, const double* p,
                      const double* p_old, double* Tx, double* Tz, double* Tbt,
                      double* Tbb, double* Cdt, double* f)
{
    if (pb->closure != 0) return -1;      /* the soil arrays of closure 1 are not given */
    orc_soil so = { lnKs, alpha, NULL, NULL, NULL, alpha_scale, 0.0, 0.0 };
    picard_system(pb, nx, nz, &so, p, p_old, Tx, Tz, Tbt, Tbb, Cdt, f);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Cell-centred multigrid (Sec. 4.2).                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nx, nz;
    double *Tx, *Tz, *Tbt, *Tbb, *Cdt, *D, *dp, *f, *r;
} mg_level;

static double diag_of(const mg_level* L, int i, int j)
{
    size_t P = (size_t)j * L->nx + i;
    double d = L->Cdt[P];
    if (i < L->nx - 1) d += L->Tx[P];
    if (i > 0)         d += L->Tx[P - 1];
    if (j < L->nz - 1) d += L->Tz[P];
    else               d += L->Tbt[i];
    if (j > 0)         d += L->Tz[P - L->nx];
    else               d += L->Tbb[i];
    return d;
}

/* sum over the neighbours of T * dp_nb (dp = 0 beyond Dirichlet faces) */
static double offdiag_sum(const mg_level* L, const double* x, int i, int j)
{
    size_t P = (size_t)j * L->nx + i;
    double s = 0.0;
    if (i < L->nx - 1) s += L->Tx[P] * x[P + 1];
    if (i > 0)         s += L->Tx[P - 1] * x[P - 1];
    if (j < L->nz - 1) s += L->Tz[P] * x[P + L->nx];
    if (j > 0)         s += L->Tz[P - L->nx] * x[P - L->nx];
    return s;
}

/* one red-black Gauss-Seidel step: red cells (i + j even) first, then black */
static void rbgs(mg_level* L)
{
    for (int colour = 0; colour < 2; ++colour)
        for (int j = 0; j < L->nz; ++j)
            for (int i = 0; i < L->nx; ++i) {
                if (((i + j) & 1) != colour) continue;
                size_t P = (size_t)j * L->nx + i;
                L->dp[P] = (L->f[P] + offdiag_sum(L, L->dp, i, j)) / L->D[P];
            }
}

/* r = f - A dp, returns ||r||_inf */
static double residual(mg_level* L)
{
    double m = 0.0;
    for (int j = 0; j < L->nz; ++j)
        for (int i = 0; i < L->nx; ++i) {
            size_t P = (size_t)j * L->nx + i;
            L->r[P] = L->f[P] - (L->D[P] * L->dp[P] - offdiag_sum(L, L->dp, i, j));
            double a = fabs(L->r[P]);
            if (!(a <= m)) m = a;   /* NaN propagates */
        }
    return m;
}

/* coarse operator: face coefficients are the arithmetic mean of the two fine
 * faces they cover, rescaled by (h/H)^2 = 1/4 (Fig. diffUpscale); mass term
 * and Dirichlet faces likewise (reading R6). */
static void coarsen_operator(const mg_level* F, mg_level* C)
{
    int nx = C->nx, nz = C->nz, fx = F->nx;
    for (int J = 0; J < nz; ++J)
        for (int I = 0; I < nx; ++I) {
            size_t P = (size_t)J * nx + I;
            size_t f00 = (size_t)(2 * J) * fx + 2 * I, f01 = f00 + fx;
            C->Tx[P] = (I < nx - 1) ? 0.25 * (0.5 * (F->Tx[f00 + 1] + F->Tx[f01 + 1])) : 0.0;
            C->Tz[P] = (J < nz - 1) ? 0.25 * (0.5 * (F->Tz[f01] + F->Tz[f01 + 1])) : 0.0;
            C->Cdt[P] = 0.25 * (F->Cdt[f00] + F->Cdt[f00 + 1] + F->Cdt[f01] + F->Cdt[f01 + 1]);
        }
    for (int I = 0; I < nx; ++I) {
        C->Tbt[I] = 0.25 * (0.5 * (F->Tbt[2 * I] + F->Tbt[2 * I + 1]));
        C->Tbb[I] = 0.25 * (0.5 * (F->Tbb[2 * I] + F->Tbb[2 * I + 1]));
    }
}

static void set_diag(mg_level* L)
{
    for (int j = 0; j < L->nz; ++j)
        for (int i = 0; i < L->nx; ++i) L->D[(size_t)j * L->nx + i] = diag_of(L, i, j);
}

/* exact solve on the coarsest grid: dense Gaussian elimination with partial
 * pivoting of the assembled five-point matrix */
static void coarse_solve(mg_level* L)
{
    int n = L->nx * L->nz;
    double* A = (double*)calloc((size_t)n * n, sizeof(double));
    double* b = (double*)malloc(sizeof(double) * n);
    for (int j = 0; j < L->nz; ++j)
        for (int i = 0; i < L->nx; ++i) {
            int P = j * L->nx + i;
            A[(size_t)P * n + P] = L->D[P];
            if (i < L->nx - 1) A[(size_t)P * n + P + 1] = -L->Tx[P];
            if (i > 0)         A[(size_t)P * n + P - 1] = -L->Tx[P - 1];
            if (j < L->nz - 1) A[(size_t)P * n + P + L->nx] = -L->Tz[P];
            if (j > 0)         A[(size_t)P * n + P - L->nx] = -L->Tz[P - L->nx];
            b[P] = L->f[P];
        }
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[(size_t)r * n + k]) > fabs(A[(size_t)piv * n + k])) piv = r;
        if (piv != k) {
            for (int c = 0; c < n; ++c) {
                double t = A[(size_t)k * n + c]; A[(size_t)k * n + c] = A[(size_t)piv * n + c]; A[(size_t)piv * n + c] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double m = A[(size_t)r * n + k] / A[(size_t)k * n + k];
            for (int c = k; c < n; ++c) A[(size_t)r * n + c] -= m * A[(size_t)k * n + c];
            b[r] -= m * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < n; ++c) s -= A[(size_t)k * n + c] * L->dp[c];
        L->dp[k] = s / A[(size_t)k * n + k];
    }
    free(A); free(b);
}

/* multigrid cycle on level l (recursive, Sec. 4.2): gamma = 1 gives the
 * V(nu1, nu2)-cycle, gamma = 2 the W(nu1, nu2)-cycle (gamma coarse-grid
 * cycles per visit; the exact coarsest solve is done once) */
static void mgcycle(mg_level* Ls, int l, int nlev, int nu1, int nu2, int gamma)
{
    mg_level* L = &Ls[l];
    if (l == nlev - 1) { coarse_solve(L); return; }
    for (int s = 0; s < nu1; ++s) rbgs(L);
    residual(L);
    mg_level* C = &Ls[l + 1];
    /* restriction R = 1/4 (sum of the four children), Eq. transfer */
    for (int J = 0; J < C->nz; ++J)
        for (int I = 0; I < C->nx; ++I) {
            size_t f00 = (size_t)(2 * J) * L->nx + 2 * I, f01 = f00 + L->nx;
            C->f[(size_t)J * C->nx + I] = 0.25 * (L->r[f00] + L->r[f00 + 1] + L->r[f01] + L->r[f01 + 1]);
            C->dp[(size_t)J * C->nx + I] = 0.0;
        }
    int reps = (l + 1 == nlev - 1) ? 1 : gamma;
    for (int g = 0; g < reps; ++g) mgcycle(Ls, l + 1, nlev, nu1, nu2, gamma);
    /* piecewise-constant prolongation, Eq. transfer */
    for (int j = 0; j < L->nz; ++j)
        for (int i = 0; i < L->nx; ++i)
            L->dp[(size_t)j * L->nx + i] += C->dp[(size_t)(j / 2) * C->nx + i / 2];
    for (int s = 0; s < nu2; ++s) rbgs(L);
}

/* number of levels: halve while both sides are even and more than 4 cells
 * remain; the coarsest grid must have at most 64 cells */
static int count_levels(int nx, int nz)
{
    int n = 1;
    while (nx % 2 == 0 && nz % 2 == 0 && nx * nz > 4) { nx /= 2; nz /= 2; ++n; }
    return (nx * nz <= 64) ? n : -1;
}

static mg_level* alloc_levels(int nx, int nz, int nlev)
{
    mg_level* Ls = (mg_level*)calloc(nlev, sizeof(mg_level));
    for (int l = 0; l < nlev; ++l) {
        size_t n = (size_t)nx * nz;
        Ls[l].nx = nx; Ls[l].nz = nz;
        Ls[l].Tx = (double*)calloc(n, 8); Ls[l].Tz = (double*)calloc(n, 8);
        Ls[l].Cdt = (double*)calloc(n, 8); Ls[l].D = (double*)calloc(n, 8);
        Ls[l].dp = (double*)calloc(n, 8); Ls[l].f = (double*)calloc(n, 8);
        Ls[l].r = (double*)calloc(n, 8);
        Ls[l].Tbt = (double*)calloc(nx, 8); Ls[l].Tbb = (double*)calloc(nx, 8);
        nx /= 2; nz /= 2;
    }
    return Ls;
}

static void free_levels(mg_level* Ls, int nlev)
{
    for (int l = 0; l < nlev; ++l) {
        free(Ls[l].Tx); free(Ls[l].Tz); free(Ls[l].Cdt); free(Ls[l].D);
        free(Ls[l].dp); free(Ls[l].f); free(Ls[l].r); free(Ls[l].Tbt); free(Ls[l].Tbb);
    }
    free(Ls);
}

static double inf_norm(const double* x, size_t n)
{
    double m = 0.0;
    for (size_t q = 0; q < n; ++q) { double a = fabs(x[q]); if (!(a <= m)) m = a; }
    return m;
}

/* MG solve of A dp = f from dp = 0: V-cycles until
 * ||f - A dp||_inf < tol * max(1, ||f||_inf) (reading R10) or maxit cycles.
 * Returns 0 if converged, 1 if not, 3 if the residual is not finite. */
static int mg_solve_levels(mg_level* Ls, int nlev, double tol, int maxit, int nu1, int nu2,
                           int gamma, int* cycles, double* res_hist)
{
    if (gamma < 1) gamma = 1;          /* cycle index 0 means the V-cycle, as in the C ABI */
    mg_level* L = &Ls[0];
    size_t n = (size_t)L->nx * L->nz;
    for (int l = 0; l < nlev; ++l) {
        if (l > 0) coarsen_operator(&Ls[l - 1], &Ls[l]);
        set_diag(&Ls[l]);
    }
    memset(L->dp, 0, sizeof(double) * n);
    double fn = inf_norm(L->f, n);
    double target = tol * (fn > 1.0 ? fn : 1.0);
    double rn = fn;
    int it = 0;
    if (res_hist) res_hist[0] = rn;
    while (rn >= target && it < maxit) {
        mgcycle(Ls, 0, nlev, nu1, nu2, gamma < 1 ? 1 : gamma);
        rn = residual(L);
        ++it;
        if (res_hist) res_hist[it] = rn;
        if (!isfinite(rn)) { *cycles = it; return 3; }
    }
    *cycles = it;
    if (!isfinite(rn)) return 3;
    return rn < target ? 0 : 1;
}

int orc_mg_solve(int32_t nx, int32_t nz, double h, const double* Tx, const double* Tz,
                 const double* Tbt, const double* Tbb, const double* Cdt, const double* f,
                 double tol, int32_t maxit, int32_t nu1, int32_t nu2, int32_t gamma, double* dp,
                 int32_t* cycles, double* res_hist)
{
    (void)h;
    int nlev = count_levels(nx, nz);
    if (nlev < 1) return -1;
    mg_level* Ls = alloc_levels(nx, nz, nlev);
    size_t n = (size_t)nx * nz;
    memcpy(Ls[0].Tx, Tx, n * 8); memcpy(Ls[0].Tz, Tz, n * 8); memcpy(Ls[0].Cdt, Cdt, n * 8);
    memcpy(Ls[0].Tbt, Tbt, nx * 8); memcpy(Ls[0].Tbb, Tbb, nx * 8); memcpy(Ls[0].f, f, n * 8);
    int cyc = 0;
    int rc = mg_solve_levels(Ls, nlev, tol, maxit, nu1, nu2, gamma, &cyc, res_hist);
    memcpy(dp, Ls[0].dp, n * 8);
    *cycles = cyc;
    free_levels(Ls, nlev);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Time loop with modified Picard (Sec. 4.1) and the bottom-flux QoI.         */
/* ------------------------------------------------------------------------- */
static int solve_soil(const orc_problem* pb, int32_t nx, int32_t nz, const orc_soil* so,
                      const double* src, const double* p_init, double* p_final, double* qoi,
                      orc_stats* st)
{
    int nlev = count_levels(nx, nz);
    if (nlev < 1 || nx < 1 || nz < 1) return -1;
    if (pb->closure != 0 && (pb->closure != 1 || !so->n)) return -1;
    const size_t n = (size_t)nx * nz;
    const double h = 1.0 / nz;
    mg_level* Ls = alloc_levels(nx, nz, nlev);
    mg_level* L = &Ls[0];
    double* p = (double*)malloc(n * 8);
    double* p_old = (double*)malloc(n * 8);
    /* initial head: given, uniform, or p_init (1 - exp(-init_decay z)) at the
     * cell centres z_j = (j + 1/2) h (Eq. travellingwave) */
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t q = (size_t)j * nx + i;
            if (p_init) p[q] = p_init[q];
            else if (pb->init_decay > 0.0) p[q] = pb->p_init * (1.0 - exp(-pb->init_decay * (j + 0.5) * h));
            else p[q] = pb->p_init;
        }
    int status = ORC_OK;
    orc_stats S = { 0, 0, 0, 0 };
    for (int step = 0; step < pb->nsteps && status != ORC_PICARD_MAXIT && status != ORC_NONFINITE; ++step) {
        memcpy(p_old, p, n * 8);                 /* p^{j+1,0} = p^j */
        int k = 0, converged = 0;
        while (!converged) {
            if (k >= pb->picard_maxit) { status = ORC_PICARD_MAXIT; break; }
            picard_system(pb, nx, nz, so, p, p_old, L->Tx, L->Tz, L->Tbt, L->Tbb, L->Cdt, L->f);
            if (src) for (size_t q = 0; q < n; ++q) L->f[q] += src[q];
            int cyc = 0;
            int rc = mg_solve_levels(Ls, nlev, pb->mg_tol, pb->mg_maxit, pb->nu1, pb->nu2, pb->gamma, &cyc,
                                     NULL);
            S.mg_cycles += cyc;
            if (cyc > S.max_mg) S.max_mg = cyc;
            if (rc == 3) { status = ORC_NONFINITE; break; }
            if (rc == 1 && status < ORC_MG_MAXIT) status = ORC_MG_MAXIT;
            for (size_t q = 0; q < n; ++q) p[q] += L->dp[q];   /* p^{k+1} = p^k + dp */
            ++k;
            double dn = inf_norm(L->dp, n);
            if (!isfinite(dn)) { status = ORC_NONFINITE; break; }
            converged = dn < pb->picard_tol;
        }
        S.picard_iters += k;
        if (k > S.max_picard) S.max_picard = k;
    }
    /* QoI: outward (downward) Darcy flux through the bottom faces, averaged
     * over the nx faces: q.n = K_b (2 (p_P - p_bot)/h + 1). */
    double Q = 0.0;
    for (int i = 0; i < nx; ++i) {
        cellp c = cell_at(pb, so, (size_t)i);
        double Kb = k_dirichlet(pb->closure, &c, pb->p_bottom);
        Q += Kb * (2.0 * (p[i] - pb->p_bottom) / h + 1.0);
    }
    Q /= nx;
    if (status == ORC_PICARD_MAXIT || status == ORC_NONFINITE) Q = NAN;
    if (qoi) *qoi = Q;
    if (p_final) memcpy(p_final, p, n * 8);
    if (st) *st = S;
    free(p); free(p_old);
    free_levels(Ls, nlev);
    return status;
}

int orc_solve_one_soil(const orc_problem* pb, int32_t nx, int32_t nz, const orc_soil* so,
                       const double* src, const double* p_init, double* p_final, double* qoi,
                       orc_stats* st)
{
    return solve_soil(pb, nx, nz, so, src, p_init, p_final, qoi, st);
}

int orc_solve_one(const orc_problem* pb, int32_t nx, int32_t nz, const double* lnKs,
                  const double* alpha, double alpha_scale, const double* src,
                  const double* p_init, double* p_final, double* qoi, orc_stats* st)
{
    if (pb->closure != 0) return -1;
    orc_soil so = { lnKs, alpha, NULL, NULL, NULL, alpha_scale, 0.0, 0.0 };
    return solve_soil(pb, nx, nz, &so, src, p_init, p_final, qoi, st);
}

typedef struct {
    const orc_problem* pb; int32_t nx, nz, ns; const orc_soil* so;
    double *p_final, *qoi; int32_t* status; orc_stats st; int32_t nthreads, tid;
} orc_solve_job;

static void* solve_worker(void* arg)
{
    orc_solve_job* J = (orc_solve_job*)arg;
    size_t n = (size_t)J->nx * J->nz;
    orc_stats acc = { 0, 0, 0, 0 };
    for (int s = J->tid; s < J->ns; s += J->nthreads) {
        const orc_soil* B = J->so;
        size_t o = (size_t)s * n;
        orc_soil so = { B->lnKs + o, B->alpha + o, B->n ? B->n + o : NULL,
                        B->theta_s ? B->theta_s + o : NULL, B->theta_r ? B->theta_r + o : NULL,
                        B->alpha_scale, B->alpha_shift, B->n_shift };
        orc_stats st;
        int rc = solve_soil(J->pb, J->nx, J->nz, &so, NULL, NULL, J->p_final ? J->p_final + o : NULL,
                            &J->qoi[s], &st);
        J->status[s] = rc;
        acc.picard_iters += st.picard_iters; acc.mg_cycles += st.mg_cycles;
        if (st.max_picard > acc.max_picard) acc.max_picard = st.max_picard;
        if (st.max_mg > acc.max_mg) acc.max_mg = st.max_mg;
    }
    J->st = acc;
    return NULL;
}

int orc_solve_batch_soil(const orc_problem* pb, int32_t nx, int32_t nz, int32_t nsamples,
                         const orc_soil* soil, double* p_final, double* qoi, int32_t* status,
                         orc_stats* st, int32_t nthreads)
{
    if (count_levels(nx, nz) < 1 || nsamples < 0) return -1;
    if (pb->closure != 0 && (pb->closure != 1 || !soil->n)) return -1;
    if (nthreads < 1) nthreads = 1;
    orc_solve_job* jobs = (orc_solve_job*)malloc(sizeof(orc_solve_job) * nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        orc_solve_job J = { pb, nx, nz, nsamples, soil, p_final, qoi, status, { 0, 0, 0, 0 }, nthreads, t };
        jobs[t] = J;
        pthread_create(&th[t], NULL, solve_worker, &jobs[t]);
    }
    orc_stats acc = { 0, 0, 0, 0 };
    int worst = 0;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        acc.picard_iters += jobs[t].st.picard_iters; acc.mg_cycles += jobs[t].st.mg_cycles;
        if (jobs[t].st.max_picard > acc.max_picard) acc.max_picard = jobs[t].st.max_picard;
        if (jobs[t].st.max_mg > acc.max_mg) acc.max_mg = jobs[t].st.max_mg;
    }
    for (int s = 0; s < nsamples; ++s) if (status[s] > worst) worst = status[s];
    if (st) *st = acc;
    free(jobs); free(th);
    return worst;
}

int orc_solve_batch(const orc_problem* pb, int32_t nx, int32_t nz, int32_t nsamples,
                    const double* lnKs, const double* alpha, double alpha_scale,
                    double* p_final, double* qoi, int32_t* status, orc_stats* st,
                    int32_t nthreads)
{
    if (pb->closure != 0) return -1;
    orc_soil so = { lnKs, alpha, NULL, NULL, NULL, alpha_scale, 0.0, 0.0 };
    return orc_solve_batch_soil(pb, nx, nz, nsamples, &so, p_final, qoi, status, st, nthreads);
}
