/*
 * Plain FP64 CPU oracle for the stochastic Richards' equation solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Method (Kumar, Rodrigo, Gaspar, Oosterlee, arXiv 1903.08741):
 *   - mixed form of Richards' equation, backward Euler (Sec. 4.1, Eq. Mixed_based)
 *   - modified Picard iteration of Celia et al. (Sec. 4.1, Eqs. taylorThetap,
 *     Mixed_based_2, Mixed_based_3; stop on ||dp||_inf < eps_PI)
 *   - cell-centred FV with harmonic-mean faces (Sec. 4.2, Eqs. Grid_fine,
 *     five_stencil)
 *   - cell-centred multigrid: piecewise-constant prolongation, 1/4-sum
 *     restriction (Eq. transfer), coarse operator by rediscretisation with
 *     arithmetic means of fine face coefficients (Fig. diffUpscale), stop on
 *     ||L dp - f||_inf < eps_MG (Sec. 4.2)
 *   - FFT moving-average Gaussian fields (Appendix A, Eqs. convol1-product2)
 *   - closures: Gardner exponential model (the configured instance), with the
 *     saturated branch for p >= 0 as in Eqs. Sw, Krw; van Genuchten-Mualem
 *     (Sec. 2.1, Eqs. Sw, sc_van, Krw) with per-cell Ks, alpha, n, theta_s,
 *     theta_r fields (Table soilparams).
 */
#ifndef RICHARDS_ORACLE_H
#define RICHARDS_ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t nsteps;        /* implicit-Euler steps                          */
    double dt;             /* time step                                     */
    double theta_r, theta_s;
    double p_top, p_bottom;/* Dirichlet heads on z = top and z = 0           */
    double p_init;         /* uniform initial head (if no array is given)    */
    double picard_tol;     /* eps_PI on ||dp||_inf                           */
    int32_t picard_maxit;  /* failure if exceeded in a step (Sec. 4.3)       */
    double mg_tol;         /* eps_MG; applied as eps_MG * max(1, ||f||_inf)  */
    int32_t mg_maxit;
    int32_t nu1, nu2;      /* pre/post red-black GS steps                    */
    int32_t gamma;         /* cycle index: 1 = V-cycle, 2 = W-cycle          */
    int32_t closure;       /* 0 Gardner exponential, 1 van Genuchten-Mualem  */
    double init_decay;     /* > 0: p(x,z,0) = p_init (1 - exp(-init_decay z))
                              (the infiltration problem, Eq. travellingwave) */
} orc_problem;

/* Per-cell soil parameters of a batch, each [S][nz][nx].  n, theta_s and
 * theta_r are read by the van Genuchten-Mualem closure only (theta arrays may
 * be NULL: the problem's constants).  Effective parameters:
 * Ks = exp(lnKs), alpha_eff = alpha * alpha_scale + alpha_shift,
 * n_eff = n + n_shift (the parametric continuation of Sec. 5). */
typedef struct {
    const double *lnKs, *alpha, *n, *theta_s, *theta_r;
    double alpha_scale, alpha_shift, n_shift;
} orc_soil;

/* Marginals of the five soil fields (Table soilparams): ln Ks = lnks_mean + Z,
 * every other field lo + span * Phi(g) with g a unit-variance field of the
 * same covariance (Y = F_Y^-1(F_Z(Z)) for a uniform marginal, Sec. 3.1). */
typedef struct {
    double lnks_mean;
    double alpha_lo, alpha_span, n_lo, n_span;
    double theta_s_lo, theta_s_span, theta_r_lo, theta_r_span;
} orc_soil_model;

typedef struct {
    int64_t picard_iters;  /* total Picard iterations over all steps        */
    int64_t mg_cycles;     /* total V-cycles over all steps                 */
    int32_t max_picard;    /* largest Picard count in one step              */
    int32_t max_mg;        /* largest V-cycle count in one Picard iteration */
} orc_stats;

/* covariance of the Gaussian fields: nu = 0 exponential sigma2 exp(-r/corr_len);
 * nu > 0 Matern (Eq. nonIsotropic) with correlation lengths corr_len (x) and
 * corr_len_z (z; <= 0: same as x) */
typedef struct { double sigma2, corr_len, corr_len_z, nu; } orc_cov;

enum { ORC_OK = 0, ORC_PICARD_MAXIT = 1, ORC_MG_MAXIT = 2, ORC_NONFINITE = 3 };

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_white_noise(uint64_t seed, uint32_t level, uint64_t sample, uint32_t field,
                     int64_t npts, double* y);
int  orc_fft2(double* re, double* im, int32_t nx, int32_t nz, int32_t inverse);
double orc_bessel_k(double nu, double x);
double orc_covariance(const orc_cov* cv, double dx, double dz);
int  orc_fftma_spectrum(int32_t px, int32_t pz, double h, const orc_cov* cv,
                        double* sqrt_lambda, double* min_ratio);
int  orc_torus_size(int32_t nx, int32_t nz, double h, const orc_cov* cv, int32_t* px, int32_t* pz);
int  orc_sample_fields(uint64_t seed, const orc_cov* cv, double alpha_lo,
                       double alpha_span, int32_t nx, int32_t nz, uint32_t level,
                       int64_t first_sample, int32_t nsamples, int32_t coarsen_times,
                       double* lnKs, double* alpha, int32_t nthreads);
int  orc_sample_fields_pair(uint64_t seed, const orc_cov* cv, double alpha_lo,
                            double alpha_span, int32_t nx, int32_t nz, uint32_t level,
                            int64_t first_sample, int32_t nsamples, double* lnKs_f, double* alpha_f,
                            double* lnKs_c, double* alpha_c);
int  orc_sample_soil(uint64_t seed, const orc_cov* cv, const orc_soil_model* sm, int32_t nx, int32_t nz,
                     uint32_t level, int64_t first_sample, int32_t nsamples, int32_t coarsen_times,
                     double* lnKs, double* alpha, double* n, double* theta_s, double* theta_r,
                     int32_t nthreads);
int  orc_sample_soil_pair(uint64_t seed, const orc_cov* cv, const orc_soil_model* sm, int32_t nx, int32_t nz,
                          uint32_t level, int64_t first_sample, int32_t nsamples, double** fine,
                          double** coarse);
int  orc_closure(int32_t kind, double Ks, double a, double n, double theta_r, double theta_s,
                 double p, double* K, double* theta, double* C);
int  orc_solve_one_soil(const orc_problem* pb, int32_t nx, int32_t nz, const orc_soil* soil,
                        const double* src, const double* p_init, double* p_final, double* qoi,
                        orc_stats* st);
int  orc_solve_batch_soil(const orc_problem* pb, int32_t nx, int32_t nz, int32_t nsamples,
                          const orc_soil* soil, double* p_final, double* qoi, int32_t* status,
                          orc_stats* st, int32_t nthreads);
int  orc_solve_one(const orc_problem* pb, int32_t nx, int32_t nz, const double* lnKs,
                   const double* alpha, double alpha_scale, const double* src,
                   const double* p_init, double* p_final, double* qoi, orc_stats* st);
int  orc_solve_batch(const orc_problem* pb, int32_t nx, int32_t nz, int32_t nsamples,
                     const double* lnKs, const double* alpha, double alpha_scale,
                     double* p_final, double* qoi, int32_t* status, orc_stats* st,
                     int32_t nthreads);
int  orc_picard_system(const orc_problem* pb, int32_t nx, int32_t nz, const double* lnKs,
                       const double* alpha, double alpha_scale, const double* p,
                       const double* p_old, double* Tx, double* Tz, double* Tbt,
                       double* Tbb, double* Cdt, double* f);
int  orc_mg_solve(int32_t nx, int32_t nz, double h, const double* Tx, const double* Tz,
                  const double* Tbt, const double* Tbb, const double* Cdt, const double* f,
                  double tol, int32_t maxit, int32_t nu1, int32_t nu2, int32_t gamma, double* dp,
                  int32_t* cycles, double* res_hist);
#endif
