/*
 * librichards -- batched Monte Carlo solves of the stochastic Richards'
 * equation on one GB300 GPU (sm_103a), following
 *   P. Kumar, C. Rodrigo, F. J. Gaspar, C. W. Oosterlee, "A parametric
 *   acceleration of multilevel Monte Carlo convergence for nonlinear
 *   variably saturated flow", arXiv 1903.08741.
 *
 * C ABI: plain pointers and sizes only.  Unless stated otherwise every array
 * argument is DEVICE memory owned by the caller (the library never frees it),
 * laid out row-major [sample][nz][nx] with x fastest and row z = 0 at the
 * bottom of the unit-height domain; the mesh width is h = 1/nz (Eq. Grid_fine).
 *
 * Return codes: 0 = OK; < 0 = fatal error of the call (nothing is guaranteed
 * about the outputs); > 0 = the call completed and the value is the most
 * severe per-sample status, in the order RICH_NONFINITE, RICH_PICARD_MAXIT
 * (both: the sample failed, its QoI is NaN), RICH_ADJ_MAXIT (an adjoint J^T
 * solve stopped at its cap; QoI usable, gradient not to tolerance),
 * RICH_MG_MAXIT (a multigrid solve stopped at its cycle cap; the sample's
 * result is still usable), with the per-sample details in the status array.
 * A sample that fails after an earlier MG_MAXIT carries the failure status.  No C++ exception crosses the
 * ABI.  Streams are cudaStream_t passed as void* (NULL = legacy default).
 */
#ifndef RICHARDS_H
#define RICHARDS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RICH_OK = 0,
    RICH_PICARD_MAXIT = 1, /* a time step needed more Picard iterations than allowed (Sec. 4.3) */
    RICH_MG_MAXIT = 2,     /* an MG solve stopped at mg_maxit cycles above tolerance           */
    RICH_NONFINITE = 3,    /* NaN/Inf met in a residual or correction                          */
    RICH_ADJ_MAXIT = 4,    /* an adjoint J^T solve stopped at its cap above tolerance          */
    RICH_ERR_INVALID = -1, /* bad argument: sizes, pointers, unsupported grid                  */
    RICH_ERR_CUDA = -2,    /* a CUDA runtime call failed                                       */
    RICH_ERR_OOM = -3      /* device workspace could not be allocated                          */
};

enum { RICH_FP64 = 0, RICH_MIXED = 1 };
/* closures (rich_problem_t.closure) */
enum { RICH_GARDNER = 0, RICH_VAN_GENUCHTEN = 1 };

typedef struct rich_ctx* rich_ctx_t;

/* Physics and solver settings of one batch (Sec. 2: Gardner or van
 * Genuchten-Mualem closure; Picard, Sec. 4.1; CCMG, Sec. 4.2). */
typedef struct {
    int32_t nx, nz;          /* cells per side; must coarsen by 2 to <= 64 cells  */
    int32_t nsteps;          /* implicit-Euler steps (Eq. Mixed_based)            */
    double dt;
    double theta_r, theta_s; /* residual / saturated water content                */
    double p_top, p_bottom;  /* Dirichlet heads on the top and bottom faces       */
    double p_init;           /* uniform initial head                              */
    double picard_tol;       /* stop when ||dp||_inf < picard_tol (Sec. 4.1)      */
    int32_t picard_maxit;    /* failure beyond this many iterations in a step     */
    double mg_tol;           /* stop when ||f - A dp||_inf < mg_tol*max(1,||f||)  */
    int32_t mg_maxit;
    int32_t nu1, nu2;        /* red-black Gauss-Seidel steps before / after       */
    int32_t precision;       /* RICH_FP64, or RICH_MIXED: FP32 V-cycles inside an
                                FP64 defect-correction loop                       */
    int32_t cycle;           /* multigrid cycle index: 1 (or 0) V-cycle, 2 W-cycle
                                (the paper's W(2,2), Sec. 4.2), at most 4         */
    int32_t closure;         /* RICH_GARDNER (zero-initialised default) or
                                RICH_VAN_GENUCHTEN (Sec. 2.1, Eqs. Sw, sc_van,
                                Krw; needs per-cell n: rich_solve_soil)           */
    double init_decay;       /* 0: uniform p_init; > 0: initial head
                                p_init (1 - exp(-init_decay z)) at the cell
                                centres (the infiltration problem, Eq.
                                travellingwave: p_init -0.4, init_decay 80)       */
} rich_problem_t;

/* Random-field model: ln Ks Gaussian, drawn by FFT moving average (Appendix A,
 * Eqs. convol1-product2); alpha = alpha_lo + alpha_span * Phi(g) with g an
 * independent unit-variance field of the same correlation (the marginal
 * transform Y = F_Y^-1(F_Z(Z)) of Sec. 3.1).  Covariance at offset (dx, dz),
 * r = sqrt((dx/corr_len)^2 + (dz/corr_len_z)^2):
 *   nu = 0       sigma2 exp(-r)  (exponential; the zero-initialised default)
 *   0 < nu <= 16 the Matern function of Eq. nonIsotropic,
 *                sigma2 2^(1-nu)/Gamma(nu) (2 sqrt(nu) r)^nu K_nu(2 sqrt(nu) r);
 *                the paper's Phi_1 = (nu 1, 0.2, 0.2, 1), Phi_2 = (0.5, 0.1, 0.01, 1).
 * Invalid (RICH_ERR_INVALID): sigma2 <= 0, corr_len <= 0, corr_len_z < 0, nu
 * outside [0, 16]. */
typedef struct {
    double sigma2, corr_len;
    double alpha_lo, alpha_span;
    uint64_t seed;
    double nu;               /* Matern smoothness; 0 selects the exponential      */
    double corr_len_z;       /* correlation length along z; 0: equal to corr_len  */
} rich_field_t;

/* Host-side counters of a solve (summed over samples). */
typedef struct {
    int64_t picard_iters;    /* sum over samples and steps                        */
    int64_t mg_cycles;       /* sum over samples of V-cycles                      */
    int64_t cell_vcycles;    /* sum of V-cycles x fine cells                      */
    int32_t max_picard;      /* largest Picard count of one step of one sample    */
    int32_t failed;          /* samples with status PICARD_MAXIT or NONFINITE     */
    double seconds;          /* wall time of the call                             */
    double sm_seconds;       /* SM-seconds the solves held: sum over samples of the
                                sample's solve time on its CTA / the CTAs resident
                                per SM (the cost on a fully occupied GPU is
                                sm_seconds / the number of SMs)                   */
} rich_stats_t;

/* Create a context on CUDA device `device`.  The context owns its device
 * workspaces (grown on demand) and is not thread-safe. */
int rich_create(rich_ctx_t* out, int device);
void rich_destroy(rich_ctx_t ctx);
const char* rich_status_str(int code);
/* Text of the last fatal error seen by the calling thread (never NULL). */
const char* rich_last_error(void);

/* Launch tuning of this context's solves (set by the autotuner of the Python
 * package, which times the candidates and caches the choice per grid,
 * precision and batch): block_threads 32 (thirty-two resident CTAs per SM,
 * one warp per sample, every level in the sample's slot), 128 (eight), 256
 * (four), 512 (two) or 1024 (one), 0 = default 512; mixed_inner = FP32 V-cycles per FP64 defect in
 * RICH_MIXED solves, 0 = default 2 (1..16).  The computed solution does not
 * depend on block_threads; mixed_inner changes how often the FP64 stopping
 * test is evaluated (the FP64 tolerance holds either way). */
int rich_set_tuning(rich_ctx_t ctx, int32_t block_threads, int32_t mixed_inner);

/* Draw ln Ks and alpha for samples first_sample .. first_sample+nsamples-1 of
 * MLMC level `level` on an nx x nz grid, then average them over 2x2 blocks
 * coarsen_times times.  Outputs lnKs, alpha: device [nsamples][nz>>c][nx>>c].
 * White noise: Philox4x32-10 keyed by (seed, level), counter (cell pair,
 * field, sample) with Box-Muller; FFT-MA on the smallest power-of-two torus of
 * at least twice the grid whose circulant spectrum is non-negative
 * (Appendix A).  Asynchronous on `stream`.  nx, nz must be powers of two. */
int rich_sample_fields(rich_ctx_t ctx, const rich_field_t* field, int32_t nx, int32_t nz,
                       uint32_t level, int64_t first_sample, int32_t nsamples,
                       int32_t coarsen_times, double* lnKs, double* alpha, void* stream);

/* As rich_sample_fields, with the index of the first sample read from DEVICE
 * memory (*first_sample_dev) when the kernels run, so that a captured CUDA
 * graph can draw a new sample range on every replay.  The spectrum and the
 * work buffer of a grid are set up (with a host synchronisation) on its first
 * use; make one call outside the capture first. */
int rich_sample_fields_at(rich_ctx_t ctx, const rich_field_t* field, int32_t nx, int32_t nz,
                          uint32_t level, const int64_t* first_sample_dev, int32_t nsamples,
                          int32_t coarsen_times, double* lnKs, double* alpha, void* stream);

/* Coupled pair of fields by covariance upscaling (Appendix A, Eqs. averaging,
 * cov_upscale): the fine fields on nx x nz as rich_sample_fields draws them,
 * and the coarse fields on (nx/2) x (nz/2) from the SAME white noise averaged
 * over 2x2 torus blocks (scaled by 1/2, so it stays standard normal) and
 * filtered with the coarse grid's spectrum on the half-size torus.  Each member
 * is an exact sample of its own grid's field, so MLMC telescoping is exact.
 * Outputs (device): lnKs_f, alpha_f [S][nz][nx]; lnKs_c, alpha_c
 * [S][nz/2][nx/2].  Asynchronous on `stream`. */
int rich_sample_fields_pair(rich_ctx_t ctx, const rich_field_t* field, int32_t nx, int32_t nz,
                            uint32_t level, int64_t first_sample, int32_t nsamples,
                            double* lnKs_f, double* alpha_f, double* lnKs_c, double* alpha_c,
                            void* stream);

/* Solve nsamples independent problems (Sec. 4: backward Euler, modified
 * Picard, CCMG V(nu1,nu2) with red-black GS, harmonic-mean faces, piecewise-
 * constant transfers, rediscretised coarse operators).  Inputs lnKs, alpha
 * [S][nz][nx]; the nonlinearity used is alpha * alpha_scale (the parametric
 * continuation of Sec. 5).  Outputs: qoi[S] = mean outward Darcy flux through
 * the bottom faces at t = nsteps*dt (NaN for failed samples); p_final
 * [S][nz][nx] or NULL; status[S].  stats (HOST) may be NULL.  The call returns
 * once the batch is solved (the host reads convergence counters on `stream`). */
int rich_solve_batch(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                     const double* lnKs, const double* alpha, double alpha_scale,
                     double* qoi, double* p_final, int32_t* status, rich_stats_t* stats,
                     void* stream);

/* Enqueue-only form of rich_solve_batch: launches the fused solve on `stream`
 * and returns without waiting, reading back nothing (no stats, return value 0
 * or a negative error; per-sample results in status[]).  Stream-capturable
 * once a first call with the same grid, precision and a batch at least as
 * large has set up the device buffers. */
int rich_solve_batch_async(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                           const double* lnKs, const double* alpha, double alpha_scale,
                           double* qoi, double* p_final, int32_t* status, void* stream);

/* As rich_solve_batch, but lnKs, alpha, qoi, p_final and status are HOST
 * arrays: the library copies inputs to its workspace and results back (the
 * end-to-end path of a caller that holds no device memory). */
int rich_solve_batch_host(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                          const double* lnKs, const double* alpha, double alpha_scale,
                          double* qoi, double* p_final, int32_t* status, rich_stats_t* stats,
                          void* stream);

/* Per-cell soil fields of a batch, each [S][nz][nx] DEVICE memory owned by
 * the caller: outputs of rich_sample_soil, inputs of rich_solve_soil.  The
 * van Genuchten-Mualem closure reads ln Ks, alpha, n and (when non-NULL)
 * theta_s, theta_r (NULL: the problem's constants); Gardner reads ln Ks and
 * alpha only. */
typedef struct {
    double* lnKs;
    double* alpha;
    double* n;
    double* theta_s;
    double* theta_r;
} rich_soil_t;

/* Marginals of the five soil fields (Table soilparams): ln Ks = lnks_mean + Z
 * (Eq. RandK with Ks^(bl) = exp(lnks_mean)); alpha, n, theta_s, theta_r are
 * lo + span * Phi(g) with g a unit-variance field of the same covariance
 * (uniform marginals, Sec. 3.1).  The paper's table: alpha_bl +- 0.2,
 * n_bl +- 0.05, theta_s 0.5 +- 0.05, theta_r 0.05 +- 0.005, Ks_bl = 0.2. */
typedef struct {
    double lnks_mean;
    double n_lo, n_span;
    double theta_s_lo, theta_s_span;
    double theta_r_lo, theta_r_span;
} rich_soil_model_t;

/* The five soil fields of samples first_sample .. +nsamples-1 by FFT-MA
 * (Appendix A), with the covariance and the alpha marginal of `field` and
 * the other marginals of `soil`.  Field k of a sample uses the white-noise
 * stream k (0 ln Ks, 1 alpha, 2 n, 3 theta_s, 4 theta_r), so ln Ks and alpha
 * are the draws rich_sample_fields makes (ln Ks shifted by lnks_mean).
 * coarsen_times 2x2 averages as rich_sample_fields.  out->theta_s/theta_r may
 * be NULL (not drawn).  Asynchronous on `stream`. */
int rich_sample_soil(rich_ctx_t ctx, const rich_field_t* field, const rich_soil_model_t* soil,
                     int32_t nx, int32_t nz, uint32_t level, int64_t first_sample,
                     int32_t nsamples, int32_t coarsen_times, const rich_soil_t* out, void* stream);

/* The five soil fields as fine (nx x nz) / coarse (nx/2 x nz/2) couples by
 * covariance upscaling (Appendix A, Eqs. averaging, cov_upscale), as
 * rich_sample_fields_pair does for two: the fine members are the
 * rich_sample_soil draws; the theta outputs of both members may be NULL. */
int rich_sample_soil_pair(rich_ctx_t ctx, const rich_field_t* field, const rich_soil_model_t* soil,
                          int32_t nx, int32_t nz, uint32_t level, int64_t first_sample, int32_t nsamples,
                          const rich_soil_t* fine, const rich_soil_t* coarse, void* stream);

/* As rich_solve_batch with per-cell soil fields (either closure) and the
 * additive continuation of Sec. 5: alpha_eff = alpha * alpha_scale +
 * alpha_shift, n_eff = n + n_shift (the paper's (grad alpha, grad n)
 * hierarchy uses negative alpha shifts and positive n shifts on coarse
 * levels).  RICH_ERR_INVALID if the closure needs n and soil->n is NULL. */
int rich_solve_soil(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                    const rich_soil_t* soil, double alpha_scale, double alpha_shift, double n_shift,
                    double* qoi, double* p_final, int32_t* status, rich_stats_t* stats, void* stream);

/* Per-sample totals of the context's last solve (rich_solve_batch, _soil,
 * _async, _host): Picard iterations and multigrid cycles summed over the
 * time steps of each of the first nsamples samples (the cost measure of the
 * paper's Sec. 4.3 study), copied to DEVICE arrays (either may be NULL) on
 * `stream`, which must be ordered after that solve.  RICH_ERR_INVALID if
 * nsamples exceeds the last solve's batch. */
int rich_sample_counters(rich_ctx_t ctx, int32_t nsamples, int64_t* picard_iters, int64_t* mg_cycles,
                         void* stream);

/* Multilevel Monte Carlo with parametric continuation (Sec. 5, Eqs.
 * telescope_ch6, MLMCestimator_ch6, SMC_ch6, MC_var_ch6, ML_var_ch6,
 * eq:MLMCVar, MLMCSAMP_ch6).  Level l (0..L) pairs a fine solve on an
 * (n0 2^l)^2 grid with steps0 2^l time steps of dt_l = t_final/(steps0 2^l)
 * and nonlinearity alpha_l with a coarse solve on the level-(l-1) grid, time
 * step and nonlinearity, both from ONE seeded random draw (the coarse member
 * uses its 2x2 block means).  With continuation, alpha_l = alpha (l+1)/(L+1):
 * only the finest level carries the full alpha field. */
#define RICH_MLMC_MAX_LEVELS 8
typedef struct {
    rich_problem_t base;      /* physics and solver settings; nx, nz, nsteps, dt are set per level */
    rich_field_t field;
    int32_t nlevels;          /* L + 1, at most RICH_MLMC_MAX_LEVELS                      */
    int32_t n0;               /* cells per side on level 0                                */
    int32_t steps0;           /* time steps on level 0                                    */
    double t_final;
    int32_t nsamples[RICH_MLMC_MAX_LEVELS];  /* N_l                                       */
    int32_t coupling;         /* 0: draw on the finest grid and average ln Ks, alpha down
                                 (every level's fine member has the law of the next level's
                                 coarse member: exact telescoping, Eq. fine_coarse);
                                 1: draw on the pair's fine grid, coarse member = 2x2 means
                                 of ln Ks, alpha (cheap, not exact);
                                 2: covariance upscaling, rich_sample_fields_pair (exact,
                                 cheap; Appendix A)                                         */
    int32_t continuation;     /* Gardner: 1 gives alpha_l = alpha (l+1)/(L+1); van Genuchten:
                                 1 gives the additive (d_alpha, d_n) hierarchy below; 0: the
                                 original parameters on every level                       */
    int32_t batch;            /* pairs per launch; 0 = automatic: B = 2^31/(16 n_L^2) on
                                 the finest level (n_L its grid), B (n_L/n_l)^2 on level l  */
    double eps;               /* RMSE target of the optimal-allocation report              */
    uint32_t key_offset;      /* added to the level in the noise key (independent reruns)  */
    int32_t tune_threads[RICH_MLMC_MAX_LEVELS];  /* per-level launch shape (0: context's)    */
    int32_t tune_inner[RICH_MLMC_MAX_LEVELS];    /* per-level FP32 cycles per defect (0: ctx) */
    /* van Genuchten-Mualem levels (base.closure == RICH_VAN_GENUCHTEN): the
     * five soil fields of `soil` (alpha's range is field.alpha_lo/span) and
     * the additive continuation of Sec. 5.2: with k_l = max(0, L + 1 -
     * fixed_levels - l), level l solves with alpha - k_l d_alpha and
     * n + k_l d_n, so the fixed_levels finest levels (at least 1) keep the
     * original parameters; continuation = 0 gives k_l = 0.  Theta fields are
     * drawn when with_thetas is 1 (else the base problem's constants). */
    rich_soil_model_t soil;
    double d_alpha, d_n;
    int32_t fixed_levels;
    int32_t with_thetas;
    /* Grid-only bias estimate (Eq. discErr): after the levels, bias_pairs
     * extra pairs of the finest level whose two members both use the original
     * parameters (alpha scale 1, no additive shift), from their own noise
     * stream; 0 = none.  With continuation the finest level's Y_L also holds
     * the parameter jump, so |E Y_L| alone does not measure the grid bias. */
    int32_t bias_pairs;
} rich_mlmc_cfg_t;

typedef struct {
    int32_t nlevels;
    int64_t n[RICH_MLMC_MAX_LEVELS], failed[RICH_MLMC_MAX_LEVELS];
    double mean[RICH_MLMC_MAX_LEVELS], var[RICH_MLMC_MAX_LEVELS];      /* Y_l = Q_l - Q_{l-1} */
    double mean_f[RICH_MLMC_MAX_LEVELS], var_f[RICH_MLMC_MAX_LEVELS];  /* Q_l (fine member)   */
    double mean_c[RICH_MLMC_MAX_LEVELS], var_c[RICH_MLMC_MAX_LEVELS];  /* Q_{l-1} (coarse)    */
    double cost[RICH_MLMC_MAX_LEVELS];        /* GPU seconds per pair (fields + both solves) */
    double cost_fine[RICH_MLMC_MAX_LEVELS];   /* seconds per single fine solve (fields + solve) */
    double n_opt[RICH_MLMC_MAX_LEVELS];       /* Eq. MLMCSAMP_ch6 for eps                 */
    double estimate;          /* sum of level means (Eq. MLMCestimator_ch6)              */
    double rmse;              /* sqrt(sum V_l / N_l) (Eq. eq:MLMCVar)                    */
    double ml_variance;       /* sum V[Q_l] - V[Q_{l-1}] (Eq. ML_var_ch6)                */
    double w_eps;             /* eps^-2 (sum sqrt(V_l C_l))^2: seconds to RMSE eps        */
    double w_mc_eps;          /* plain MC at the finest level: V[Q_L] C_L,fine / eps^2   */
    double bias_estimate;     /* |E Y_L| / (2^1 - 1) (Eq. discErr); with continuation it
                                 mixes the grid bias with the finest parameter jump        */
    double seconds;           /* wall time of the call                                   */
    int32_t rounds;           /* sampling rounds (1 for rich_mlmc_estimate)              */
    int64_t bias_pairs;       /* usable grid-only bias pairs (0: none requested)          */
    double bias_grid;         /* |E[Q_L - Q_{L-1}]| / (2^1 - 1), both at the original
                                 parameters (Eq. discErr, rate a = 1); NaN without pairs  */
    double bias_grid_se;      /* standard error of E[Q_L - Q_{L-1}]                       */
    double total_rmse;        /* sqrt(bias_grid^2 + sum V_l/N_l) (Eq. MSEMLMC_ch6)        */
    int32_t levels_for_eps;   /* levels for which the grid bias (halving per level) falls
                                 to eps/sqrt(2); 0 without bias pairs                      */
    double cost_sm[RICH_MLMC_MAX_LEVELS];  /* GPU-seconds per pair on a fully occupied GPU:
                                 field time + the solves' SM-seconds (rich_stats_t
                                 sm_seconds) / the number of SMs, per pair; equals cost[]
                                 when a level's batches fill the GPU                       */
    double w_eps_sm;          /* eps^-2 (sum sqrt(V_l cost_sm_l))^2                        */
} rich_mlmc_result_t;

/* Run the estimator with the configured N_l and fill *out (HOST).  Synchronous;
 * device memory is allocated and freed inside the call. */
int rich_mlmc_estimate(rich_ctx_t ctx, const rich_mlmc_cfg_t* cfg, rich_mlmc_result_t* out);

/* Algorithm PC_MLMC of Sec. 5.2: warm-up with N*_l = cfg->nsamples, then
 * repeatedly set N_l to the optimal allocation (Eq. MLMCSAMP_ch6) for RMSE
 * cfg->eps from the current level variances and the per-sample costs measured
 * so far, and draw the missing samples (continuing each level's sample
 * stream), until no level needs more, max_rounds rounds are done, or a level
 * would exceed nmax[l] (HOST array, may be NULL).  N_l counts the pairs with
 * a defined QoI, whose variance the RMSE uses (a failed pair is replaced by
 * further draws); nmax[l] caps the pairs run.  cfg->eps must be > 0. */
int rich_mlmc_adaptive(rich_ctx_t ctx, const rich_mlmc_cfg_t* cfg, int32_t max_rounds,
                       const int64_t* nmax, rich_mlmc_result_t* out);

/* MC / MLMC level accumulation in FP64 on the device (Sec. 5, Eqs. SMC_ch6,
 * MC_var_ch6, ML_var_ch6): for i < n with Y_i = qoi_fine[i] - qoi_coarse[i]
 * (qoi_coarse NULL: Y_i = qoi_fine[i], the plain MC or level-0 term), adds to
 * the DEVICE array acc[8]:
 *   acc[0] += sum Y, acc[1] += sum Y^2, acc[2] += count, acc[3] += failed,
 *   acc[4] += sum Qf, acc[5] += sum Qf^2, acc[6] += sum Qc, acc[7] += sum Qc^2.
 * A sample is failed (counted, excluded from the sums) when either status is
 * RICH_PICARD_MAXIT or RICH_NONFINITE or a QoI is not finite; statuses may be
 * NULL.  Deterministic summation order.  Asynchronous on `stream`.  Plain
 * sums (ranks merge them by adding); the variance (S2 - S1^2/n)/(n - 1)
 * loses digits when |mean| >> std, so for such data subtract a shift from
 * the QoIs first (rich_mlmc_estimate does this internally per level). */
int rich_mlmc_accumulate(rich_ctx_t ctx, const double* qoi_fine, const double* qoi_coarse,
                         const int32_t* status_fine, const int32_t* status_coarse, int32_t n,
                         double* acc, void* stream);

/* ln Ks fields of a Karhunen-Loeve expansion (Sec. 3, Eq. KLexp_ch6):
 * lnKs[s][c] = sum_j xi[s][j] kl_basis[j][c], with sqrt(lambda_j) folded into the
 * basis.  kl_basis [n_kl][ncell], xi [S][n_kl], lnKs [S][ncell]: device arrays.
 * S <= 65535.  Asynchronous on `stream`. */
int rich_kl_fields(rich_ctx_t ctx, const double* kl_basis, int32_t n_kl, int32_t ncell,
                   const double* xi, int32_t nsamples, double* lnKs, void* stream);

/* Discrete adjoint: the QoI of rich_solve_batch for ln Ks = KL(xi) and its
 * gradient with respect to the KL coefficients, dq_dxi [S][n_kl], by the
 * adjoint of the converged time-stepped Picard/CCMG solve (configured
 * instance; the paper has no adjoint): with R_n(p^n, p^{n-1}, m) = 0 the states
 * of backward Euler and m = ln Ks,
 *   J_N^T lam_N = dQ/dp^N,  J_n^T lam_n = diag(C(p^n)/dt) lam_{n+1},
 *   dQ/dm = dQ/dm|explicit - sum_n (dR_n/dm)^T lam_n,  dQ/dxi_j = <basis_j, dQ/dm>,
 * J_n the full Newton Jacobian (K'(p) inside the harmonic means included).
 * J^T systems are solved by BiCGStab (or defect correction, see
 * rich_set_adjoint_method) preconditioned with CCMG V-cycles of the Picard
 * operator (FP32 V-cycles when pb->precision is RICH_MIXED) to a relative
 * residual of 1e-11.  Memory: the states are checkpointed every
 * ckpt_every steps and each segment is recomputed during the reverse sweep.
 * dq_dlnKs [S][nz][nx] (device) may be NULL.  A J^T solve that stops at its
 * iteration limit sets RICH_MG_MAXIT.  Synchronous (returns when done). */
int rich_solve_batch_adjoint(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                             const double* kl_basis, int32_t n_kl, const double* xi,
                             const double* alpha, double alpha_scale, int32_t ckpt_every,
                             double* qoi, double* dq_dxi, double* dq_dlnKs, int32_t* status,
                             rich_stats_t* stats, void* stream);

/* Solver of the adjoint's J^T systems in this context's rich_solve_batch_adjoint
 * calls: 1 (default) BiCGStab (van der Vorst 1992) right-preconditioned with
 * the CCMG cycles of the Picard operator, stopped on the true residual; 2
 * restarted GMRES(12) (Saad & Schultz 1986) with the same preconditioner,
 * stopped on the true residual; 0 the plain defect correction
 * lam += M^{-1}(rhs - J^T lam).  All stop at the limits of
 * rich_set_adjoint_limits (default: relative residual 1e-11, 400
 * preconditioner applications, then RICH_ADJ_MAXIT);
 * rich_stats_t.mg_cycles counts the applications.  RICH_ERR_INVALID otherwise. */
int rich_set_adjoint_method(rich_ctx_t ctx, int32_t method);

/* Stopping rule of this context's adjoint J^T solves (any method): converged
 * when ||rhs - J^T lam||_inf <= rel_tol ||rhs||_inf, given up after
 * max_applications preconditioner applications (defect correction: outer
 * iterations), which sets RICH_ADJ_MAXIT for the sample (its QoI and its
 * not fully converged gradient are still returned).  Defaults 1e-11 and 400.
 * RICH_ERR_INVALID unless 0 < rel_tol < 1 and 1 <= max_applications <= 1e6. */
int rich_set_adjoint_limits(rich_ctx_t ctx, double rel_tol, int32_t max_applications);

/* Allocation-free solve.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc -- code embedded in a host framework
 * that owns all device memory through its own pool allocator and forbids other
 * allocations, or latency-sensitive loops that cannot afford cudaMalloc's
 * implicit device synchronisation.  It runs the fused FP64 / mixed solver of
 * rich_solve_batch on the CURRENT device with no context and allocates nothing
 * (no cudaMalloc, cudaFree or allocating library call): its scratch is a
 * library-owned static device array of RICH_NOALLOC_SCRATCH_BYTES (16 MiB),
 * present on every GPU that loads the library until the process exits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, once per device, under a lock) with that device
 *     current, and keeps it; make that first call before any stream capture.
 *     The address dies with the device's context: do not call this entry
 *     point again after cudaDeviceReset on that device.
 *   - Every call shares the one array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and give wrong results; order
 *     them on one stream.  Each call clears the state that must start at zero.
 *   - The grid is limited to the CTA slots that fit in the array; a grid whose
 *     per-CTA slot exceeds it is rejected with RICH_ERR_INVALID.  A slot holds
 *     one sample's multigrid hierarchy and fine-grid state: a 128^2 FP64
 *     problem needs 2.88 MiB per CTA, so 5 CTAs run (mixed precision: 2.18 MiB,
 *     7 CTAs); 32^2 FP64 needs 0.19 MiB (86 slots).
 * Inputs lnKs, alpha [S][nz][nx] and outputs qoi[S], status[S] (status may be
 * NULL) are caller-owned DEVICE arrays.  The call is asynchronous on `stream`
 * and returns 0 once the work is enqueued (per-sample results are in status),
 * or a negative error code. */
#define RICH_NOALLOC_SCRATCH_BYTES (16u << 20)
int rich_solve_batch_noalloc(const rich_problem_t* pb, int32_t nsamples, const double* lnKs,
                             const double* alpha, double alpha_scale, double* qoi,
                             int32_t* status, void* stream);

/* Measurement hooks.  rich_profile(ctx, 1) starts recording CUDA events around
 * every finest-level smoothing launch (the dominant kernel) on its stream and
 * resets the totals; rich_profile_read returns the summed event time (ms), the
 * number of launches and their algorithmic bytes and FLOPs.  rich_launch_count
 * returns the number of kernels this library has launched in the process. */
int rich_profile(rich_ctx_t ctx, int enable);
int rich_profile_read(rich_ctx_t ctx, double* ms, int64_t* launches, double* alg_bytes,
                      double* alg_flops);
int64_t rich_launch_count(void);

/* FP64 arithmetic rates of the context's GPU, measured by microbenchmark
 * kernels (independent FP64 chains on every SM, 256-thread CTAs, 8 per SM;
 * one warm-up and one CUDA-event-timed launch each): FMA (counted as 2 FLOP),
 * division and exp.  The fused FP64 solver is bound by the FP64 pipe, and
 * dfma_flops is its roofline denominator.  Synchronous (a private stream);
 * about a second of GPU time. */
typedef struct {
    double dfma_flops;        /* FP64 FLOP/s from FMA chains                      */
    double div_per_s;         /* FP64 divisions per second                        */
    double exp_per_s;         /* FP64 exp evaluations per second                  */
    double ms_total;          /* timed milliseconds of the three kernels          */
} rich_fp64_rates_t;
int rich_measure_fp64(rich_ctx_t ctx, rich_fp64_rates_t* out);

#ifdef __cplusplus
}
#endif
#endif
