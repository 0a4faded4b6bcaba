// Internal declarations of librichards (CUDA path).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include "../../include/richards.h"
#include <vector>

#define RICH_MAX_LEVELS 16

#define RICH_CUDA(call)                                                     \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) { rich_set_error(cudaGetErrorString(e_), __FILE__, __LINE__); \
                                 return RICH_ERR_CUDA; }                    \
    } while (0)

void rich_set_error(const char* msg, const char* file, int line);

// The more severe of two per-sample statuses: NONFINITE, then PICARD_MAXIT
// (the sample failed, its QoI is NaN), then ADJ_MAXIT (an adjoint J^T solve
// hit its cap: the gradient is not to tolerance), then MG_MAXIT (a multigrid
// solve hit its cycle cap but the sample's result is usable), then OK.
inline int rich_status_worse(int a, int b) {
    auto rank = [](int s) {
        return s == RICH_NONFINITE ? 4 : s == RICH_PICARD_MAXIT ? 3 : s == RICH_ADJ_MAXIT ? 2 : s == RICH_MG_MAXIT ? 1 : 0;
    };
    return rank(b) > rank(a) ? b : a;
}

// per-sample status and counters of the last fused solve
struct rich_samplebuf {
    void* base = nullptr;
    int cap = 0;
    int32_t *status = nullptr, *maxpic = nullptr;
    int64_t *pic_total = nullptr, *mg_total = nullptr;
    int64_t* t_ns = nullptr;                    // per-sample solve time on its CTA
    int last = 0;                               // samples of the last fused solve
    int last_occ = 1;                           // resident CTAs per SM of the last fused launch
};

// sqrt of the circulant covariance spectrum on one torus (+ FFT twiddles)
struct rich_spectrum {
    int px = 0, pz = 0;
    double h = 0, sigma2 = 0, corr_len = 0, corr_len_z = 0, nu = 0, min_ratio = 0;
    double* sq = nullptr;                       // [pz][px]
    void* tw = nullptr;                         // twiddles of both line lengths
};

// Live timing of the finest-level smoothing launches (the dominant kernel):
// CUDA events around each launch on the launching stream, harvested whenever
// the host synchronises that stream anyway.
struct rich_prof {
    int enabled = 0;
    std::vector<cudaEvent_t> ev;                   // 2 per pending launch
    std::vector<double> pend_bytes, pend_flops;
    size_t used = 0;
    double ms = 0, bytes = 0, flops = 0;
    int64_t launches = 0;
};

struct rich_ctx {
    int device = 0;
    int sm_count = 0;
    rich_samplebuf sb;
    std::vector<rich_spectrum> spectra;         // cached FFT-MA filters
    void* field_work = nullptr;                 // complex work buffer of the field sampler
    size_t field_work_bytes = 0;
    rich_prof prof;
    void* fused_scratch = nullptr;              // per-CTA slots of the fused solver
    size_t fused_bytes = 0;
    void* stage = nullptr;                      // device staging of the host-buffer entry point
    size_t stage_bytes = 0;
    int tune_threads = 0;                       // fused-kernel block size (0: default 512)
    int tune_mixed_inner = 0;                   // FP32 V-cycles per FP64 defect (0: default 2)
    double last_sm_seconds = 0;                 // SM-seconds of the last rich_solve_device
    int adj_method = 1;                         // adjoint J^T solver: 0 defect correction, 1 BiCGStab
    double adj_tol = 1e-11;                     // J^T solves: relative residual target ...
    int adj_cap = 400;                          // ... and cap on preconditioner applications
};

void rich_count_launch();
int rich_prof_begin(rich_ctx* ctx, cudaStream_t st);
int rich_prof_end(rich_ctx* ctx, cudaStream_t st, double bytes, double flops);
int rich_prof_harvest(rich_ctx* ctx);

// ---- solver (solver.cu)
int rich_samples_reserve(rich_ctx* ctx, int S);
int rich_stage_reserve(rich_ctx* ctx, size_t bytes);
// per-cell fields beyond ln Ks and alpha (van Genuchten-Mualem closure) and
// the additive continuation shifts of alpha and n
struct rich_soil_in {
    const double* n = nullptr;
    const double* theta_s = nullptr;
    const double* theta_r = nullptr;
    double alpha_shift = 0.0, n_shift = 0.0;
};
int rich_solve_device(rich_ctx* ctx, const rich_problem_t* pb, int S, const double* lnKs,
                      const double* alpha, double alpha_scale, double* qoi, double* p_final,
                      int32_t* status, rich_stats_t* stats, cudaStream_t st,
                      const rich_soil_in* soil = nullptr);
int rich_count_levels(int nx, int nz);
int rich_sm_seconds(rich_ctx* ctx, int S, cudaStream_t st, double* out);
int rich_solve_fused(rich_ctx* ctx, const rich_problem_t* pb, int S, const double* lnKs,
                     const double* alpha, double alpha_scale, double* qoi, double* p_final,
                     int32_t* status, cudaStream_t st, const rich_soil_in* soil = nullptr);
void rich_prof_amend(rich_ctx* ctx, double bytes, double flops);
int rich_adjoint_fused(rich_ctx* ctx, const rich_problem_t* pb, int S, const double* lnKs,
                       const double* alpha, double alpha_scale, int ckpt_every, double adj_tol,
                       int adj_maxit, int adj_method, double* qoi, double* g_out, cudaStream_t st);
int rich_check_problem(const rich_problem_t* pb);

// ---- fields (fields.cu)
bool bad_field(const rich_field_t* fd);
int rich_fields_pair_device(rich_ctx* ctx, const rich_field_t* fd, int nx, int nz, uint32_t level,
                            int64_t first, int S, double* lk_f, double* al_f, double* lk_c,
                            double* al_c, cudaStream_t st);
int rich_fields_average(rich_ctx* ctx, int S, int nx, int nz, const double* lk, const double* al,
                        double* lkc, double* alc, cudaStream_t st);
int rich_soil_device(rich_ctx* ctx, const rich_field_t* fd, const rich_soil_model_t* sm, int nx, int nz,
                     uint32_t level, int64_t first, int S, int coarsen, const rich_soil_t* out,
                     cudaStream_t st);
int rich_soil_pair_device(rich_ctx* ctx, const rich_field_t* fd, const rich_soil_model_t* sm, int nx, int nz,
                          uint32_t level, int64_t first, int S, const rich_soil_t* fine,
                          const rich_soil_t* coarse, cudaStream_t st);
int rich_fields_device(rich_ctx* ctx, const rich_field_t* fd, int nx, int nz, uint32_t level,
                       int64_t first, int S, int coarsen, double* lnKs, double* alpha,
                       cudaStream_t st, const int64_t* first_dev = nullptr);
