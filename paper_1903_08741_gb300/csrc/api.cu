// C-ABI entry points of librichards (declared in include/richards.h).
#include "rich_internal.cuh"
#include <cmath>
#include <stdio.h>
#include <string.h>
#include <new>
#include <algorithm>

#include <atomic>

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

void rich_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" int64_t rich_launch_count(void) { return g_launches.load(); }

int rich_prof_begin(rich_ctx* ctx, cudaStream_t st) {
    rich_prof& P = ctx->prof;
    if (!P.enabled) return 0;
    if (P.ev.size() < 2 * (P.used + 1)) {
        size_t old = P.ev.size();
        P.ev.resize(std::max<size_t>(64, 2 * old));
        for (size_t k = old; k < P.ev.size(); ++k) RICH_CUDA(cudaEventCreate(&P.ev[k]));
        P.pend_bytes.resize(P.ev.size() / 2);
        P.pend_flops.resize(P.ev.size() / 2);
    }
    RICH_CUDA(cudaEventRecord(P.ev[2 * P.used], st));
    return 0;
}

int rich_prof_end(rich_ctx* ctx, cudaStream_t st, double bytes, double flops) {
    rich_prof& P = ctx->prof;
    if (!P.enabled) return 0;
    RICH_CUDA(cudaEventRecord(P.ev[2 * P.used + 1], st));
    P.pend_bytes[P.used] = bytes;
    P.pend_flops[P.used] = flops;
    ++P.used;
    return 0;
}

// set the algorithmic work of the most recently recorded launch
void rich_prof_amend(rich_ctx* ctx, double bytes, double flops) {
    rich_prof& P = ctx->prof;
    if (!P.enabled || P.used == 0) return;
    P.pend_bytes[P.used - 1] = bytes;
    P.pend_flops[P.used - 1] = flops;
}

// all recorded events have completed (the caller synchronised their stream)
int rich_prof_harvest(rich_ctx* ctx) {
    rich_prof& P = ctx->prof;
    for (size_t k = 0; k < P.used; ++k) {
        float ms = 0;
        RICH_CUDA(cudaEventElapsedTime(&ms, P.ev[2 * k], P.ev[2 * k + 1]));
        P.ms += ms; P.bytes += P.pend_bytes[k]; P.flops += P.pend_flops[k]; ++P.launches;
    }
    P.used = 0;
    return 0;
}

extern "C" int rich_profile(rich_ctx_t ctx, int enable) {
    if (!ctx) return RICH_ERR_INVALID;
    if (int e = rich_prof_harvest(ctx)) return e;
    ctx->prof.enabled = enable;
    ctx->prof.ms = ctx->prof.bytes = ctx->prof.flops = 0;
    ctx->prof.launches = 0;
    return 0;
}

extern "C" int rich_profile_read(rich_ctx_t ctx, double* ms, int64_t* launches, double* alg_bytes,
                                 double* alg_flops) {
    if (!ctx) return RICH_ERR_INVALID;
    RICH_CUDA(cudaDeviceSynchronize());
    if (int e = rich_prof_harvest(ctx)) return e;
    if (ms) *ms = ctx->prof.ms;
    if (launches) *launches = ctx->prof.launches;
    if (alg_bytes) *alg_bytes = ctx->prof.bytes;
    if (alg_flops) *alg_flops = ctx->prof.flops;
    return 0;
}

void rich_set_error(const char* msg, const char* file, int line) {
    snprintf(g_err, sizeof(g_err), "%s (%s:%d)", msg, file, line);
}

extern "C" const char* rich_last_error(void) { return g_err; }

extern "C" const char* rich_status_str(int code) {
    switch (code) {
        case RICH_OK: return "ok";
        case RICH_PICARD_MAXIT: return "picard iteration limit reached";
        case RICH_MG_MAXIT: return "multigrid cycle limit reached";
        case RICH_NONFINITE: return "non-finite residual or correction";
        case RICH_ADJ_MAXIT: return "adjoint linear-solve limit reached";
        case RICH_ERR_INVALID: return "invalid argument";
        case RICH_ERR_CUDA: return "CUDA error";
        case RICH_ERR_OOM: return "out of device memory";
        default: return "unknown status";
    }
}

extern "C" int rich_create(rich_ctx_t* out, int device) {
    if (!out) return RICH_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        rich_set_error("no such CUDA device", __FILE__, __LINE__);
        return RICH_ERR_CUDA;
    }
    RICH_CUDA(cudaSetDevice(device));
    rich_ctx* c = new (std::nothrow) rich_ctx();
    if (!c) return RICH_ERR_OOM;
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return 0;
}

extern "C" void rich_destroy(rich_ctx_t ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->sb.base) cudaFree(ctx->sb.base);
    if (ctx->stage) cudaFree(ctx->stage);
    for (auto& e : ctx->spectra) { cudaFree(e.sq); cudaFree(e.tw); }
    if (ctx->field_work) cudaFree(ctx->field_work);
    for (auto e : ctx->prof.ev) cudaEventDestroy(e);
    if (ctx->fused_scratch) cudaFree(ctx->fused_scratch);
    delete ctx;
}

int rich_check_problem(const rich_problem_t* pb) {
    if (!pb || pb->nx < 1 || pb->nz < 1 || pb->nsteps < 0 || !(pb->dt > 0) ||
        pb->picard_maxit < 1 || pb->mg_maxit < 1 || pb->nu1 < 0 || pb->nu2 < 0 ||
        (pb->precision != RICH_FP64 && pb->precision != RICH_MIXED) || !(pb->picard_tol > 0) ||
        pb->cycle < 0 || pb->cycle > 4 || (pb->closure != RICH_GARDNER && pb->closure != RICH_VAN_GENUCHTEN) ||
        !(pb->init_decay >= 0) || !(pb->init_decay < 1e300) || !(pb->mg_tol > 0))
        return RICH_ERR_INVALID;
    if (rich_count_levels(pb->nx, pb->nz) < 1) return RICH_ERR_INVALID;
    return 0;
}

extern "C" int rich_set_tuning(rich_ctx_t ctx, int32_t block_threads, int32_t mixed_inner) {
    if (!ctx || (block_threads != 0 && block_threads != 32 && block_threads != 128 && block_threads != 256 &&
                 block_threads != 512 && block_threads != 1024) ||
        mixed_inner < 0 ||
        mixed_inner > 16)
        return RICH_ERR_INVALID;
    ctx->tune_threads = block_threads;
    ctx->tune_mixed_inner = mixed_inner;
    return 0;
}

extern "C" int rich_sample_fields(rich_ctx_t ctx, const rich_field_t* field, int32_t nx,
                                  int32_t nz, uint32_t level, int64_t first_sample,
                                  int32_t nsamples, int32_t coarsen_times, double* lnKs,
                                  double* alpha, void* stream) {
    if (!ctx || !field || nsamples < 0 || first_sample < 0) return RICH_ERR_INVALID;
    if (nsamples > 0 && (!lnKs || !alpha)) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    return rich_fields_device(ctx, field, nx, nz, level, first_sample, nsamples, coarsen_times,
                              lnKs, alpha, (cudaStream_t)stream);
}

extern "C" int rich_sample_fields_at(rich_ctx_t ctx, const rich_field_t* field, int32_t nx,
                                     int32_t nz, uint32_t level, const int64_t* first_sample_dev,
                                     int32_t nsamples, int32_t coarsen_times, double* lnKs,
                                     double* alpha, void* stream) {
    if (!ctx || !field || nsamples < 0 || !first_sample_dev) return RICH_ERR_INVALID;
    if (nsamples > 0 && (!lnKs || !alpha)) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    return rich_fields_device(ctx, field, nx, nz, level, 0, nsamples, coarsen_times, lnKs, alpha,
                              (cudaStream_t)stream, first_sample_dev);
}

extern "C" int rich_solve_batch_async(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                                      const double* lnKs, const double* alpha, double alpha_scale,
                                      double* qoi, double* p_final, int32_t* status, void* stream) {
    if (!ctx || rich_check_problem(pb) || nsamples < 0) return RICH_ERR_INVALID;
    if (nsamples == 0) return 0;
    if (!lnKs || !alpha || !qoi) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    if (int e = rich_samples_reserve(ctx, nsamples)) return e;
    return rich_solve_fused(ctx, pb, nsamples, lnKs, alpha, alpha_scale, qoi, p_final, status,
                            (cudaStream_t)stream);
}

extern "C" int rich_sample_fields_pair(rich_ctx_t ctx, const rich_field_t* field, int32_t nx,
                                       int32_t nz, uint32_t level, int64_t first_sample,
                                       int32_t nsamples, double* lnKs_f, double* alpha_f,
                                       double* lnKs_c, double* alpha_c, void* stream) {
    if (!ctx || !field || nsamples < 0 || first_sample < 0) return RICH_ERR_INVALID;
    if (nsamples > 0 && (!lnKs_f || !alpha_f || !lnKs_c || !alpha_c)) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    return rich_fields_pair_device(ctx, field, nx, nz, level, first_sample, nsamples, lnKs_f, alpha_f,
                                   lnKs_c, alpha_c, (cudaStream_t)stream);
}

extern "C" int rich_solve_batch(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                                const double* lnKs, const double* alpha, double alpha_scale,
                                double* qoi, double* p_final, int32_t* status,
                                rich_stats_t* stats, void* stream) {
    if (!ctx || rich_check_problem(pb) || nsamples < 0) return RICH_ERR_INVALID;
    if (nsamples == 0) { if (stats) *stats = rich_stats_t{}; return 0; }
    if (!lnKs || !alpha || !qoi) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    return rich_solve_device(ctx, pb, nsamples, lnKs, alpha, alpha_scale, qoi, p_final, status,
                             stats, (cudaStream_t)stream);
}

extern "C" int rich_solve_soil(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                               const rich_soil_t* soil, double alpha_scale, double alpha_shift,
                               double n_shift, double* qoi, double* p_final, int32_t* status,
                               rich_stats_t* stats, void* stream) {
    if (!ctx || rich_check_problem(pb) || nsamples < 0 || !soil) return RICH_ERR_INVALID;
    if (!std::isfinite(alpha_scale) || !std::isfinite(alpha_shift) || !std::isfinite(n_shift))
        return RICH_ERR_INVALID;
    if (nsamples == 0) { if (stats) *stats = rich_stats_t{}; return 0; }
    if (!soil->lnKs || !soil->alpha || !qoi) return RICH_ERR_INVALID;
    if (pb->closure == RICH_VAN_GENUCHTEN && !soil->n) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    rich_soil_in in;
    in.n = soil->n; in.theta_s = soil->theta_s; in.theta_r = soil->theta_r;
    in.alpha_shift = alpha_shift; in.n_shift = n_shift;
    return rich_solve_device(ctx, pb, nsamples, soil->lnKs, soil->alpha, alpha_scale, qoi, p_final, status,
                             stats, (cudaStream_t)stream, &in);
}

extern "C" int rich_sample_soil(rich_ctx_t ctx, const rich_field_t* field, const rich_soil_model_t* soil,
                                int32_t nx, int32_t nz, uint32_t level, int64_t first_sample,
                                int32_t nsamples, int32_t coarsen_times, const rich_soil_t* out,
                                void* stream) {
    if (!ctx || !field || !soil || !out || nsamples < 0 || first_sample < 0) return RICH_ERR_INVALID;
    if (nsamples > 0 && (!out->lnKs || !out->alpha || !out->n)) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    return rich_soil_device(ctx, field, soil, nx, nz, level, first_sample, nsamples, coarsen_times, out,
                            (cudaStream_t)stream);
}

extern "C" int rich_sample_soil_pair(rich_ctx_t ctx, const rich_field_t* field, const rich_soil_model_t* soil,
                                     int32_t nx, int32_t nz, uint32_t level, int64_t first_sample,
                                     int32_t nsamples, const rich_soil_t* fine, const rich_soil_t* coarse,
                                     void* stream) {
    if (!ctx || !field || !soil || !fine || !coarse || nsamples < 0 || first_sample < 0) return RICH_ERR_INVALID;
    if (nsamples > 0 && (!fine->lnKs || !fine->alpha || !fine->n || !coarse->lnKs || !coarse->alpha || !coarse->n))
        return RICH_ERR_INVALID;
    if (!(soil->n_span >= 0) || !(soil->theta_s_span >= 0) || !(soil->theta_r_span >= 0)) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    return rich_soil_pair_device(ctx, field, soil, nx, nz, level, first_sample, nsamples, fine, coarse,
                                 (cudaStream_t)stream);
}

extern "C" int rich_sample_counters(rich_ctx_t ctx, int32_t nsamples, int64_t* picard_iters,
                                    int64_t* mg_cycles, void* stream) {
    if (!ctx || nsamples < 0 || nsamples > ctx->sb.last) return RICH_ERR_INVALID;
    if (nsamples == 0) return 0;
    RICH_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (picard_iters)
        RICH_CUDA(cudaMemcpyAsync(picard_iters, ctx->sb.pic_total, 8 * (size_t)nsamples, cudaMemcpyDeviceToDevice, st));
    if (mg_cycles)
        RICH_CUDA(cudaMemcpyAsync(mg_cycles, ctx->sb.mg_total, 8 * (size_t)nsamples, cudaMemcpyDeviceToDevice, st));
    return 0;
}

extern "C" int rich_solve_batch_host(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                                     const double* lnKs, const double* alpha, double alpha_scale,
                                     double* qoi, double* p_final, int32_t* status,
                                     rich_stats_t* stats, void* stream) {
    if (!ctx || rich_check_problem(pb) || nsamples < 0) return RICH_ERR_INVALID;
    if (nsamples == 0) { if (stats) *stats = rich_stats_t{}; return 0; }
    if (!lnKs || !alpha || !qoi) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nc = (size_t)nsamples * pb->nx * pb->nz;
    int e = rich_stage_reserve(ctx, 3 * nc * 8 + (size_t)nsamples * 12 + 256);
    if (e) return e;
    double* d_lk = (double*)ctx->stage;
    double* d_al = d_lk + nc;
    double* d_p = d_al + nc;
    double* d_q = d_p + nc;
    int32_t* d_st = (int32_t*)(d_q + nsamples);
    RICH_CUDA(cudaMemcpyAsync(d_lk, lnKs, nc * 8, cudaMemcpyHostToDevice, st));
    RICH_CUDA(cudaMemcpyAsync(d_al, alpha, nc * 8, cudaMemcpyHostToDevice, st));
    int rc = rich_solve_device(ctx, pb, nsamples, d_lk, d_al, alpha_scale, d_q,
                               p_final ? d_p : nullptr, d_st, stats, st);
    if (rc < 0) return rc;
    RICH_CUDA(cudaMemcpyAsync(qoi, d_q, (size_t)nsamples * 8, cudaMemcpyDeviceToHost, st));
    if (status) RICH_CUDA(cudaMemcpyAsync(status, d_st, (size_t)nsamples * 4, cudaMemcpyDeviceToHost, st));
    if (p_final) RICH_CUDA(cudaMemcpyAsync(p_final, d_p, nc * 8, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaStreamSynchronize(st));
    return rc;
}

// ---------------------------------------------------------------------------
// FP64 rate microbenchmark (the roofline denominator of the FP64-bound fused
// solver): independent chains of FP64 FMAs, divisions and exp calls on every
// SM, timed with CUDA events.  Chains are long enough to hide the pipeline
// latency; the results feed a store behind a data-dependent test so that the
// compiler keeps every operation.
// ---------------------------------------------------------------------------
namespace {
constexpr int PK_TPB = 256;
__device__ double g_peak_sink;

__global__ void __launch_bounds__(PK_TPB) k_peak_dfma(int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 1234.5678) g_peak_sink = s;
}

__global__ void __launch_bounds__(PK_TPB) k_peak_ddiv(int iters, double c) {
    double x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = c / (x[k] + 1.0);
    }
    const double s = x[0] + x[1] + x[2] + x[3];
    if (s == 1234.5678) g_peak_sink = s;
}

__global__ void __launch_bounds__(PK_TPB) k_peak_dexp(int iters, double c) {
    double x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = exp(-c * x[k]);
    }
    const double s = x[0] + x[1] + x[2] + x[3];
    if (s == 1234.5678) g_peak_sink = s;
}
}  // namespace

extern "C" int rich_measure_fp64(rich_ctx_t ctx, rich_fp64_rates_t* out) {
    if (!ctx || !out) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    float ms[3] = {0, 0, 0};
    const int grid = ctx->sm_count * (2048 / PK_TPB);
    const double threads = (double)grid * PK_TPB;
    const int it_fma = 1 << 16, it_div = 1 << 12, it_exp = 1 << 11;
    auto run = [&](int which, float* t) -> int {
        for (int rep = 0; rep < 2; ++rep) {      // first launch warms up, second is timed
            RICH_CUDA(cudaEventRecord(e0, st));
            rich_count_launch();
            if (which == 0) k_peak_dfma<<<grid, PK_TPB, 0, st>>>(it_fma, 0.999999, 1e-7);
            else if (which == 1) k_peak_ddiv<<<grid, PK_TPB, 0, st>>>(it_div, 0.75);
            else k_peak_dexp<<<grid, PK_TPB, 0, st>>>(it_exp, 0.5);
            RICH_CUDA(cudaGetLastError());
            RICH_CUDA(cudaEventRecord(e1, st));
            RICH_CUDA(cudaEventSynchronize(e1));
            RICH_CUDA(cudaEventElapsedTime(t, e0, e1));
        }
        return 0;
    };
    RICH_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        rich_set_error("cudaEventCreate failed", __FILE__, __LINE__);
        rc = RICH_ERR_CUDA;
    }
    for (int w = 0; w < 3 && rc == 0; ++w) rc = run(w, &ms[w]);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (rc) return rc;
    out->dfma_flops = 2.0 * 8.0 * it_fma * threads / (1e-3 * ms[0]);
    out->div_per_s = 4.0 * it_div * threads / (1e-3 * ms[1]);
    out->exp_per_s = 4.0 * it_exp * threads / (1e-3 * ms[2]);
    out->ms_total = ms[0] + ms[1] + ms[2];
    return 0;
}
