// FP64 accumulation of MC / MLMC level statistics on the device
// (arXiv 1903.08741, Sec. 5: Eqs. SMC_ch6, MC_var_ch6, ML_var_ch6).
#include "rich_internal.cuh"

namespace {

constexpr int ACC_TPB = 1024;

// Sums of eight per-thread values over the block in a fixed order (strided
// per-thread sums, then a fixed tree), so that repeated calls give
// bit-identical sums; the totals are in sm[k][0] for every thread on return.
__device__ void tree_sum8(const double (&v)[8], double (*sm)[ACC_TPB]) {
    for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = ACC_TPB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + w];
        __syncthreads();
    }
}

// One block.  Sample i counts when both statuses are RICH_OK, RICH_MG_MAXIT
// or RICH_ADJ_MAXIT (the QoI is defined); failed samples are counted
// separately and excluded from the sums.  With `shift` (the estimator's own
// statistics) the sums are of Y - K_Y, Qf - K_f, Qc - K_c about shifts fixed
// by the means of the first batch that has a defined sample (shift[3] = 1
// once set): the variance (S2 - S1^2/n)/(n - 1) of shifted data does not
// cancel when |mean| >> standard deviation (Chan, Golub & LeVeque 1983).
// Without it: plain sums, the layout of rich_mlmc_accumulate.
__global__ void __launch_bounds__(ACC_TPB)
k_accumulate(int n, const double* __restrict__ qf, const double* __restrict__ qc,
             const int32_t* __restrict__ sf, const int32_t* __restrict__ sc, double* acc, double* shift) {
    __shared__ double sm[8][ACC_TPB];
    auto bad = [&](int i) {
        return (sf && (sf[i] == RICH_PICARD_MAXIT || sf[i] == RICH_NONFINITE)) ||
               (qc && sc && (sc[i] == RICH_PICARD_MAXIT || sc[i] == RICH_NONFINITE)) || !isfinite(qf[i]) ||
               (qc && !isfinite(qc[i]));
    };
    double ky = 0.0, kf = 0.0, kc = 0.0;
    if (shift) {
        if (shift[3] == 0.0) {                  // first defined batch: its means become the shifts
            double m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                if (bad(i)) continue;
                const double f = qf[i], c = qc ? qc[i] : 0.0;
                m[0] += f - c; m[1] += f; m[2] += c; m[3] += 1;
            }
            tree_sum8(m, sm);
            const double cnt = sm[3][0];
            if (cnt > 0) { ky = sm[0][0] / cnt; kf = sm[1][0] / cnt; kc = sm[2][0] / cnt; }
            __syncthreads();
            if (threadIdx.x == 0 && cnt > 0) { shift[0] = ky; shift[1] = kf; shift[2] = kc; shift[3] = 1.0; }
        } else {
            ky = shift[0]; kf = shift[1]; kc = shift[2];
        }
    }
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};    // Y, Y^2, count, Qf, Qf^2, Qc, Qc^2, failed
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (bad(i)) { v[7] += 1; continue; }
        const double f = qf[i], c = qc ? qc[i] : 0.0;
        const double y = (f - c) - ky, fs = f - kf, cs = c - kc;
        v[0] += y; v[1] += y * y; v[2] += 1;
        v[3] += fs; v[4] += fs * fs; v[5] += cs; v[6] += cs * cs;
    }
    tree_sum8(v, sm);
    if (threadIdx.x == 0) {
        acc[0] += sm[0][0]; acc[1] += sm[1][0]; acc[2] += sm[2][0]; acc[3] += sm[7][0];
        acc[4] += sm[3][0]; acc[5] += sm[4][0]; acc[6] += sm[5][0]; acc[7] += sm[6][0];
    }
}

}  // namespace

extern "C" int rich_mlmc_accumulate(rich_ctx_t ctx, const double* qoi_fine, const double* qoi_coarse,
                                    const int32_t* status_fine, const int32_t* status_coarse,
                                    int32_t n, double* acc, void* stream) {
    if (!ctx || n < 0 || !acc || (n > 0 && !qoi_fine)) return RICH_ERR_INVALID;
    if (n == 0) return 0;
    RICH_CUDA(cudaSetDevice(ctx->device));
    rich_count_launch();
    k_accumulate<<<1, ACC_TPB, 0, (cudaStream_t)stream>>>(n, qoi_fine, qoi_coarse, status_fine,
                                                         status_coarse, acc, nullptr);
    RICH_CUDA(cudaGetLastError());
    return 0;
}

namespace {
// the estimator's accumulation: shifted sums (acc[8]) about shift[4]
int accumulate_shifted(const double* qf, const double* qc, const int32_t* sf, const int32_t* sc, int n,
                       double* acc, double* shift, cudaStream_t st) {
    if (n == 0) return 0;
    rich_count_launch();
    k_accumulate<<<1, ACC_TPB, 0, st>>>(n, qf, qc, sf, sc, acc, shift);
    RICH_CUDA(cudaGetLastError());
    return 0;
}
}  // namespace

// ------------------------------------------------------------------ estimator
#include <chrono>
#include <math.h>
#include <vector>
#include <algorithm>
#include <utility>

namespace {

// per level (and the bias pairs): 8 shifted sums (k_accumulate) + 4 shift values
constexpr int ACC_W = 12;

// mean and unbiased variance of n values from the sums s1, s2 of their
// deviations from the shift k (Eqs. SMC_ch6, MC_var_ch6)
void mean_var(double s1, double s2, double n, double k, double* m, double* v) {
    *m = n > 0 ? k + s1 / n : NAN;
    *v = n > 1 ? (s2 - s1 * (s1 / n)) / (n - 1) : NAN;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

// One estimator run: device buffers for a batch of B pairs, FP64 level sums on
// the device, per-level CUDA-event times.  Level l's samples are the indices
// 0, 1, 2, ... of its own noise stream (key level + key_offset), so adding
// samples later continues the stream exactly where it stopped.
struct MlmcRun {
    rich_ctx* ctx;
    const rich_mlmc_cfg_t* cfg;
    int NL, L, nL, B = 0;
    long long qcap = 0;                         // pairs the QoI / status buffers hold
    cudaStream_t st = nullptr;
    cudaEvent_t ev[4] = {};
    // the coarse member of each pair is solved at the same time as the fine
    // one, by a second context on a second stream: the two solves are
    // independent, and a level with fewer samples than the GPU has SMs
    // (e.g. 80 pairs at 256^2) would otherwise leave SMs idle twice
    rich_ctx* ctx2 = nullptr;
    cudaStream_t st2 = nullptr;
    cudaEvent_t evc = nullptr;
    DevBuf lkf, alf, lkc, alc, qf, qc, sf, sc, acc;
    DevBuf nf, tsf, trf, ncb, tsc, trc;     // van Genuchten: n, theta_s, theta_r (fine, coarse)
    bool vg = false, thetas = false;
    std::vector<double> t_pair, t_fine, t_sm;   // wall time; GPU-seconds at full occupancy
    std::vector<long long> n_done;
    int worst = 0;
    // grid-only bias pairs: both members of the finest pair with the original
    // parameters (no continuation), own noise stream, own accumulator slot NL
    bool bias_mode = false;
    long long n_bias = 0;
    static constexpr uint32_t BIAS_KEY = 64;

    MlmcRun(rich_ctx* c, const rich_mlmc_cfg_t* g) : ctx(c), cfg(g) {
        NL = g->nlevels; L = NL - 1; nL = g->n0 << L;
        vg = g->base.closure == RICH_VAN_GENUCHTEN;
        thetas = vg && g->with_thetas;
        t_pair.assign(NL, 0.0); t_fine.assign(NL, 0.0); t_sm.assign(NL, 0.0); n_done.assign(NL, 0);
    }
    ~MlmcRun() {
        for (auto& e : ev) if (e) cudaEventDestroy(e);
        if (evc) cudaEventDestroy(evc);
        if (st) cudaStreamDestroy(st);
        if (st2) cudaStreamDestroy(st2);
        if (ctx2) rich_destroy(ctx2);
    }
    int grid(int l) const { return cfg->n0 << l; }
    int steps(int l) const { return cfg->steps0 << l; }
    double ascale(int l) const {
        return (cfg->continuation && !vg && !bias_mode) ? (double)(l + 1) / (double)NL : 1.0;
    }
    // van Genuchten continuation steps of level l (Sec. 5.2): the
    // fixed_levels finest levels keep the original alpha and n
    int vg_steps(int l) const {
        if (!cfg->continuation || bias_mode) return 0;
        const int fixed = std::max(1, (int)cfg->fixed_levels);
        return std::max(0, L + 1 - fixed - l);
    }
    rich_soil_in soil_in(int l, bool coarse) const {
        rich_soil_in in;
        in.n = (const double*)(coarse ? ncb.p : nf.p);
        in.theta_s = thetas ? (const double*)(coarse ? tsc.p : tsf.p) : nullptr;
        in.theta_r = thetas ? (const double*)(coarse ? trc.p : trf.p) : nullptr;
        in.alpha_shift = -vg_steps(l) * cfg->d_alpha;
        in.n_shift = vg_steps(l) * cfg->d_n;
        return in;
    }

    int init(int batch_hint) {
        RICH_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        RICH_CUDA(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
        for (auto& e : ev) RICH_CUDA(cudaEventCreate(&e));
        RICH_CUDA(cudaEventCreateWithFlags(&evc, cudaEventDisableTiming));
        if (int e = rich_create(&ctx2, ctx->device)) return e;
        B = cfg->batch > 0 ? cfg->batch : (int)std::max<long long>(1, (1ll << 31) / (16ll * nL * nL));
        B = std::max(1, std::min(B, batch_hint));
        const size_t fine_cells = (size_t)B * nL * nL;       // worst case: level L fine member
        auto dalloc = [&](DevBuf& b, size_t bytes) -> int {
            cudaError_t e = cudaMalloc(&b.p, std::max<size_t>(bytes, 256));
            if (e != cudaSuccess) { cudaGetLastError(); return RICH_ERR_OOM; }
            return 0;
        };
        if (dalloc(lkf, fine_cells * 8) || dalloc(alf, fine_cells * 8) || dalloc(lkc, fine_cells * 2) ||
            dalloc(alc, fine_cells * 2) || dalloc(acc, 8 * ACC_W * (NL + 1)))
            return RICH_ERR_OOM;
        if (vg && (dalloc(nf, fine_cells * 8) || dalloc(ncb, fine_cells * 2)))
            return RICH_ERR_OOM;
        if (thetas && (dalloc(tsf, fine_cells * 8) || dalloc(trf, fine_cells * 8) || dalloc(tsc, fine_cells * 2) ||
                       dalloc(trc, fine_cells * 2)))
            return RICH_ERR_OOM;
        RICH_CUDA(cudaMemsetAsync(acc.p, 0, 8 * ACC_W * (NL + 1), st));
        return 0;
    }

    // pairs per launch on level l: the field buffers hold B finest-level
    // fields, i.e. B (n_L / M)^2 fields of a level on an M x M grid, so a
    // coarse level runs in few large launches (each launch ends with a tail
    // in which its last samples finish); cfg->batch > 0 fixes B for all
    long long level_batch(int l) const {
        if (cfg->batch > 0) return B;
        const long long r = nL / grid(l);
        return (long long)B * r * r;
    }
    // QoI and status buffers for n pairs (grown between levels; the previous
    // batch has completed: batch() ends with a synchronisation)
    int ensure_q(long long n) {
        if (n <= qcap) return 0;
        for (DevBuf* b : {&qf, &qc, &sf, &sc}) {
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
        }
        qcap = 0;
        for (auto [b, w] : {std::pair<DevBuf*, size_t>{&qf, 8}, {&qc, 8}, {&sf, 4}, {&sc, 4}}) {
            cudaError_t e = cudaMalloc(&b->p, std::max<size_t>((size_t)n * w, 256));
            if (e != cudaSuccess) { cudaGetLastError(); return RICH_ERR_OOM; }
        }
        qcap = n;
        return 0;
    }

    // pairs first .. first+count-1 of level l: fields, fine and coarse solves, sums
    int run_level(int l, long long first, long long count) {
        const int M = grid(l);
        rich_problem_t pf = cfg->base;
        pf.nx = pf.nz = M; pf.nsteps = steps(l); pf.dt = cfg->t_final / steps(l);
        rich_problem_t pc = cfg->base;
        if (l > 0) { pc.nx = pc.nz = grid(l - 1); pc.nsteps = steps(l - 1); pc.dt = cfg->t_final / steps(l - 1); }
        const int ndraw = cfg->coupling == 0 ? nL : M;
        const int coarsen = cfg->coupling == 0 ? L - l : 0;
        const int save_t = ctx->tune_threads, save_i = ctx->tune_mixed_inner;
        if (cfg->tune_threads[l]) ctx->tune_threads = cfg->tune_threads[l];
        if (cfg->tune_inner[l]) ctx->tune_mixed_inner = cfg->tune_inner[l];
        const long long Bl = level_batch(l);
        if (int e = ensure_q(std::min(count, Bl))) return e;
        int rc_all = 0;
        for (long long b0 = 0; b0 < count && rc_all >= 0; b0 += Bl) {
            const int nb = (int)std::min<long long>(Bl, count - b0);
            const long long s0 = first + b0;
            rc_all = batch(l, s0, nb, M, ndraw, coarsen, pf, pc);
        }
        ctx->tune_threads = save_t; ctx->tune_mixed_inner = save_i;
        if (rc_all < 0) return rc_all;
        if (bias_mode) n_bias += count; else n_done[l] += count;
        return 0;
    }
    // `count` pairs (finest grid, next coarser grid) that differ only in the
    // grid: the discretisation-bias estimate of Eq. discErr without the
    // parameter jump that the continuation puts into the finest level
    int run_bias(long long count) {
        if (L < 1 || count < 1) return 0;
        bias_mode = true;
        const int e = run_level(L, n_bias, count);
        bias_mode = false;
        return e;
    }
    int batch(int l, long long s0, int nb, int M, int ndraw, int coarsen, const rich_problem_t& pf,
              const rich_problem_t& pc) {
        RICH_CUDA(cudaEventRecord(ev[0], st));
        int e;
        const uint32_t key = (bias_mode ? BIAS_KEY : (uint32_t)l) + cfg->key_offset;
        const rich_soil_t fine{(double*)lkf.p, (double*)alf.p, (double*)nf.p, thetas ? (double*)tsf.p : nullptr,
                               thetas ? (double*)trf.p : nullptr};
        const rich_soil_t crs{(double*)lkc.p, (double*)alc.p, (double*)ncb.p, thetas ? (double*)tsc.p : nullptr,
                              thetas ? (double*)trc.p : nullptr};
        if (vg) {
            if (cfg->coupling == 2 && l > 0)
                e = rich_soil_pair_device(ctx, &cfg->field, &cfg->soil, M, M, key, s0, nb, &fine, &crs, st);
            else
                e = rich_soil_device(ctx, &cfg->field, &cfg->soil, ndraw, ndraw, key, s0, nb, coarsen, &fine, st);
        } else if (cfg->coupling == 2 && l > 0) {
            e = rich_fields_pair_device(ctx, &cfg->field, M, M, key, s0, nb, (double*)lkf.p, (double*)alf.p,
                                        (double*)lkc.p, (double*)alc.p, st);
        } else {
            e = rich_fields_device(ctx, &cfg->field, ndraw, ndraw, key, s0, nb, coarsen, (double*)lkf.p,
                                   (double*)alf.p, st);
        }
        if (e) return e;
        if (l > 0 && cfg->coupling != 2) {
            e = rich_fields_average(ctx, nb, M, M, (double*)lkf.p, (double*)alf.p, (double*)lkc.p,
                                    (double*)alc.p, st);
            if (!e && vg)
                e = rich_fields_average(ctx, nb, M, M, fine.n, fine.theta_s, crs.n, crs.theta_s, st);
            if (!e && thetas)
                e = rich_fields_average(ctx, nb, M, M, fine.theta_r, nullptr, crs.theta_r, nullptr, st);
            if (e) return e;
        }
        RICH_CUDA(cudaEventRecord(ev[1], st));
        const rich_soil_in in_f = soil_in(l, false), in_c = soil_in(l > 0 ? l - 1 : 0, true);
        // fine member on (ctx, st); coarse member on (ctx2, st2) once the fields exist
        if (int e2 = rich_samples_reserve(ctx, nb)) return e2;
        int rc = rich_solve_fused(ctx, &pf, nb, (double*)lkf.p, (double*)alf.p, ascale(l), (double*)qf.p, nullptr,
                                  (int32_t*)sf.p, st, vg ? &in_f : nullptr);
        if (rc < 0) return rc;
        RICH_CUDA(cudaEventRecord(ev[2], st));
        if (l > 0) {
            if (int e2 = rich_samples_reserve(ctx2, nb)) return e2;
            ctx2->tune_threads = cfg->tune_threads[l - 1] ? cfg->tune_threads[l - 1] : ctx->tune_threads;
            ctx2->tune_mixed_inner = cfg->tune_inner[l - 1] ? cfg->tune_inner[l - 1] : ctx->tune_mixed_inner;
            RICH_CUDA(cudaStreamWaitEvent(st2, ev[1], 0));
            rc = rich_solve_fused(ctx2, &pc, nb, (double*)lkc.p, (double*)alc.p, ascale(l - 1), (double*)qc.p,
                                  nullptr, (int32_t*)sc.p, st2, vg ? &in_c : nullptr);
            if (rc < 0) return rc;
            RICH_CUDA(cudaEventRecord(evc, st2));
            RICH_CUDA(cudaStreamWaitEvent(st, evc, 0));
        }
        double* lacc = (double*)acc.p + ACC_W * (bias_mode ? NL : l);
        e = accumulate_shifted((double*)qf.p, l > 0 ? (double*)qc.p : nullptr, (int32_t*)sf.p,
                               l > 0 ? (int32_t*)sc.p : nullptr, nb, lacc, lacc + 8, st);
        if (e) return e;
        RICH_CUDA(cudaEventRecord(ev[3], st));
        RICH_CUDA(cudaEventSynchronize(ev[3]));
        // most severe status of the batch, and the solves' SM-seconds
        {
            std::vector<int32_t> hs(2 * (size_t)nb, 0);
            RICH_CUDA(cudaMemcpy(hs.data(), sf.p, 4 * (size_t)nb, cudaMemcpyDeviceToHost));
            if (l > 0) RICH_CUDA(cudaMemcpy(hs.data() + nb, sc.p, 4 * (size_t)nb, cudaMemcpyDeviceToHost));
            for (int32_t v : hs) worst = rich_status_worse(worst, (int)v);
        }
        double sm_s = 0.0, sm_c = 0.0;
        if (int e2 = rich_sm_seconds(ctx, nb, st, &sm_s)) return e2;
        if (l > 0) {
            if (int e2 = rich_sm_seconds(ctx2, nb, st2, &sm_c)) return e2;
            sm_s += sm_c;
        }
        float a = 0, b = 0, c = 0;
        RICH_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
        RICH_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
        RICH_CUDA(cudaEventElapsedTime(&c, ev[2], ev[3]));
        if (bias_mode) return 0;
        t_sm[l] += 1e-3 * a + sm_s / std::max(ctx->sm_count, 1);
        t_pair[l] += 1e-3 * (a + b + c);
        t_fine[l] += 1e-3 * (a + b);      // one draw + one fine solve (plain MC sample)
        return 0;
    }

    // level statistics from the device sums (Eqs. SMC_ch6, MC_var_ch6,
    // eq:MLMCVar, ML_var_ch6, MLMCSAMP_ch6)
    int finalize(rich_mlmc_result_t* out) {
        std::vector<double> h(ACC_W * (NL + 1));
        RICH_CUDA(cudaMemcpyAsync(h.data(), acc.p, 8 * ACC_W * (NL + 1), cudaMemcpyDeviceToHost, st));
        RICH_CUDA(cudaStreamSynchronize(st));
        rich_mlmc_result_t r{};
        r.nlevels = NL;
        double rmse2 = 0, ssum = 0, ssum_sm = 0;
        for (int l = 0; l < NL; ++l) {
            const double* a = &h[ACC_W * l];
            const double n = a[2];
            r.n[l] = (int64_t)n; r.failed[l] = (int64_t)a[3];
            mean_var(a[0], a[1], n, a[8], &r.mean[l], &r.var[l]);
            mean_var(a[4], a[5], n, a[9], &r.mean_f[l], &r.var_f[l]);
            if (l > 0) mean_var(a[6], a[7], n, a[10], &r.mean_c[l], &r.var_c[l]);
            r.cost[l] = n_done[l] > 0 ? t_pair[l] / n_done[l] : NAN;
            r.cost_fine[l] = n_done[l] > 0 ? t_fine[l] / n_done[l] : NAN;
            r.cost_sm[l] = n_done[l] > 0 ? t_sm[l] / n_done[l] : NAN;
            r.estimate += r.mean[l];
            rmse2 += r.var[l] / n;
            r.ml_variance += r.var_f[l] - (l > 0 ? r.var_c[l] : 0.0);
            ssum += sqrt(std::max(r.var[l], 0.0) * r.cost[l]);
            ssum_sm += sqrt(std::max(r.var[l], 0.0) * r.cost_sm[l]);
        }
        r.rmse = sqrt(rmse2);
        if (cfg->eps > 0) {
            const double e2 = cfg->eps * cfg->eps;
            for (int l = 0; l < NL; ++l) r.n_opt[l] = ssum * sqrt(std::max(r.var[l], 0.0) / r.cost[l]) / e2;
            r.w_eps = ssum * ssum / e2;
            r.w_eps_sm = ssum_sm * ssum_sm / e2;
            r.w_mc_eps = r.var_f[L] * r.cost_fine[L] / e2;
        }
        r.bias_estimate = L > 0 ? fabs(r.mean[L]) / (2.0 - 1.0) : NAN;
        // grid-only bias (Eq. discErr with rate a = 1): |E[Q_L - Q_{L-1}]| at the
        // original parameters / (2^a - 1); total RMSE sqrt(bias^2 + sum V_l/N_l)
        // (Eq. MSEMLMC_ch6); levels needed so that the bias, halving per level,
        // falls to eps / sqrt 2 (half of the MSE budget)
        const double* b = &h[ACC_W * NL];
        r.bias_pairs = (int64_t)b[2];
        if (b[2] > 0) {
            double m, v;
            mean_var(b[0], b[1], b[2], b[8], &m, &v);
            r.bias_grid = fabs(m) / (2.0 - 1.0);
            r.bias_grid_se = b[2] > 1 ? sqrt(std::max(v, 0.0) / b[2]) : NAN;
            r.total_rmse = sqrt(r.bias_grid * r.bias_grid + rmse2);
            if (cfg->eps > 0) {
                const double lim = cfg->eps / sqrt(2.0);
                int extra = 0;
                for (double bb = r.bias_grid; bb > lim && extra < 64; bb *= 0.5) ++extra;
                r.levels_for_eps = NL + extra;
            }
        } else {
            r.bias_grid = r.bias_grid_se = r.total_rmse = NAN;
        }
        *out = r;
        return 0;
    }
};

int check_cfg(const rich_mlmc_cfg_t* cfg) {
    const int NL = cfg->nlevels;
    if (NL < 1 || NL > RICH_MLMC_MAX_LEVELS || cfg->n0 < 2 || cfg->steps0 < 1 || !(cfg->t_final > 0) ||
        cfg->coupling < 0 || cfg->coupling > 2)
        return RICH_ERR_INVALID;
    rich_problem_t p0 = cfg->base;
    p0.nx = p0.nz = cfg->n0; p0.nsteps = cfg->steps0; p0.dt = cfg->t_final / cfg->steps0;
    if (rich_check_problem(&p0)) return RICH_ERR_INVALID;
    if (cfg->base.closure == RICH_VAN_GENUCHTEN &&
        (!(cfg->d_alpha >= 0) || !(cfg->d_n >= 0) || cfg->fixed_levels < 0 || !(cfg->soil.n_span >= 0) ||
         !(cfg->soil.theta_s_span >= 0) || !(cfg->soil.theta_r_span >= 0)))
        return RICH_ERR_INVALID;
    for (int l = 0; l < NL; ++l) {
        if (cfg->nsamples[l] < 2) return RICH_ERR_INVALID;
        if (cfg->bias_pairs < 0) return RICH_ERR_INVALID;
        if (cfg->tune_threads[l] != 0 && cfg->tune_threads[l] != 32 && cfg->tune_threads[l] != 128 &&
            cfg->tune_threads[l] != 256 &&
            cfg->tune_threads[l] != 512 &&
            cfg->tune_threads[l] != 1024)
            return RICH_ERR_INVALID;
        if (cfg->tune_inner[l] < 0 || cfg->tune_inner[l] > 16) return RICH_ERR_INVALID;
    }
    return 0;
}

}  // namespace

extern "C" int rich_mlmc_estimate(rich_ctx_t ctx, const rich_mlmc_cfg_t* cfg, rich_mlmc_result_t* out) {
    if (!ctx || !cfg || !out || check_cfg(cfg)) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    auto t0 = std::chrono::steady_clock::now();
    MlmcRun run(ctx, cfg);
    int maxN = 0;
    for (int l = 0; l < cfg->nlevels; ++l) maxN = std::max(maxN, cfg->nsamples[l]);
    if (int e = run.init(maxN)) return e;
    for (int l = 0; l < cfg->nlevels; ++l)
        if (int e = run.run_level(l, 0, cfg->nsamples[l])) return e;
    if (int e = run.run_bias(cfg->bias_pairs)) return e;
    if (int e = run.finalize(out)) return e;
    out->rounds = 1;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return run.worst;
}

// Algorithm PC_MLMC (Sec. 5.2): warm-up with N*_l = cfg->nsamples, then repeat
// {N_l <- optimal allocation (Eq. MLMCSAMP_ch6) from the current V_l and the
// per-sample costs measured so far; run the missing samples of every level,
// N_l counting the pairs with a defined QoI}
// until no level needs more samples, at most max_rounds rounds or until a
// level would exceed nmax[l] (NULL: no cap).
extern "C" int rich_mlmc_adaptive(rich_ctx_t ctx, const rich_mlmc_cfg_t* cfg, int32_t max_rounds,
                                  const int64_t* nmax, rich_mlmc_result_t* out) {
    if (!ctx || !cfg || !out || check_cfg(cfg) || !(cfg->eps > 0) || max_rounds < 1) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    auto t0 = std::chrono::steady_clock::now();
    MlmcRun run(ctx, cfg);
    int maxN = 0;
    for (int l = 0; l < cfg->nlevels; ++l) maxN = std::max(maxN, cfg->nsamples[l]);
    if (int e = run.init(std::max(maxN, 4096))) return e;
    for (int l = 0; l < cfg->nlevels; ++l)
        if (int e = run.run_level(l, 0, cfg->nsamples[l])) return e;
    int rounds = 1;
    for (;;) {
        if (int e = run.finalize(out)) return e;
        if (rounds >= max_rounds) break;
        bool more = false;
        std::vector<long long> add(cfg->nlevels, 0);
        for (int l = 0; l < cfg->nlevels; ++l) {
            // V_l / N_l counts the pairs with a defined QoI (failed pairs are
            // excluded), so those must reach the optimal N_l; nmax caps the
            // pairs run, failed or not
            // (a level with fewer than two defined pairs has no variance and
            // every n_opt is NaN: top that level up to two defined pairs first)
            const double no = out->n_opt[l];
            long long want = (std::isfinite(no) ? (long long)ceil(no) : 2) - out->n[l];
            if (nmax) want = std::min<long long>(want, nmax[l] - run.n_done[l]);
            if (want > 0) { add[l] = want; more = true; }
        }
        if (!more) break;
        for (int l = 0; l < cfg->nlevels; ++l)
            if (add[l] > 0)
                if (int e = run.run_level(l, run.n_done[l], add[l])) return e;
        ++rounds;
    }
    if (cfg->bias_pairs > 0) {
        if (int e = run.run_bias(cfg->bias_pairs)) return e;
        if (int e = run.finalize(out)) return e;
    }
    out->rounds = rounds;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return run.worst;
}
