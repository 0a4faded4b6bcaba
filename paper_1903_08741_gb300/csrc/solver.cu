// Host side of the batched solve: argument checks, per-sample buffers, the
// fused persistent kernel (fused.cu), per-sample counters -> rich_stats_t.
#include "rich_internal.cuh"
#include <algorithm>
#include <chrono>
#include <vector>

// Multigrid hierarchy depth: halve while both sides are even and more than 4
// cells remain; the coarsest grid (solved exactly) must have at most 64 cells.
int rich_count_levels(int nx, int nz) {
    if (nx < 1 || nz < 1) return -1;
    int n = 1;
    while (nx % 2 == 0 && nz % 2 == 0 && nx * nz > 4) { nx /= 2; nz /= 2; ++n; }
    if (n > RICH_MAX_LEVELS) return -1;
    return (nx * nz <= 64) ? n : -1;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// per-sample status and counters of the last solve, grown on demand
int rich_samples_reserve(rich_ctx* ctx, int S) {
    rich_samplebuf& b = ctx->sb;
    if (b.base && b.cap >= S) return 0;
    if (b.base) cudaFree(b.base);
    b.base = nullptr; b.cap = 0;
    const size_t n = (size_t)std::max(S, 1);
    size_t off = 0;
    const size_t o_st = off; off = al256(off + 4 * n);
    const size_t o_mx = off; off = al256(off + 4 * n);
    const size_t o_pt = off; off = al256(off + 8 * n);
    const size_t o_mt = off; off = al256(off + 8 * n);
    const size_t o_tn = off; off = al256(off + 8 * n);
    cudaError_t e = cudaMalloc(&b.base, off);
    if (e != cudaSuccess) { cudaGetLastError(); b.base = nullptr; return RICH_ERR_OOM; }
    char* c = (char*)b.base;
    b.status = (int32_t*)(c + o_st); b.maxpic = (int32_t*)(c + o_mx);
    b.pic_total = (int64_t*)(c + o_pt); b.mg_total = (int64_t*)(c + o_mt); b.t_ns = (int64_t*)(c + o_tn);
    b.cap = (int)n;
    return 0;
}

// device staging for the host-buffer entry point
int rich_stage_reserve(rich_ctx* ctx, size_t bytes) {
    if (ctx->stage && ctx->stage_bytes >= bytes) return 0;
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr; ctx->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->stage, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return RICH_ERR_OOM; }
    ctx->stage_bytes = bytes;
    return 0;
}

// SM-seconds of the context's last fused solve of S samples: each sample held
// 1/occ of an SM for its solve time on its CTA (synchronises `st`)
int rich_sm_seconds(rich_ctx* ctx, int S, cudaStream_t st, double* out) {
    std::vector<int64_t> ht(std::max(S, 1));
    if (S > 0) RICH_CUDA(cudaMemcpyAsync(ht.data(), ctx->sb.t_ns, 8 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaStreamSynchronize(st));
    double cta_ns = 0;
    for (int s = 0; s < S; ++s) cta_ns += (double)ht[s];
    *out = 1e-9 * cta_ns / std::max(ctx->sb.last_occ, 1);
    return 0;
}

int rich_solve_device(rich_ctx* ctx, const rich_problem_t* pb, int S, const double* lnKs,
                      const double* alpha, double alpha_scale, double* qoi, double* p_final,
                      int32_t* status, rich_stats_t* stats, cudaStream_t st, const rich_soil_in* soil) {
    auto t0 = std::chrono::steady_clock::now();
    if (int e = rich_samples_reserve(ctx, S)) return e;
    if (int e = rich_solve_fused(ctx, pb, S, lnKs, alpha, alpha_scale, qoi, p_final, status, st, soil))
        return e;
    rich_samplebuf& b = ctx->sb;
    std::vector<int32_t> hs(S), hmax(S);
    std::vector<int64_t> hp(S), hm(S), ht(S);
    RICH_CUDA(cudaMemcpyAsync(ht.data(), b.t_ns, 8 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hs.data(), b.status, 4 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hmax.data(), b.maxpic, 4 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hp.data(), b.pic_total, 8 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hm.data(), b.mg_total, 8 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaStreamSynchronize(st));
    int worst = 0;
    rich_stats_t acc{};
    double cta_ns = 0;
    for (int s = 0; s < S; ++s) cta_ns += (double)ht[s];
    // SM-seconds: each sample held 1/occ of an SM for its solve time
    ctx->last_sm_seconds = 1e-9 * cta_ns / std::max(b.last_occ, 1);
    acc.sm_seconds = ctx->last_sm_seconds;
    for (int s = 0; s < S; ++s) {
        worst = rich_status_worse(worst, (int)hs[s]);
        acc.picard_iters += hp[s];
        acc.mg_cycles += hm[s];
        acc.max_picard = std::max(acc.max_picard, hmax[s]);
        if (hs[s] == RICH_PICARD_MAXIT || hs[s] == RICH_NONFINITE) acc.failed++;
    }
    acc.cell_vcycles = acc.mg_cycles * (int64_t)pb->nx * pb->nz;
    // algorithmic work of the fused launch (for the live roofline), per fine
    // cell.  V-cycle (V(2,2), FMA = 2 FLOP): on the finest level 2 x 2 sweeps of
    // 8 FLOP per cell (4 FMA per Gauss-Seidel update) = 32, the red-only
    // residual restriction 23 per coarse cell = 5.75, prolongation 1: 38.75;
    // each coarser level the same less the seeded first red half-sweep (4):
    // 34.75, hierarchy factor 1/3; the red-only stopping norm 5: 55 FLOP.
    // Picard iteration: closure 6 (+ one exp), harmonic faces 8, mixed-form
    // residual 20, scaled coefficients 6, coarse operators ~26 per coarse cell
    // (8.7), update 1: 51 FLOP.  Bytes: the two-fused-passes model, 16.7 words
    // per cell and V-cycle and 10 FP64 words per cell and Picard iteration.
    const double nc = (double)pb->nx * pb->nz;
    const double w8 = pb->precision == RICH_MIXED ? 4.0 : 8.0;
    const double flops = nc * (55.0 * acc.mg_cycles + 51.0 * acc.picard_iters);
    const double bytes = nc * (16.7 * w8 * acc.mg_cycles + 10.0 * 8.0 * acc.picard_iters);
    rich_prof_amend(ctx, bytes, flops);
    acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = acc;
    return worst;
}
