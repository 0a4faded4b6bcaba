// KL fields and the gradient of the bottom-flux QoI with respect to the KL
// coefficients (Sec. 3, Eq. KLexp_ch6; adjoint of the time-stepped solve in
// fused.cu):  ln Ks_s = sum_j xi_sj B_j,  dQ_s/dxi_sj = sum_c B_j(c) dQ_s/d lnKs_s(c).
#include "rich_internal.cuh"
#include <algorithm>
#include <vector>
#include <chrono>

namespace {

constexpr int KT = 256;

// ln Ks[s][c] = sum_j xi[s][j] basis[j][c]; xi of the block's sample staged in
// shared memory, one thread per cell (coalesced over the basis rows)
__global__ void k_kl_fields(int nkl, int nc, const double* __restrict__ basis,
                            const double* __restrict__ xi, double* lnKs) {
    extern __shared__ double sx[];
    const int s = blockIdx.y;
    for (int j = threadIdx.x; j < nkl; j += blockDim.x) sx[j] = xi[(size_t)s * nkl + j];
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double v = 0.0;
    for (int j = 0; j < nkl; ++j) v += sx[j] * basis[(size_t)j * nc + c];
    lnKs[(size_t)s * nc + c] = v;
}

// out[s][j] = sum_c basis[j][c] g[s][c]: one block per (sample, mode), block
// reduction in a fixed order (deterministic)
__global__ void k_kl_project(int nkl, int nc, const double* __restrict__ basis,
                             const double* __restrict__ g, double* out) {
    __shared__ double sm[KT];
    const int j = blockIdx.x, s = blockIdx.y;
    const double* b = basis + (size_t)j * nc;
    const double* gs = g + (size_t)s * nc;
    double v = 0.0;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) v += b[c] * gs[c];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int w = KT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)s * nkl + j] = sm[0];
}

}  // namespace

extern "C" int rich_kl_fields(rich_ctx_t ctx, const double* basis, int32_t n_kl, int32_t ncell,
                              const double* xi, int32_t nsamples, double* lnKs, void* stream) {
    if (!ctx || n_kl < 1 || ncell < 1 || nsamples < 0 || !basis) return RICH_ERR_INVALID;
    if (nsamples == 0) return 0;
    if (!xi || !lnKs || nsamples > 65535) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    dim3 grid((ncell + KT - 1) / KT, nsamples);
    rich_count_launch();
    k_kl_fields<<<grid, KT, sizeof(double) * n_kl, (cudaStream_t)stream>>>(n_kl, ncell, basis, xi, lnKs);
    RICH_CUDA(cudaGetLastError());
    return 0;
}

extern "C" int rich_solve_batch_adjoint(rich_ctx_t ctx, const rich_problem_t* pb, int32_t nsamples,
                                        const double* kl_basis, int32_t n_kl, const double* xi,
                                        const double* alpha, double alpha_scale, int32_t ckpt_every,
                                        double* qoi, double* dq_dxi, double* dq_dlnKs,
                                        int32_t* status, rich_stats_t* stats, void* stream) {
    if (!ctx || rich_check_problem(pb) || nsamples < 0 || n_kl < 1 || ckpt_every < 1)
        return RICH_ERR_INVALID;
    if (nsamples == 0) { if (stats) *stats = rich_stats_t{}; return 0; }
    if (!kl_basis || !xi || !alpha || !qoi || !dq_dxi || nsamples > 65535) return RICH_ERR_INVALID;
    RICH_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int nc = pb->nx * pb->nz;
    // device scratch: ln Ks and (if the caller did not ask for it) dQ/d ln Ks
    size_t need = sizeof(double) * (size_t)nsamples * nc * (dq_dlnKs ? 1 : 2);
    if (int e = rich_stage_reserve(ctx, need)) return e;
    double* lk = (double*)ctx->stage;
    double* g = dq_dlnKs ? dq_dlnKs : lk + (size_t)nsamples * nc;
    if (int e = rich_kl_fields(ctx, kl_basis, n_kl, nc, xi, nsamples, lk, stream)) return e;
    if (int e = rich_samples_reserve(ctx, nsamples)) return e;
    auto t0 = std::chrono::steady_clock::now();
    // adjoint linear solves to the context's relative residual (default 1e-11),
    // at most its cap of preconditioner applications (default 400)
    if (int e = rich_adjoint_fused(ctx, pb, nsamples, lk, alpha, alpha_scale, ckpt_every, ctx->adj_tol, ctx->adj_cap,
                                   ctx->adj_method, qoi, g, st))
        return e;
    dim3 grid(n_kl, nsamples);
    rich_count_launch();
    k_kl_project<<<grid, KT, 0, st>>>(n_kl, nc, kl_basis, g, dq_dxi);
    RICH_CUDA(cudaGetLastError());
    rich_samplebuf& b = ctx->sb;
    std::vector<int32_t> hs(nsamples), hmax(nsamples);
    std::vector<int64_t> hp(nsamples), hm(nsamples);
    RICH_CUDA(cudaMemcpyAsync(hs.data(), b.status, 4 * (size_t)nsamples, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hmax.data(), b.maxpic, 4 * (size_t)nsamples, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hp.data(), b.pic_total, 8 * (size_t)nsamples, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hm.data(), b.mg_total, 8 * (size_t)nsamples, cudaMemcpyDeviceToHost, st));
    if (status)
        RICH_CUDA(cudaMemcpyAsync(status, b.status, 4 * (size_t)nsamples, cudaMemcpyDeviceToDevice, st));
    RICH_CUDA(cudaStreamSynchronize(st));
    int worst = 0;
    rich_stats_t acc{};
    for (int s = 0; s < nsamples; ++s) {
        worst = rich_status_worse(worst, (int)hs[s]);
        acc.picard_iters += hp[s];
        acc.mg_cycles += hm[s];          // adjoint: preconditioner applications of the J^T solves
        acc.max_picard = std::max(acc.max_picard, hmax[s]);
        if (hs[s] == RICH_PICARD_MAXIT || hs[s] == RICH_NONFINITE) acc.failed++;
    }
    acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = acc;
    return worst;
}

extern "C" int rich_set_adjoint_method(rich_ctx_t ctx, int32_t method) {
    if (!ctx || method < 0 || method > 2) return RICH_ERR_INVALID;
    ctx->adj_method = method;
    return 0;
}

extern "C" int rich_set_adjoint_limits(rich_ctx_t ctx, double rel_tol, int32_t max_applications) {
    if (!ctx || !(rel_tol > 0.0 && rel_tol < 1.0) || max_applications < 1 || max_applications > 1000000)
        return RICH_ERR_INVALID;
    ctx->adj_tol = rel_tol;
    ctx->adj_cap = max_applications;
    return 0;
}
