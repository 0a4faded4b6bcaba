// FP64 accumulation of MC / MLMC level statistics on the device
// (arXiv 1903.08741, Sec. 5: Eqs. SMC_ch6, MC_var_ch6, ML_var_ch6).
#include "rich_internal.cuh"

namespace {

constexpr int ACC_TPB = 1024;

// One block, fixed summation order (strided per-thread sums, then a fixed
// tree), so that repeated calls give bit-identical sums.  Sample i counts when
// both statuses are RICH_OK or RICH_MG_MAXIT (the QoI is defined); failed
// samples are counted separately and excluded from the sums.
__global__ void __launch_bounds__(ACC_TPB)
k_accumulate(int n, const double* __restrict__ qf, const double* __restrict__ qc,
             const int32_t* __restrict__ sf, const int32_t* __restrict__ sc, double* acc) {
    double v[7] = {0, 0, 0, 0, 0, 0, 0};   // sum Y, sum Y^2, count, sum Qf, sum Qf^2, sum Qc, sum Qc^2
    double nfail = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        bool bad = (sf && (sf[i] == RICH_PICARD_MAXIT || sf[i] == RICH_NONFINITE)) ||
                   (qc && sc && (sc[i] == RICH_PICARD_MAXIT || sc[i] == RICH_NONFINITE));
        double f = qf[i], c = qc ? qc[i] : 0.0;
        if (bad || !isfinite(f) || !isfinite(c)) { nfail += 1; continue; }
        double y = f - c;
        v[0] += y; v[1] += y * y; v[2] += 1;
        v[3] += f; v[4] += f * f; v[5] += c; v[6] += c * c;
    }
    __shared__ double sm[8][ACC_TPB];
    for (int k = 0; k < 7; ++k) sm[k][threadIdx.x] = v[k];
    sm[7][threadIdx.x] = nfail;
    __syncthreads();
    for (int w = ACC_TPB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + w];
        __syncthreads();
    }
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
                                                         status_coarse, acc);
    RICH_CUDA(cudaGetLastError());
    return 0;
}
