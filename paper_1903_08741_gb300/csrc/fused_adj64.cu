// FP64 instantiations of the discrete-adjoint kernel (V-cycle and
// cycle-index-gamma preconditioners), in a translation unit of their own so
// that they compile in parallel with the rest of the library.
#include "fused_adjoint.cuh"

namespace rich_fused {

const void* rich_adjoint_kernel64(bool wcycle) {
    return wcycle ? (const void*)k_adjoint<double, true> : (const void*)k_adjoint<double, false>;
}

void rich_adjoint_launch64(const FParams& P, int grid, size_t smem, cudaStream_t st) {
    if (P.gamma > 1) k_adjoint<double, true><<<grid, 512, smem, st>>>(P);
    else k_adjoint<double, false><<<grid, 512, smem, st>>>(P);
}

}  // namespace rich_fused
