// Mixed-precision (FP32 cycles), Gardner-closure instantiations of the persistent fused solver, in a
// translation unit of their own so that the instantiations compile in parallel.
#include "fused_kernel.cuh"

namespace rich_fused {

int rich_occ_g32(const FParams& P, size_t smem, int nt, int* occ) {
    return occ_shapes<float, 0>(P, smem, nt, occ);
}

void rich_launch_g32(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st) {
    launch_shapes<float, 0>(P, grid, smem, nt, st);
}

}  // namespace rich_fused
