// FP64, van Genuchten-Mualem (closure 1: Sec. 2.1, Eqs. Sw, sc_van, Krw) instantiations of the persistent fused solver, in a
// translation unit of their own so that the instantiations compile in parallel.
#include "fused_kernel.cuh"

namespace rich_fused {

int rich_occ_vg64(const FParams& P, size_t smem, int nt, int* occ) {
    return occ_shapes<double, 1>(P, smem, nt, occ);
}

void rich_launch_vg64(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st) {
    launch_shapes<double, 1>(P, grid, smem, nt, st);
}

}  // namespace rich_fused
