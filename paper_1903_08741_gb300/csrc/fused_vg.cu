// van Genuchten-Mualem instantiations of the persistent fused solver (closure
// 1: Sec. 2.1, Eqs. Sw, sc_van, Krw), in a translation unit of their own so
// that the two closures' kernels compile in parallel.
#include "fused_kernel.cuh"

namespace {

template <int NT, bool WC>
int occ_vg(const FParams& P, size_t smem, int* occ) {
    if (P.mixed) {
        if (int e = allow_dyn_smem((const void*)k_fused<float, NT, WC, 1>, smem)) return e;
        RICH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_fused<float, NT, WC, 1>, NT, smem));
    } else {
        if (int e = allow_dyn_smem((const void*)k_fused<double, NT, WC, 1>, smem)) return e;
        RICH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_fused<double, NT, WC, 1>, NT, smem));
    }
    if (*occ < 1) *occ = 1;
    return 0;
}

template <int NT, bool WC>
void launch_vg(const FParams& P, int grid, size_t smem, cudaStream_t st) {
    if (P.mixed) k_fused<float, NT, WC, 1><<<grid, NT, smem, st>>>(P);
    else k_fused<double, NT, WC, 1><<<grid, NT, smem, st>>>(P);
}

}  // namespace

namespace rich_fused {

int rich_vg_occupancy(const FParams& P, size_t smem, int nt, int* occ) {
    const bool wc = P.gamma > 1;
    if (nt == 1024) return wc ? occ_vg<1024, true>(P, smem, occ) : occ_vg<1024, false>(P, smem, occ);
    if (nt == 256) return wc ? occ_vg<256, true>(P, smem, occ) : occ_vg<256, false>(P, smem, occ);
    return wc ? occ_vg<512, true>(P, smem, occ) : occ_vg<512, false>(P, smem, occ);
}

void rich_vg_launch(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st) {
    const bool wc = P.gamma > 1;
    if (nt == 1024) { if (wc) launch_vg<1024, true>(P, grid, smem, st); else launch_vg<1024, false>(P, grid, smem, st); }
    else if (nt == 256) { if (wc) launch_vg<256, true>(P, grid, smem, st); else launch_vg<256, false>(P, grid, smem, st); }
    else if (wc) launch_vg<512, true>(P, grid, smem, st);
    else launch_vg<512, false>(P, grid, smem, st);
}

}  // namespace rich_fused
