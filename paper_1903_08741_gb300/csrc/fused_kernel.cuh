// Device side of the persistent fused solver (kernel templates), shared by
// the translation units that instantiate them.
//
// Each CTA takes samples from an atomic queue and runs, for its sample, the
// complete method of arXiv 1903.08741 Sec. 4: backward-Euler time loop,
// modified Picard iteration on the mixed form (Eq. Mixed_based_3), and for
// every Picard step the cell-centred multigrid solve (five-point harmonic-mean
// stencil, Eq. five_stencil; red-black Gauss-Seidel; 1/4-sum restriction and
// piecewise-constant prolongation, Eq. transfer; coarse operators by
// rediscretisation with arithmetic means of face coefficients, Fig.
// diffUpscale; exact coarsest solve).  All control flow is per CTA and uniform
// (decisions come from block-wide reductions), so a sample never waits for
// another and there is no host round trip inside a solve.
//
// Memory: every CTA owns one scratch slot holding its sample's hierarchy; the
// slots of the resident CTAs are largely L2 (small grids: L1) resident.
// Scratch arrays are read with plain loads (they are rewritten inside the
// kernel; __syncthreads orders the accesses).
//
// Precision and instruction budget.  GB300 issues 2 FP64 FMAs per SM and
// clock (1/64 of its FP32 rate), so the FP64 V-cycle is written to minimise
// FP64 instructions:
//   * every level stores the Jacobi-scaled coefficients w = T/D of its four
//     faces and the scaled right-hand side f/D, so a Gauss-Seidel update is
//     dp_P = f_P/D_P + sum w dp_nb (4 FMAs instead of 6 operations);
//   * after a black half-sweep the black residuals are zero up to rounding
//     (each black value was just solved from its red neighbours), so the
//     restriction after pre-smoothing and the stopping norm after
//     post-smoothing evaluate red cells only (exactly the same quantities in
//     exact arithmetic; full evaluation when nu = 0);
//   * divisions by dt are multiplications by 1/dt.
// TM = double is the FP64 path (the oracle's algorithm and stopping tests);
// TM = float runs FP32 V-cycles (unscaled coefficients: FP32 operations are
// cheap, bytes are not) inside an FP64 defect-correction loop that performs
// a tunable number of V-cycles per FP64 defect (FP64 Picard residual, FP64
// outer residual, FP64 correction and stopping norm).

#pragma once
#include "rich_internal.cuh"
#include <math.h>
#include <type_traits>

// launch parameters and slot layout, shared across translation units
namespace rich_fused {

constexpr unsigned long long ABS_MASK = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long INF_BITS = 0x7FF0000000000000ull;
constexpr int MAXL = RICH_MAX_LEVELS;
constexpr int MIXED_INNER_DEFAULT = 2;   // FP32 V-cycles per FP64 defect evaluation
constexpr int ADJ_M = 12;                // GMRES restart length of the adjoint's J^T solves

// FP64 unscaled operator (all levels): faces, mass term, diagonal, Dirichlet faces
enum { A_TX, A_TZ, A_CDT, A_D, A_TBT, A_TBB, N64 };
// multigrid arrays in the cycle precision, colour-split on every level but
// the coarsest.  FP64: wE wW wN wS q=1/D fh dp D.  FP32: Tx Tz - D 1/D f dp -.
enum { B_0, B_1, B_2, B_3, B_4, B_5, B_6, B_7, NMG };

struct FParams {
    int S, nlev, mixed;
    int nx[MAXL], nz[MAXL];
    unsigned mnx[MAXL], mhx[MAXL];          // magic reciprocals of nx and nx/2
    long long o64[MAXL][N64];               // byte offsets in the slot (-1: absent)
    long long omg[MAXL][NMG];
    long long osm[MAXL];                    // level's dp in dynamic shared memory at this
                                            // byte offset (-1: in the slot)
    int lw;                                 // first level run by warp 0 alone (nlev: none)
    long long s64[MAXL][N64];               // levels >= lw: every array in dynamic shared
    long long smg[MAXL][NMG];               // memory at these byte offsets (-1: not there)
    long long smem_bytes;                   // dynamic shared memory of a CTA
    long long o_f64, o_dp64, o_p, o_thold, o_Ks, o_a, o_K, o_th;
    long long slot_bytes;
    char* scratch;
    const double* lnKs;
    const double* alpha;
    double alpha_scale;
    double* qoi;
    double* p_final;
    int32_t* status;
    int64_t* pic_total;
    int64_t* mg_total;
    int64_t* t_ns;                          // per-sample solve time on its CTA (ns; may be null)
    int32_t* maxpic;
    int* queue;
    int nsteps, picard_maxit, mg_maxit, nu1, nu2, gamma;
    double inv_dt, tr, ts, p_top, p_bot, p_init, picard_tol, mg_tol, h, two_over_h2;
    // adjoint (k_adjoint only)
    int mixed_inner;            // FP32 V-cycles per FP64 defect (mixed path)
    int ckpt_every, adj_maxit, adj_inner;
    double adj_tol;
    long long o_ckpt, o_seg, o_lam, o_rhs, o_r, o_dE, o_dW, o_dN, o_dS, o_dg, o_g;
    int adj_method;             // J^T solver: 0 defect correction, 1 BiCGStab, 2 GMRES(ADJ_M)
    long long o_rh, o_pk, o_v, o_t, o_ph, o_sh;   // BiCGStab vectors
    long long o_kry;                              // GMRES: ADJ_M + 1 Krylov and ADJ_M preconditioned vectors
    double* g_out;
    // closure 1 (van Genuchten-Mualem): per-cell n, theta_s, theta_r inputs
    // (theta arrays may be null: the problem's constants), continuation
    // shifts, and the slot arrays n, m = 1 - 1/n, theta_r, theta_s
    int closure;
    double alpha_shift, n_shift, init_decay;
    const double* n_in;
    const double* ts_in;
    const double* tr_in;
    long long o_n, o_m, o_trc, o_tsc;
};

// allow a kernel `bytes` of dynamic shared memory above the 48 KB default; the
// attribute is set once per (kernel, device, larger size)
inline int allow_dyn_smem(const void* kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return 0;
    struct Grant { const void* k; int dev; size_t bytes; };
    static Grant grants[128];
    static int ngrants = 0;
    int dev = 0;
    RICH_CUDA(cudaGetDevice(&dev));
    int i = 0;
    while (i < ngrants && !(grants[i].k == kernel && grants[i].dev == dev)) ++i;
    if (i < ngrants && grants[i].bytes >= bytes) return 0;
    RICH_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (i == ngrants && ngrants < 128) ++ngrants;
    if (i < 128) grants[i] = Grant{kernel, dev, bytes};
    return 0;
}

// Occupancy query and launch of the fused kernel's instantiations, one
// translation unit per (cycle precision, closure) so that they compile in
// parallel: fused_g64.cu (FP64, Gardner), fused_g32.cu (mixed, Gardner),
// fused_vg64.cu, fused_vg32.cu (van Genuchten-Mualem).
int rich_occ_g64(const FParams& P, size_t smem, int nt, int* occ);
int rich_occ_g32(const FParams& P, size_t smem, int nt, int* occ);
int rich_occ_vg64(const FParams& P, size_t smem, int nt, int* occ);
int rich_occ_vg32(const FParams& P, size_t smem, int nt, int* occ);
void rich_launch_g64(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st);
void rich_launch_g32(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st);
void rich_launch_vg64(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st);
void rich_launch_vg32(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st);
// the adjoint kernel's instantiations (fused_adj64.cu, fused_adj32.cu): the
// kernel's address (occupancy queries) and its launch with 512 threads
const void* rich_adjoint_kernel64(bool wcycle);
const void* rich_adjoint_kernel32(bool wcycle);
void rich_adjoint_launch64(const FParams& P, int grid, size_t smem, cudaStream_t st);
void rich_adjoint_launch32(const FParams& P, int grid, size_t smem, cudaStream_t st);

}  // namespace rich_fused

namespace {
using namespace rich_fused;

// c / d for c * d < 2^32 (m = floor(2^32 / d) + 1), d = 1 handled apart
__device__ __forceinline__ int fdiv(int c, int d, unsigned m) {
    return d == 1 ? c : (int)__umulhi((unsigned)c, m);
}

// the GPU's global nanosecond timer (per-sample solve times)
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & ABS_MASK;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// block-wide sum of v in a fixed order (warp trees, then the warp partials in
// warp order), returned to every thread
__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    const double r = red[32];
    __syncthreads();
    return r;
}

// block-wide max of v, returned to every thread
__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max_u64(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? red[lane] : 0ull;
        v = warp_max_u64(v);
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    unsigned long long r = red[32];
    __syncthreads();
    return r;
}

struct Lv64 {
    int nx, nz, nc;
    unsigned mnx;
    double *Tx, *Tz, *Cdt, *D, *Tbt, *Tbb;
};

// multigrid level in cycle precision T.  FP64 (scaled): c = {wE, wW, wN, wS},
// q = 1/D, f = f/D (the coarsest level keeps f unscaled for the direct solve).
// FP32 (unscaled): c = {Tx, Tz, -, -}, q = 1/D, f = f.
// Layout: every level that is smoothed stores its cells colour-split, the red
// cells ((i + j) even) first and then the black ones, each half row-major with
// hx = nx/2 cells per row: cell (i, j) sits at ((i + j) & 1) H + j hx + i/2
// (H = hx nz).  A half-sweep then reads its own cells, and the neighbours of
// the other colour, at unit stride (no shared-memory bank conflicts, full
// sectors from L2).  The coarsest level (direct solve; its sides may be odd)
// keeps the natural row-major order (H = 0).
template <typename T>
struct Lv {
    int nx, nz, hx, nc, H;
    unsigned mnx, mhx;
    T *c0, *c1, *c2, *c3, *D, *q, *f, *dp;
};

// storage index of cell (i, j) on a level
template <typename T>
__device__ __forceinline__ int sidx(const Lv<T>& L, int i, int j) {
    return L.H ? ((i + j) & 1) * L.H + j * L.hx + (i >> 1) : j * L.nx + i;
}

// storage indices of cell (i, j) and of its east, west, north and south
// neighbours (valid where the neighbour exists)
struct Nb { int own, e, w, n, s; };
template <typename T>
__device__ __forceinline__ Nb nb_of(const Lv<T>& L, int i, int j) {
    if (L.H) {
        const int col = (i + j) & 1, c = j * L.hx + (i >> 1), oth = (1 - col) * L.H + c;
        return Nb{col * L.H + c, oth + (i & 1), oth - 1 + (i & 1), oth + L.hx, oth - L.hx};
    }
    const int P = j * L.nx + i;
    return Nb{P, P + 1, P - 1, P + L.nx, P - L.nx};
}

template <typename T> struct Scaled { static constexpr bool value = sizeof(T) == 8; };

// Thread groups that run a level's loops: the whole CTA (barrier
// __syncthreads), or warp 0 alone (barrier __syncwarp) on the small coarse
// levels, whose few hundred cells do not pay for CTA-wide barriers; those
// levels keep every array in shared memory.  Each level function ends with
// its group synchronised.
struct GCta {
    static __device__ __forceinline__ int rank() { return threadIdx.x; }
    static __device__ __forceinline__ int size() { return blockDim.x; }
    static __device__ __forceinline__ void sync() { __syncthreads(); }
};
struct GWarp {
    static __device__ __forceinline__ int rank() { return threadIdx.x & 31; }
    static __device__ __forceinline__ int size() { return 32; }
    static __device__ __forceinline__ void sync() { __syncwarp(); }
};

// Gauss-Seidel value of a cell (storage indices b) from its current
// neighbours, with the level's arrays passed as restrict-qualified pointers:
// every caller reads dp only at cells that it does not write in the same pass
// (see rbgs_cells), so the compiler may keep several cells' loads in flight
// ahead of the stores.
//   FP64 (scaled): c0..c3 = wE, wW, wN, wS; value f + sum w dp_nb.
//   FP32 (unscaled): c0 = Tx (east face), c1 = Tz (north face); the west and
//   south faces are the neighbours'; value (f + sum T dp_nb) / D.
template <typename T>
__device__ __forceinline__ T gs_at(const Nb& b, bool hE, bool hW, bool hN, bool hS, const T* __restrict__ f,
                                   const T* __restrict__ c0, const T* __restrict__ c1,
                                   const T* __restrict__ c2, const T* __restrict__ c3,
                                   const T* __restrict__ q, const T* __restrict__ dp) {
    if constexpr (Scaled<T>::value) {
        T v = f[b.own];
        if (hE) v += c0[b.own] * dp[b.e];
        if (hW) v += c1[b.own] * dp[b.w];
        if (hN) v += c2[b.own] * dp[b.n];
        if (hS) v += c3[b.own] * dp[b.s];
        return v;
    } else {
        T t = T(0);
        if (hE) t += c0[b.own] * dp[b.e];
        if (hW) t += c0[b.w] * dp[b.w];
        if (hN) t += c1[b.own] * dp[b.n];
        if (hS) t += c1[b.s] * dp[b.s];
        return (f[b.own] + t) * q[b.own];
    }
}

// residual f - A dp at a cell (unscaled): FP64 D (value - dp), FP32
// f - (D dp - sum T dp_nb)
template <typename T>
__device__ __forceinline__ T resid_at(const Nb& b, bool hE, bool hW, bool hN, bool hS,
                                      const T* __restrict__ f, const T* __restrict__ c0,
                                      const T* __restrict__ c1, const T* __restrict__ c2,
                                      const T* __restrict__ c3, const T* __restrict__ q,
                                      const T* __restrict__ D, const T* __restrict__ dp) {
    if constexpr (Scaled<T>::value) {
        return D[b.own] * (gs_at<T>(b, hE, hW, hN, hS, f, c0, c1, c2, c3, q, dp) - dp[b.own]);
    } else {
        T t = T(0);
        if (hE) t += c0[b.own] * dp[b.e];
        if (hW) t += c0[b.w] * dp[b.w];
        if (hN) t += c1[b.own] * dp[b.n];
        if (hS) t += c1[b.s] * dp[b.s];
        return f[b.own] - (D[b.own] * dp[b.own] - t);
    }
}

template <typename T>
__device__ __forceinline__ T resid_cell(const Lv<T>& L, int i, int j) {
    return resid_at<T>(nb_of(L, i, j), i < L.nx - 1, i > 0, j < L.nz - 1, j > 0, L.f, L.c0, L.c1, L.c2, L.c3,
                       L.q, L.D, L.dp);
}

// one colour of red-black Gauss-Seidel over a colour-split level (red:
// i + j even).  The corrections are read through one restrict-qualified view
// and written through another: a half-sweep writes cells of one colour and
// reads only cells of the other, so the two views never touch one element.
template <typename T, typename G>
__device__ __forceinline__ void rbgs_cells(int nx, int nz, int hx, int H, unsigned mhx, int colour,
                                           const T* __restrict__ f, const T* __restrict__ c0,
                                           const T* __restrict__ c1, const T* __restrict__ c2,
                                           const T* __restrict__ c3, const T* __restrict__ q,
                                           const T* __restrict__ dpr, T* __restrict__ dpw) {
#pragma unroll 4
    for (int c = G::rank(); c < H; c += G::size()) {
        const int j = fdiv(c, hx, mhx);
        const int i = 2 * (c - j * hx) + ((j + colour) & 1);
        const int oth = (1 - colour) * H + c;
        const Nb b{colour * H + c, oth + (i & 1), oth - 1 + (i & 1), oth + hx, oth - hx};
        dpw[b.own] = gs_at<T>(b, i < nx - 1, i > 0, j < nz - 1, j > 0, f, c0, c1, c2, c3, q, dpr);
    }
    G::sync();
}

template <typename T, typename G>
__device__ __forceinline__ void rbgs(const Lv<T>& L, int colour) {
    rbgs_cells<T, G>(L.nx, L.nz, L.hx, L.H, L.mhx, colour, L.f, L.c0, L.c1, L.c2, L.c3, L.q, L.dp, L.dp);
}

template <typename T, typename G>
__device__ __forceinline__ void prolong(const Lv<T>& F, const Lv<T>& C);

// nu red-black sweeps; with seeded true the first red half-sweep is skipped
// because the restriction already stored its result (see restrict_cells)
template <typename T, typename G>
__device__ __forceinline__ void smooth(const Lv<T>& L, int nu, bool seeded = false) {
    for (int it = 0; it < nu; ++it) {
        if (!(seeded && it == 0)) rbgs<T, G>(L, 0);
        rbgs<T, G>(L, 1);
    }
}

// prolongation and post-smoothing of level l from level l+1
template <typename T, typename G>
__device__ __forceinline__ void prolong_smooth(const Lv<T>& F, const Lv<T>& C, int nu2) {
    prolong<T, G>(F, C);
    smooth<T, G>(F, nu2);
}

// restricted residual (Eq. transfer, R = 1/4 sum of the children); after a
// black half-sweep only the two red children carry a residual.  Reads the
// fine level, writes the coarse one (distinct arrays: restrict views).  The
// fine level is colour-split: the children of coarse cell (I, J) are the red
// cells r0 = 2J hx + I and r0 + hx and the black cells H + r0, H + r0 + hx.
// The coarse correction starts at zero; when the coarse level is smoothed
// next (seed), its red cells get at once the value the first red half-sweep
// would compute from all-zero neighbours, f q (FP64: the scaled f), so that
// half-sweep is skipped.
template <typename T, typename G>
__device__ __forceinline__ void restrict_cells(const Lv<T>& F, const Lv<T>& C, bool red_only, bool scale, bool seed,
                                               const T* __restrict__ f, const T* __restrict__ c0,
                                               const T* __restrict__ c1, const T* __restrict__ c2,
                                               const T* __restrict__ c3, const T* __restrict__ q,
                                               const T* __restrict__ D, const T* __restrict__ dp,
                                               const T* __restrict__ cq, T* __restrict__ cf, T* __restrict__ cdp) {
    const int nx = F.nx, nz = F.nz, hx = F.hx, H = F.H;
#pragma unroll(Scaled<T>::value ? 1 : 2)
    for (int c = G::rank(); c < C.nc; c += G::size()) {
        const int J = fdiv(c, C.nx, C.mnx), I = c - J * C.nx;
        const int i = 2 * I, j = 2 * J, r0 = j * hx + I;
        // red (i, j): neighbours black; red (i+1, j+1) likewise
        const Nb b00{r0, H + r0, H + r0 - 1, H + r0 + hx, H + r0 - hx};
        const Nb b11{r0 + hx, H + r0 + hx + 1, H + r0 + hx, H + r0 + 2 * hx, H + r0};
        const T r00 = resid_at<T>(b00, true, i > 0, true, j > 0, f, c0, c1, c2, c3, q, D, dp);
        const T r11 = resid_at<T>(b11, i + 1 < nx - 1, true, j + 1 < nz - 1, true, f, c0, c1, c2, c3, q, D, dp);
        T sum;
        if (red_only) {
            sum = r00 + r11;
        } else {
            const Nb b10{H + r0, r0 + 1, r0, r0 + hx, r0 - hx};
            const Nb b01{H + r0 + hx, r0 + hx, r0 + hx - 1, r0 + 2 * hx, r0};
            const T r10 = resid_at<T>(b10, i + 1 < nx - 1, true, true, j > 0, f, c0, c1, c2, c3, q, D, dp);
            const T r01 = resid_at<T>(b01, true, i > 0, j + 1 < nz - 1, true, f, c0, c1, c2, c3, q, D, dp);
            sum = r00 + r10 + r01 + r11;
        }
        const int cs = sidx(C, I, J);
        T fc = T(0.25) * sum;
        if (scale) fc *= cq[cs];
        cf[cs] = fc;
        T d0 = T(0);
        if (seed && !((I + J) & 1)) {
            if constexpr (Scaled<T>::value) d0 = fc;
            else d0 = fc * cq[cs];
        }
        cdp[cs] = d0;
    }
    G::sync();
}

template <typename T, typename G>
__device__ __forceinline__ void resid_restrict(const Lv<T>& F, const Lv<T>& C, bool red_only, bool coarsest,
                                               bool seed = false) {
    restrict_cells<T, G>(F, C, red_only, Scaled<T>::value && !coarsest, seed && !coarsest, F.f, F.c0, F.c1, F.c2,
                         F.c3, F.q, F.D, F.dp, C.q, C.f, C.dp);
}

// piecewise-constant prolongation and correction: each coarse cell adds its
// value to its own four children, so no two iterations touch one element
template <typename T, typename G>
__device__ __forceinline__ void prolong(const Lv<T>& F, const Lv<T>& C) {
    const T* __restrict__ e = C.dp;
    T* __restrict__ d = F.dp;
    const int hx = F.hx, H = F.H;
#pragma unroll 2
    for (int c = G::rank(); c < C.nc; c += G::size()) {
        const int J = fdiv(c, C.nx, C.mnx), I = c - J * C.nx;
        const T v = e[sidx(C, I, J)];
        const int r0 = 2 * J * hx + I;
        d[r0] += v; d[r0 + hx] += v; d[H + r0] += v; d[H + r0 + hx] += v;
    }
    G::sync();
}

// exact coarsest solve: Gaussian elimination of the assembled five-point
// matrix by one warp in shared memory (symmetric, diagonally dominant); run
// by warp 0 only, synchronised with __syncwarp
template <typename T>
__device__ __forceinline__ void coarse_solve_warp(int nx, int nz, const T* Tx, const T* Tz, const T* D,
                                                  const T* f, T* dp, T* A) {
    const int nn = nx * nz, ld = nn + 1, lane = threadIdx.x & 31;
    for (int r = lane; r < nn; r += 32) {
        for (int c = 0; c < nn; ++c) A[r * ld + c] = T(0);
        int j = r / nx, i = r - j * nx;
        A[r * ld + r] = D[r];
        if (i < nx - 1) A[r * ld + r + 1] = -Tx[r];
        if (i > 0)      A[r * ld + r - 1] = -Tx[r - 1];
        if (j < nz - 1) A[r * ld + r + nx] = -Tz[r];
        if (j > 0)      A[r * ld + r - nx] = -Tz[r - nx];
        A[r * ld + nn] = f[r];
    }
    __syncwarp();
    for (int k = 0; k < nn; ++k) {
        for (int r = k + 1 + lane; r < nn; r += 32) {
            T m = A[r * ld + k] / A[k * ld + k];
            for (int c = k; c <= nn; ++c) A[r * ld + c] -= m * A[k * ld + c];
        }
        __syncwarp();
    }
    if (lane == 0) {
        for (int k = nn - 1; k >= 0; --k) {
            T sum = A[k * ld + nn];
            for (int c = k + 1; c < nn; ++c) sum -= A[k * ld + c] * A[c * ld + nn];
            A[k * ld + nn] = sum / A[k * ld + k];
        }
    }
    __syncwarp();
    for (int r = lane; r < nn; r += 32) dp[r] = A[r * ld + nn];
    __syncwarp();
}

// exact solve on the coarsest level c (FP64 levels: the unscaled FP64
// operator; f0 is the unscaled right-hand side when c is the finest level),
// by warp 0; the CTA group waits for it at a barrier
template <typename T, typename G>
__device__ __forceinline__ void coarsest(const Lv<T>* L, const Lv64* L64, int c, T* A, const T* f0) {
    if (threadIdx.x < 32) {
        if constexpr (Scaled<T>::value)
            coarse_solve_warp<T>(L64[c].nx, L64[c].nz, L64[c].Tx, L64[c].Tz, L64[c].D, c == 0 ? f0 : L[c].f,
                                 L[c].dp, A);
        else
            coarse_solve_warp<T>(L[c].nx, L[c].nz, L[c].c0, L[c].c1, L[c].D, L[c].f, L[c].dp, A);
    }
    if constexpr (std::is_same<G, GCta>::value) __syncthreads();
}

// One multigrid cycle rooted at level `root`: V-cycle for gamma = 1, else the
// cycle of index gamma (W-cycle for gamma = 2, the paper's cycle, Sec. 4.2):
// every visit of level l < nlev-2 runs gamma cycles on level l+1, the visit
// of nlev-2 one exact coarsest solve.  The recursion is unrolled into a
// depth-first walk whose per-level visit counts sit in 4-bit fields of one
// register (no device stack).  Run by the CTA, each visit of level lw (the
// first small level) is handed to warp 0 as a complete cycle rooted at lw.
// A level entered right after the restriction into it (fresh) skips its
// first red half-sweep, which the restriction seeded; a level cycled again
// (gamma > 1) starts from its previous correction and smooths in full.
template <typename T, typename G>
__device__ __forceinline__ void gwalk(const Lv<T>* L, const Lv64* L64, int root, int nlev, int lw, int nu1, int nu2,
                                      int gamma, T* A, const T* f0, bool root_fresh) {
    static_assert(RICH_MAX_LEVELS * 4 <= 64, "visit counters must fit one 64-bit word");
    unsigned long long cnt = 0;
    int l = root;
    bool fresh = root_fresh;
    const bool seed = nu1 > 0;
    for (;;) {
        for (; l < nlev - 1 && l != lw; ++l) {            // enter l: pre-smooth, restrict
            smooth<T, G>(L[l], nu1, fresh && seed);
            resid_restrict<T, G>(L[l], L[l + 1], nu1 > 0, l + 1 == nlev - 1, seed);
            cnt &= ~(15ull << (4 * l));
            fresh = true;
        }
        if constexpr (std::is_same<G, GCta>::value) {
            if (l == lw && lw < nlev - 1) {
                if (threadIdx.x < 32)
                    gwalk<T, GWarp>(L, L64, lw, nlev, nlev, nu1, nu2, gamma, A, f0, fresh && seed);
                __syncthreads();
            } else {
                coarsest<T, G>(L, L64, nlev - 1, A, f0);
            }
        } else {
            coarsest<T, G>(L, L64, nlev - 1, A, f0);
        }
        for (;;) {                                        // leave l+1, back on l
            if (--l < root) return;
            cnt += 1ull << (4 * l);
            const int reps = (l + 1 == nlev - 1) ? 1 : gamma;
            if ((int)((cnt >> (4 * l)) & 15) < reps) { ++l; fresh = false; break; }   // cycle l+1 again
            prolong_smooth<T, G>(L[l], L[l + 1], nu2);
        }
    }
}

// V-cycle with the levels from lw down handed to warp 0 (lw = nlev: none);
// every level below the finest is fresh (seeded by its restriction)
template <typename T>
__device__ __forceinline__ void vcycle(const Lv<T>* L, const Lv64* L64, int nlev, int lw, int nu1, int nu2, T* A,
                                       const T* f0) {
    const bool seed = nu1 > 0;
    const int top = min(lw, nlev - 1);       // levels 0 .. top-1 run on the whole CTA
    for (int l = 0; l < top; ++l) {
        smooth<T, GCta>(L[l], nu1, l > 0 && seed);
        resid_restrict<T, GCta>(L[l], L[l + 1], nu1 > 0, l + 1 == nlev - 1, seed);
    }
    if (lw < nlev - 1) {
        if (threadIdx.x < 32) {
            for (int l = lw; l < nlev - 1; ++l) {
                smooth<T, GWarp>(L[l], nu1, seed);
                resid_restrict<T, GWarp>(L[l], L[l + 1], nu1 > 0, l + 1 == nlev - 1, seed);
            }
            coarsest<T, GWarp>(L, L64, nlev - 1, A, f0);
            for (int l = nlev - 2; l >= lw; --l) prolong_smooth<T, GWarp>(L[l], L[l + 1], nu2);
        }
        __syncthreads();
    } else {
        coarsest<T, GCta>(L, L64, nlev - 1, A, f0);
    }
    for (int l = top - 1; l >= 0; --l) prolong_smooth<T, GCta>(L[l], L[l + 1], nu2);
}

// ||f - A dp||_inf on a level after a cycle ending with a black half-sweep
// (red cells only) or, with red_only false, over every cell
template <typename T>
__device__ __forceinline__ unsigned long long resid_norm(const Lv<T>& L, bool red_only,
                                                         unsigned long long* red) {
    unsigned long long m = 0;
    if (red_only) {
        const int n = L.hx * L.nz;
#pragma unroll 2
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            const int j = fdiv(c, L.hx, L.mhx);
            const int i = 2 * (c - j * L.hx) + (j & 1);
            const unsigned long long b = abs_bits((double)resid_cell(L, i, j));
            m = b > m ? b : m;
        }
    } else {
        for (int c = threadIdx.x; c < L.nc; c += blockDim.x) {
            const int j = fdiv(c, L.nx, L.mnx), i = c - j * L.nx;
            const unsigned long long b = abs_bits((double)resid_cell(L, i, j));
            m = b > m ? b : m;
        }
    }
    return block_max(m, red);
}

// van Genuchten-Mualem closure at p < 0 (Eqs. Sw, sc_van, Krw) with
// m = 1 - 1/n and an = (a|p|)^n: S = (1 + an)^-m, K_rw = S^(1/2) (1 - (an /
// (1 + an))^m)^2 (1 - S^(1/m) = an/(1 + an) exactly) and dS/dp = m n S an /
// ((1 + an) |p|), the Eq. sc_van capacity divided by theta_s - theta_r.  In
// logarithms: an = exp(n log(a|p|)), S = exp(-m log1p(an)), and since
// m n = n - 1, (an / (1 + an))^m = an^m S = (an / (a|p|)) S: one exp fewer
// than exp(m (n log(a|p|) - log1p(an))), and no cancellation between the two
// logarithms in the dry limit.
__device__ __forceinline__ double vg_sat(double a, double n, double m, double p) {
    return exp(-m * log1p(exp(n * log(-a * p))));
}

__device__ __forceinline__ void vg_eval(double a, double n, double m, double p, double& S, double& krw,
                                        double& dS) {
    const double ap = -a * p;
    const double an = exp(n * log(ap));
    const double l1 = log1p(an);
    S = exp(-m * l1);
    const double b = 1.0 - S * (an / ap);
    krw = sqrt(S) * b * b;
    dS = m * n * S * an / ((1.0 + an) * (-p));
}

// CTA-cooperative building blocks of one sample's solve.  Every method is
// called by all threads of the CTA and ends with the CTA synchronised.
template <typename TM, bool WC = false, int CL = 0>
struct Cta {
    static constexpr bool SC = Scaled<TM>::value;
    const FParams& P;
    Lv64* L64;
    Lv<TM>* LM;
    TM* Amat;
    unsigned long long* red;
    double *f64, *dp64, *p, *thold, *Ks, *aa, *K, *th;
    double *nn, *mm, *trc, *tsc;          // closure 1: per-cell n, m, theta_r, theta_s
    int nx, nz, nc, nlev, tid, nt;
    double h, t2h, idt, tr, ts;

    __device__ Cta(const FParams& P_, char* slot, Lv64* l64, Lv<TM>* lm, TM* A, unsigned long long* r)
        : P(P_), L64(l64), LM(lm), Amat(A), red(r) {
        f64 = (double*)(slot + P.o_f64);
        dp64 = SC ? (double*)LM[0].dp : (double*)(slot + P.o_dp64);
        p = (double*)(slot + P.o_p);
        thold = (double*)(slot + P.o_thold);
        Ks = (double*)(slot + P.o_Ks);
        aa = (double*)(slot + P.o_a);
        K = (double*)(slot + P.o_K);
        th = (double*)(slot + P.o_th);
        if constexpr (CL == 1) {
            nn = (double*)(slot + P.o_n); mm = (double*)(slot + P.o_m);
            trc = (double*)(slot + P.o_trc); tsc = (double*)(slot + P.o_tsc);
        } else {
            nn = mm = trc = tsc = nullptr;
        }
        nx = L64[0].nx; nz = L64[0].nz; nc = L64[0].nc; nlev = P.nlev;
        tid = threadIdx.x; nt = blockDim.x;
        h = P.h; t2h = P.two_over_h2; idt = P.inv_dt; tr = P.tr; ts = P.ts;
    }

    // conductivity of cell q's soil at head pp (Dirichlet faces, QoI)
    __device__ __forceinline__ double k_at(int q, double pp) const {
        if constexpr (CL == 0) {
            return pp < 0.0 ? Ks[q] * exp(aa[q] * pp) : Ks[q];
        } else {
            if (!(pp < 0.0)) return Ks[q];
            double S, krw, dS;
            vg_eval(aa[q], nn[q], mm[q], pp, S, krw, dS);
            return Ks[q] * krw;
        }
    }

    // Ks, alpha * scale + shift, (closure 1: n + shift, m, theta_r, theta_s),
    // initial head (uniform, or p_init (1 - exp(-init_decay z)) at the cell
    // centres, Eq. travellingwave), Dirichlet faces (fixed for the solve)
    __device__ void setup(int s) {
        const Lv64& F = L64[0];
        const size_t o = (size_t)s * nc;
        const double* lk = P.lnKs + o;
        const double* al = P.alpha + o;
        for (int q = tid; q < nc; q += nt) {
            Ks[q] = exp(lk[q]);
            aa[q] = al[q] * P.alpha_scale + P.alpha_shift;
            if (P.init_decay > 0.0) {
                const int j = fdiv(q, nx, F.mnx);
                p[q] = P.p_init * (1.0 - exp(-P.init_decay * (j + 0.5) * h));
            } else {
                p[q] = P.p_init;
            }
            if constexpr (CL == 1) {
                const double n = P.n_in[o + q] + P.n_shift;
                nn[q] = n;
                mm[q] = 1.0 - 1.0 / n;
                trc[q] = P.tr_in ? P.tr_in[o + q] : tr;
                tsc[q] = P.ts_in ? P.ts_in[o + q] : ts;
            }
        }
        __syncthreads();
        for (int i = tid; i < nx; i += nt) {
            int T = (nz - 1) * nx + i, B = i;
            F.Tbt[i] = t2h * k_at(T, P.p_top);
            F.Tbb[i] = t2h * k_at(B, P.p_bot);
        }
        __syncthreads();
        for (int l = 1; l < nlev; ++l) {
            for (int I = tid; I < L64[l].nx; I += nt) {
                L64[l].Tbt[I] = 0.25 * (0.5 * (L64[l - 1].Tbt[2 * I] + L64[l - 1].Tbt[2 * I + 1]));
                L64[l].Tbb[I] = 0.25 * (0.5 * (L64[l - 1].Tbb[2 * I] + L64[l - 1].Tbb[2 * I + 1]));
            }
            __syncthreads();
        }
    }

    // theta^n of the step's old head
    __device__ void theta_old() {
        for (int q = tid; q < nc; q += nt) {
            double pp = p[q];
            if constexpr (CL == 0) {
                thold[q] = pp < 0.0 ? tr + (ts - tr) * exp(aa[q] * pp) : ts;
            } else {
                const double r = trc[q], t = tsc[q];
                thold[q] = pp < 0.0 ? r + (t - r) * vg_sat(aa[q], nn[q], mm[q], pp) : t;
            }
        }
        __syncthreads();
    }

    // Picard system at p (Gardner closure, harmonic faces, f = -R), all levels;
    // returns ||f||_inf as a bit pattern
    __device__ unsigned long long assemble() {
        const Lv64& F = L64[0];
        const Lv<TM>& M0 = LM[0];
        for (int q = tid; q < nc; q += nt) {
            double pp = p[q], ks = Ks[q];
            if constexpr (CL == 0) {
                if (pp < 0.0) {
                    double a = aa[q];
                    double E = exp(a * pp);
                    K[q] = ks * E;
                    th[q] = tr + (ts - tr) * E;
                    F.Cdt[q] = ((ts - tr) * a * E) * idt;
                } else {
                    K[q] = ks; th[q] = ts; F.Cdt[q] = 0.0;
                }
            } else {
                const double r = trc[q], t = tsc[q];
                if (pp < 0.0) {
                    double S, krw, dS;
                    vg_eval(aa[q], nn[q], mm[q], pp, S, krw, dS);
                    K[q] = ks * krw;
                    th[q] = r + (t - r) * S;
                    F.Cdt[q] = ((t - r) * dS) * idt;
                } else {
                    K[q] = ks; th[q] = t; F.Cdt[q] = 0.0;
                }
            }
        }
        __syncthreads();
        for (int q = tid; q < nc; q += nt) {
            int j = fdiv(q, nx, F.mnx), i = q - j * nx;
            double kp = K[q];
            if (i < nx - 1) { double ke = K[q + 1]; F.Tx[q] = t2h * kp * ke / (kp + ke); }
            else F.Tx[q] = 0.0;
            if (j < nz - 1) { double kn = K[q + nx]; F.Tz[q] = t2h * kp * kn / (kp + kn); }
            else F.Tz[q] = 0.0;
        }
        __syncthreads();
        unsigned long long m = 0;
        for (int q = tid; q < nc; q += nt) {
            int j = fdiv(q, nx, F.mnx), i = q - j * nx;
            double pp = p[q];
            double R = (th[q] - thold[q]) * idt;
            double d = F.Cdt[q];
            double te = 0.0, tw = 0.0, tn = 0.0, tsf = 0.0;
            if (i < nx - 1) { te = F.Tx[q];     R += -te * (p[q + 1] - pp); d += te; }
            if (i > 0)      { tw = F.Tx[q - 1]; R += -tw * (p[q - 1] - pp); d += tw; }
            if (j < nz - 1) { tn = F.Tz[q];     R += -tn * (p[q + nx] - pp) - tn * h; d += tn; }
            else { double t = F.Tbt[i]; R += -t * (P.p_top - pp) - t * h / 2.0; d += t; }
            if (j > 0)      { tsf = F.Tz[q - nx]; R += -tsf * (p[q - nx] - pp) + tsf * h; d += tsf; }
            else { double t = F.Tbb[i]; R += t * (pp - P.p_bot) + t * h / 2.0; d += t; }
            F.D[q] = d;
            f64[q] = -R;
            dp64[q] = 0.0;
            const int sq = sidx(M0, i, j);
            if constexpr (SC) {
                double inv = 1.0 / d;
                M0.q[sq] = inv; M0.D[sq] = d;
                M0.c0[sq] = te * inv; M0.c1[sq] = tw * inv; M0.c2[sq] = tn * inv; M0.c3[sq] = tsf * inv;
                M0.f[sq] = -R * inv;
            } else {
                M0.c0[sq] = (TM)te; M0.c1[sq] = (TM)tn; M0.D[sq] = (TM)d;
                M0.q[sq] = (TM)(1.0f / (float)d);
                M0.f[sq] = (TM)(-R); M0.dp[q] = TM(0);
            }
            unsigned long long b = abs_bits(R);
            m = b > m ? b : m;
        }
        const unsigned long long fb = block_max(m, red);
        // coarse operators (Fig. diffUpscale)
        for (int l = 1; l < nlev; ++l) {
            const Lv64& Fl = L64[l - 1];
            const Lv64& Cl = L64[l];
            const Lv<TM>& Ml = LM[l];
            const int fx = Fl.nx;
            for (int c = tid; c < Cl.nc; c += nt) {
                int J = fdiv(c, Cl.nx, Cl.mnx), I = c - J * Cl.nx;
                int f00 = (2 * J) * fx + 2 * I, f01 = f00 + fx;
                double cd = 0.25 * (Fl.Cdt[f00] + Fl.Cdt[f00 + 1] + Fl.Cdt[f01] + Fl.Cdt[f01 + 1]);
                double d = cd, te = 0.0, tw = 0.0, tn = 0.0, tsf = 0.0;
                if (I < Cl.nx - 1) { te = 0.25 * (0.5 * (Fl.Tx[f00 + 1] + Fl.Tx[f01 + 1])); d += te; }
                if (I > 0)         { tw = 0.25 * (0.5 * (Fl.Tx[f00 - 1] + Fl.Tx[f01 - 1])); d += tw; }
                if (J < Cl.nz - 1) { tn = 0.25 * (0.5 * (Fl.Tz[f01] + Fl.Tz[f01 + 1])); d += tn; }
                else d += Cl.Tbt[I];
                if (J > 0)         { tsf = 0.25 * (0.5 * (Fl.Tz[f00 - fx] + Fl.Tz[f00 - fx + 1])); d += tsf; }
                else d += Cl.Tbb[I];
                Cl.Tx[c] = te; Cl.Tz[c] = tn; Cl.Cdt[c] = cd; Cl.D[c] = d;
                const int sc = sidx(Ml, I, J);
                if constexpr (SC) {
                    double inv = 1.0 / d;
                    Ml.q[sc] = inv; Ml.D[sc] = d;
                    Ml.c0[sc] = te * inv; Ml.c1[sc] = tw * inv; Ml.c2[sc] = tn * inv; Ml.c3[sc] = tsf * inv;
                } else {
                    Ml.c0[sc] = (TM)te; Ml.c1[sc] = (TM)tn; Ml.D[sc] = (TM)d;
                    Ml.q[sc] = (TM)(1.0f / (float)d);
                }
            }
            __syncthreads();
        }
        return fb;
    }

    // one multigrid cycle: the V-cycle, or (WC, a separate kernel
    // instantiation so the V kernels keep their register allocation) the
    // cycle of index P.gamma
    __device__ void mgcycle(const TM* f0) {
        if constexpr (WC) gwalk<TM, GCta>(LM, L64, 0, nlev, P.lw, P.nu1, P.nu2, P.gamma, Amat, f0, false);
        else vcycle<TM>(LM, L64, nlev, P.lw, P.nu1, P.nu2, Amat, f0);
    }

    // x += e (FP64, natural order += FP32 finest-level correction), then the
    // CTA synchronises
    __device__ __forceinline__ void add_correction(double* __restrict__ x, const TM* __restrict__ e) const {
        const Lv<TM>& M0 = LM[0];
        const unsigned mnx = L64[0].mnx;
#pragma unroll 4
        for (int q = tid; q < nc; q += nt) {
            const int j = fdiv(q, nx, mnx), i = q - j * nx;
            x[q] += (double)e[sidx(M0, i, j)];
        }
        __syncthreads();
    }

    // FP64 defect r = f - A x of the finest operator, stored as the next FP32
    // right-hand side rf (with the FP32 correction ef cleared); returns this
    // thread's max |r| as a bit pattern (distinct arrays: restrict views)
    __device__ __forceinline__ unsigned long long defect(const double* __restrict__ f, const double* __restrict__ x,
                                                         const double* __restrict__ Tx,
                                                         const double* __restrict__ Tz,
                                                         const double* __restrict__ D, TM* __restrict__ rf,
                                                         TM* __restrict__ ef) const {
        const unsigned mnx = L64[0].mnx;
        unsigned long long mm = 0;
#pragma unroll 2
        for (int q = tid; q < nc; q += nt) {
            const int j = fdiv(q, nx, mnx), i = q - j * nx;
            double sn = 0.0;
            if (i < nx - 1) sn += Tx[q] * x[q + 1];
            if (i > 0)      sn += Tx[q - 1] * x[q - 1];
            if (j < nz - 1) sn += Tz[q] * x[q + nx];
            if (j > 0)      sn += Tz[q - nx] * x[q - nx];
            const double r = f[q] - (D[q] * x[q] - sn);
            const int sq = sidx(LM[0], i, j);
            rf[sq] = (TM)r;
            ef[sq] = TM(0);
            const unsigned long long b = abs_bits(r);
            mm = b > mm ? b : mm;
        }
        return mm;
    }

    // multigrid solve of A dp = f from dp = 0 (set up by assemble()); stops
    // when ||f - A dp||_inf < mg_tol max(1, ||f||_inf).  Returns false when a
    // norm is not finite.
    __device__ bool mg_solve(unsigned long long fb, long long& mg_tot, int& status) {
        const Lv<TM>& M0 = LM[0];
        const double fn = __longlong_as_double((long long)fb);
        const double target = P.mg_tol * (fn > 1.0 ? fn : 1.0);
        double rn = fn;
        int cyc = 0;
        while (rn >= target && cyc < P.mg_maxit) {
            unsigned long long rb;
            if constexpr (SC) {
                mgcycle((const TM*)f64);
                ++cyc;
                rb = resid_norm<TM>(M0, P.nu2 > 0 && nlev > 1, red);
            } else {
                for (int in = 0; in < P.mixed_inner && cyc < P.mg_maxit; ++in) {
                    mgcycle(nullptr);
                    ++cyc;
                }
                // dp += e in FP64, then the FP64 defect: stopping norm and the
                // next FP32 right-hand side
                add_correction(dp64, M0.dp);
                rb = block_max(defect(f64, dp64, L64[0].Tx, L64[0].Tz, L64[0].D, M0.f, M0.dp), red);
            }
            if (rb > INF_BITS - 1) { mg_tot += cyc; return false; }
            rn = __longlong_as_double((long long)rb);
        }
        mg_tot += cyc;
        if (!(rn < target)) status = max(status, (int)RICH_MG_MAXIT);
        return true;
    }

    // one implicit-Euler step by modified Picard (Sec. 4.1); returns false if
    // the sample failed.  A failure (PICARD_MAXIT, NONFINITE) replaces any
    // earlier MG_MAXIT flag: the sample's QoI is undefined, whatever happened
    // in its multigrid solves before
    __device__ bool time_step(long long& pic_tot, long long& mg_tot, int& maxpic, int& status) {
        theta_old();
        int k = 0;
        bool alive = true;
        for (;;) {
            const unsigned long long fb = assemble();
            if (fb > INF_BITS - 1) { status = RICH_NONFINITE; alive = false; break; }
            if (!mg_solve(fb, mg_tot, status)) { status = RICH_NONFINITE; alive = false; break; }
            unsigned long long dm = 0;
            for (int q = tid; q < nc; q += nt) {
                double d;
                if constexpr (SC) {
                    const int j = fdiv(q, nx, L64[0].mnx);
                    d = dp64[sidx(LM[0], q - j * nx, j)];
                } else {
                    d = dp64[q];
                }
                p[q] += d;
                unsigned long long b = abs_bits(d);
                dm = b > dm ? b : dm;
            }
            const unsigned long long db = block_max(dm, red);
            ++k;
            ++pic_tot;
            if (db > INF_BITS - 1) { status = RICH_NONFINITE; alive = false; break; }
            if (__longlong_as_double((long long)db) < P.picard_tol) break;
            if (k >= P.picard_maxit) { status = RICH_PICARD_MAXIT; alive = false; break; }
        }
        maxpic = max(maxpic, k);
        return alive;
    }

    // mean outward Darcy flux through the bottom faces (valid in warp 0)
    __device__ double qoi_warp0() const {
        double acc = 0.0;
        for (int i = tid; i < nx; i += 32) {
            double kb = k_at(i, P.p_bot);
            acc += kb * (2.0 * (p[i] - P.p_bot) / h + 1.0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        return acc / nx;
    }

    // ------------------------------------------------------------ adjoint
    // Jacobian pieces at the assembled state p = p^n: for every cell c and each
    // interior face f (E, W, N, S) D_fc = T_f - g_cf dT_f/dp_c with
    // g_cf = p_nb - p_c + s h (s = +1 north, -1 south), and the diagonal
    // C_c/dt + Dirichlet T_b; so (J^T lam)_c = dg_c lam_c + sum_f D_fc (lam_c - lam_nb).
    __device__ void adj_prepare(double* dE, double* dW, double* dN, double* dS, double* dg) {
        const Lv64& F = L64[0];
        for (int q = tid; q < nc; q += nt) {
            int j = fdiv(q, nx, F.mnx), i = q - j * nx;
            const double pc = p[q], kc = K[q];
            const double dk = pc < 0.0 ? aa[q] * kc : 0.0;      // dK_c/dp_c
            double e = 0.0, w = 0.0, n = 0.0, s = 0.0, d = F.Cdt[q];
            if (i < nx - 1) { double kn = K[q + 1], den = kc + kn;
                e = F.Tx[q] - (p[q + 1] - pc) * (t2h * kn * kn / (den * den)) * dk; }
            if (i > 0)      { double kn = K[q - 1], den = kc + kn;
                w = F.Tx[q - 1] - (p[q - 1] - pc) * (t2h * kn * kn / (den * den)) * dk; }
            if (j < nz - 1) { double kn = K[q + nx], den = kc + kn;
                n = F.Tz[q] - (p[q + nx] - pc + h) * (t2h * kn * kn / (den * den)) * dk; }
            else d += F.Tbt[i];
            if (j > 0)      { double kn = K[q - nx], den = kc + kn;
                s = F.Tz[q - nx] - (p[q - nx] - pc - h) * (t2h * kn * kn / (den * den)) * dk; }
            else d += F.Tbb[i];
            dE[q] = e; dW[q] = w; dN[q] = n; dS[q] = s; dg[q] = d;
        }
        __syncthreads();
    }

    __device__ __forceinline__ double jt_apply(const double* dE, const double* dW, const double* dN,
                                               const double* dS, const double* dg, const double* lam,
                                               int q) const {
        int j = fdiv(q, nx, L64[0].mnx), i = q - j * nx;
        const double l = lam[q];
        double v = dg[q] * l;
        if (i < nx - 1) v += dE[q] * (l - lam[q + 1]);
        if (i > 0)      v += dW[q] * (l - lam[q - 1]);
        if (j < nz - 1) v += dN[q] * (l - lam[q + nx]);
        if (j > 0)      v += dS[q] * (l - lam[q - nx]);
        return v;
    }

    // approximate e = A^{-1} r by ninner V-cycles from e = 0 (A: the Picard
    // operator assembled at the same state); e is returned in dp64 / M0.dp
    __device__ void mg_apply(const double* r, int ninner) {
        const Lv<TM>& M0 = LM[0];
        for (int q = tid; q < nc; q += nt) {
            const int j = fdiv(q, nx, L64[0].mnx), sq = sidx(M0, q - j * nx, j);
            if constexpr (SC) M0.f[sq] = r[q] * M0.q[sq];
            else M0.f[sq] = (TM)r[q];
            M0.dp[q] = TM(0);
        }
        __syncthreads();
        for (int k = 0; k < ninner; ++k) {
            if constexpr (SC) mgcycle(r);
            else mgcycle(nullptr);
        }
    }

    // J^T lam = rhs by defect correction preconditioned with CCMG on A:
    // lam += A^{-1}(rhs - J^T lam) until ||rhs - J^T lam|| <= adj_tol ||rhs||.
    // Returns the number of outer iterations (adj_maxit + 1 when not converged).
    __device__ int adj_solve(const double* dE, const double* dW, const double* dN, const double* dS,
                             const double* dg, const double* rhs, double* lam, double* r) {
        const Lv<TM>& M0 = LM[0];
        unsigned long long m = 0;
        for (int q = tid; q < nc; q += nt) {
            lam[q] = 0.0;
            r[q] = rhs[q];
            unsigned long long b = abs_bits(rhs[q]);
            m = b > m ? b : m;
        }
        const unsigned long long b0 = block_max(m, red);
        const double target = P.adj_tol * __longlong_as_double((long long)b0);
        if (b0 == 0) return 0;
        for (int it = 1; it <= P.adj_maxit; ++it) {
            mg_apply(r, P.adj_inner);
            for (int q = tid; q < nc; q += nt) {
                const int j = fdiv(q, nx, L64[0].mnx);
                lam[q] += (double)M0.dp[sidx(M0, q - j * nx, j)];
            }
            __syncthreads();
            unsigned long long mm = 0;
            for (int q = tid; q < nc; q += nt) {
                double v = rhs[q] - jt_apply(dE, dW, dN, dS, dg, lam, q);
                r[q] = v;
                unsigned long long b = abs_bits(v);
                mm = b > mm ? b : mm;
            }
            const unsigned long long rb = block_max(mm, red);
            if (rb > INF_BITS - 1) return P.adj_maxit + 1;
            if (__longlong_as_double((long long)rb) <= target) return it;
        }
        return P.adj_maxit + 1;
    }

    // e = M^{-1} r: ninner cycles of the Picard operator A from zero (a fixed
    // linear operator: the same cycles on the same matrix), copied to out
    __device__ void precond(const double* r, double* out) {
        mg_apply(r, P.adj_inner);
        const TM* e = LM[0].dp;
        for (int q = tid; q < nc; q += nt) {
            const int j = fdiv(q, nx, L64[0].mnx), sq = sidx(LM[0], q - j * nx, j);
            out[q] = (double)e[sq];
        }
        __syncthreads();
    }

    // y = J^T x over all cells, then the CTA synchronises
    __device__ void jt_vec(const double* dE, const double* dW, const double* dN, const double* dS,
                           const double* dg, const double* x, double* y) {
        for (int q = tid; q < nc; q += nt) y[q] = jt_apply(dE, dW, dN, dS, dg, x, q);
        __syncthreads();
    }

    // J^T lam = rhs by BiCGStab (van der Vorst 1992) right-preconditioned with
    // the CCMG cycles of A: converged when the TRUE residual ||rhs - J^T lam||
    // <= adj_tol ||rhs|| (checked explicitly whenever the recursive residual
    // says so; a mismatch restarts the recurrence from the true residual).
    // Returns the number of preconditioner applications (adj_maxit + 1 when
    // not converged); w holds the vectors r (also s), r^, p, v, t, p^, s^.
    __device__ int adj_solve_bicgstab(const double* dE, const double* dW, const double* dN, const double* dS,
                                      const double* dg, const double* rhs, double* lam, double* r, double* rh,
                                      double* pk, double* v, double* t, double* ph, double* sh) {
        double* redd = reinterpret_cast<double*>(red);
        unsigned long long m = 0;
        for (int q = tid; q < nc; q += nt) {
            lam[q] = 0.0;
            unsigned long long b = abs_bits(rhs[q]);
            m = b > m ? b : m;
        }
        const unsigned long long b0 = block_max(m, red);
        if (b0 == 0) return 0;
        const double target = P.adj_tol * __longlong_as_double((long long)b0);
        int apps = 0;
        bool restart = true;
        double rho = 1.0, alpha = 1.0, omega = 1.0;
        while (apps < P.adj_maxit) {
            if (restart) {                          // r = r^ = rhs - J^T lam, p = v = 0
                unsigned long long rm = 0;
                for (int q = tid; q < nc; q += nt) {
                    const double rv = rhs[q] - jt_apply(dE, dW, dN, dS, dg, lam, q);
                    r[q] = rv; rh[q] = rv; pk[q] = 0.0; v[q] = 0.0;
                    unsigned long long b = abs_bits(rv);
                    rm = b > rm ? b : rm;
                }
                const unsigned long long rb = block_max(rm, red);
                if (rb > INF_BITS - 1) break;
                if (__longlong_as_double((long long)rb) <= target) return apps;
                rho = alpha = omega = 1.0;
                restart = false;
                if (apps > 0) ++apps;               // a restart counts as one application
            }
            double s1 = 0.0;
            for (int q = tid; q < nc; q += nt) s1 += rh[q] * r[q];
            const double rho_new = block_sum(s1, redd);
            if (!(fabs(rho_new) > 0.0) || !isfinite(rho_new)) { restart = true; if (!isfinite(rho_new)) break; continue; }
            const double beta = (rho_new / rho) * (alpha / omega);
            for (int q = tid; q < nc; q += nt) pk[q] = r[q] + beta * (pk[q] - omega * v[q]);
            __syncthreads();
            precond(pk, ph); ++apps;
            jt_vec(dE, dW, dN, dS, dg, ph, v);
            double s2 = 0.0;
            for (int q = tid; q < nc; q += nt) s2 += rh[q] * v[q];
            const double den = block_sum(s2, redd);
            if (!(fabs(den) > 0.0) || !isfinite(den)) { restart = true; if (!isfinite(den)) break; continue; }
            alpha = rho_new / den;
            unsigned long long sm = 0;
            for (int q = tid; q < nc; q += nt) {
                const double sv = r[q] - alpha * v[q];
                r[q] = sv;                                  // r now holds s
                unsigned long long b = abs_bits(sv);
                sm = b > sm ? b : sm;
            }
            const unsigned long long sb = block_max(sm, red);
            if (sb > INF_BITS - 1) break;
            if (__longlong_as_double((long long)sb) <= target) {
                for (int q = tid; q < nc; q += nt) lam[q] += alpha * ph[q];
                __syncthreads();
                if (true_resid_ok(dE, dW, dN, dS, dg, rhs, lam, target)) return apps;
                restart = true;
                continue;
            }
            precond(r, sh); ++apps;
            jt_vec(dE, dW, dN, dS, dg, sh, t);
            double s3 = 0.0, s4 = 0.0;
            for (int q = tid; q < nc; q += nt) { s3 += t[q] * r[q]; s4 += t[q] * t[q]; }
            const double ts = block_sum(s3, redd);
            const double tt = block_sum(s4, redd);
            omega = tt > 0.0 ? ts / tt : 0.0;
            unsigned long long rm = 0;
            for (int q = tid; q < nc; q += nt) {
                lam[q] += alpha * ph[q] + omega * sh[q];
                const double rv = r[q] - omega * t[q];
                r[q] = rv;
                unsigned long long b = abs_bits(rv);
                rm = b > rm ? b : rm;
            }
            const unsigned long long rb = block_max(rm, red);
            if (rb > INF_BITS - 1) break;
            if (__longlong_as_double((long long)rb) <= target) {
                if (true_resid_ok(dE, dW, dN, dS, dg, rhs, lam, target)) return apps;
                restart = true;
                continue;
            }
            if (!(omega != 0.0)) restart = true;
            rho = rho_new;
        }
        return P.adj_maxit + 1;
    }

    // J^T lam = rhs by restarted GMRES(ADJ_M) (Saad & Schultz 1986), right-
    // preconditioned with the CCMG cycles of A, modified Gram-Schmidt, Givens
    // rotations; each cycle ends with the update lam += Z y and the TRUE
    // residual ||rhs - J^T lam||_inf <= adj_tol ||rhs||_inf decides.  The
    // Hessenberg matrix and rotations are computed by every thread from the
    // same block sums (uniform control flow).  Returns the number of
    // preconditioner applications (adj_maxit + 1 when not converged).
    __device__ int adj_solve_gmres(const double* dE, const double* dW, const double* dN, const double* dS,
                                   const double* dg, const double* rhs, double* lam, double* kry) {
        // Hessenberg matrix, rotations, right-hand side and solution of the
        // small least-squares problem: one copy per CTA, updated by thread 0
        __shared__ double sH[ADJ_M + 1][ADJ_M], scs[ADJ_M], ssn[ADJ_M], sg[ADJ_M + 1], sy[ADJ_M];
        double* redd = reinterpret_cast<double*>(red);
        double* V = kry;                                  // [ADJ_M + 1][nc]
        double* Z = kry + (size_t)(ADJ_M + 1) * nc;       // [ADJ_M][nc]
        unsigned long long m = 0;
        for (int q = tid; q < nc; q += nt) {
            lam[q] = 0.0;
            unsigned long long b = abs_bits(rhs[q]);
            m = b > m ? b : m;
        }
        const unsigned long long b0 = block_max(m, red);
        if (b0 == 0) return 0;
        const double target = P.adj_tol * __longlong_as_double((long long)b0);
        int apps = 0;
        while (apps < P.adj_maxit) {
            // r = rhs - J^T lam (the true residual), its inf-norm and 2-norm
            unsigned long long rm = 0;
            double s2 = 0.0;
            for (int q = tid; q < nc; q += nt) {
                const double rv = rhs[q] - jt_apply(dE, dW, dN, dS, dg, lam, q);
                V[q] = rv;
                s2 += rv * rv;
                unsigned long long b = abs_bits(rv);
                rm = b > rm ? b : rm;
            }
            const unsigned long long rb = block_max(rm, red);
            const double beta = sqrt(block_sum(s2, redd));
            if (rb > INF_BITS - 1 || !(beta > 0.0)) break;
            if (__longlong_as_double((long long)rb) <= target) return apps;
            const double ib = 1.0 / beta;
            for (int q = tid; q < nc; q += nt) V[q] *= ib;
            if (tid == 0) {
                for (int i = 0; i <= ADJ_M; ++i) sg[i] = 0.0;
                sg[0] = beta;
            }
            __syncthreads();
            int k = 0;
            for (; k < ADJ_M && apps < P.adj_maxit; ++k) {
                double* vk = V + (size_t)k * nc;
                double* zk = Z + (size_t)k * nc;
                double* w = V + (size_t)(k + 1) * nc;
                precond(vk, zk); ++apps;
                jt_vec(dE, dW, dN, dS, dg, zk, w);
                for (int i = 0; i <= k; ++i) {                  // modified Gram-Schmidt
                    const double* vi = V + (size_t)i * nc;
                    double d = 0.0;
                    for (int q = tid; q < nc; q += nt) d += w[q] * vi[q];
                    const double h = block_sum(d, redd);
                    if (tid == 0) sH[i][k] = h;
                    for (int q = tid; q < nc; q += nt) w[q] -= h * vi[q];
                    __syncthreads();
                }
                double d = 0.0;
                for (int q = tid; q < nc; q += nt) d += w[q] * w[q];
                const double hn = sqrt(block_sum(d, redd));
                if (hn > 0.0) {
                    const double ih = 1.0 / hn;
                    for (int q = tid; q < nc; q += nt) w[q] *= ih;
                }
                if (tid == 0) {                                  // rotations on column k
                    sH[k + 1][k] = hn;
                    for (int i = 0; i < k; ++i) {
                        const double a = sH[i][k], b = sH[i + 1][k];
                        sH[i][k] = scs[i] * a + ssn[i] * b;
                        sH[i + 1][k] = -ssn[i] * a + scs[i] * b;
                    }
                    const double a = sH[k][k], b = sH[k + 1][k];
                    const double rr = sqrt(a * a + b * b);
                    scs[k] = rr > 0.0 ? a / rr : 1.0;
                    ssn[k] = rr > 0.0 ? b / rr : 0.0;
                    sH[k][k] = rr; sH[k + 1][k] = 0.0;
                    sg[k + 1] = -ssn[k] * sg[k];
                    sg[k] = scs[k] * sg[k];
                }
                __syncthreads();
                const double gk = sg[k + 1];
                // the 2-norm estimate bounds the inf-norm: the cycle may stop early
                if (!(hn > 0.0) || !isfinite(gk) || fabs(gk) <= target) { ++k; break; }
            }
            if (tid == 0) {                                      // y = H^{-1} g, k x k upper triangular
                for (int i = k - 1; i >= 0; --i) {
                    double t = sg[i];
                    for (int j = i + 1; j < k; ++j) t -= sH[i][j] * sy[j];
                    sy[i] = sH[i][i] != 0.0 ? t / sH[i][i] : 0.0;
                }
            }
            __syncthreads();
            for (int q = tid; q < nc; q += nt) {
                double acc = lam[q];
                for (int j = 0; j < k; ++j) acc += sy[j] * Z[(size_t)j * nc + q];
                lam[q] = acc;
            }
            __syncthreads();
        }
        return true_resid_ok(dE, dW, dN, dS, dg, rhs, lam, target) ? apps : P.adj_maxit + 1;
    }

    // ||rhs - J^T lam||_inf <= target (the true residual)
    __device__ bool true_resid_ok(const double* dE, const double* dW, const double* dN, const double* dS,
                                  const double* dg, const double* rhs, const double* lam, double target) {
        unsigned long long m = 0;
        for (int q = tid; q < nc; q += nt) {
            unsigned long long b = abs_bits(rhs[q] - jt_apply(dE, dW, dN, dS, dg, lam, q));
            m = b > m ? b : m;
        }
        const unsigned long long rb = block_max(m, red);
        return rb <= INF_BITS - 1 && __longlong_as_double((long long)rb) <= target;
    }

    // g -= (dR/dm)^T lam at the assembled state (m = ln Ks): interior faces
    // contribute -g_cf (lam_c - lam_nb) dT_f/dm_c with dT_f/dm_c =
    // (2/h^2) K_nb^2 K_c / (K_c + K_nb)^2; Dirichlet faces -g_b T_b lam_c
    __device__ void adj_grad_update(const double* lam, double* g) {
        const Lv64& F = L64[0];
        for (int q = tid; q < nc; q += nt) {
            int j = fdiv(q, nx, F.mnx), i = q - j * nx;
            const double pc = p[q], kc = K[q], lc = lam[q];
            double v = 0.0;
            if (i < nx - 1) { double kn = K[q + 1], den = kc + kn;
                v -= (p[q + 1] - pc) * (lc - lam[q + 1]) * (t2h * kn * kn * kc / (den * den)); }
            if (i > 0)      { double kn = K[q - 1], den = kc + kn;
                v -= (p[q - 1] - pc) * (lc - lam[q - 1]) * (t2h * kn * kn * kc / (den * den)); }
            if (j < nz - 1) { double kn = K[q + nx], den = kc + kn;
                v -= (p[q + nx] - pc + h) * (lc - lam[q + nx]) * (t2h * kn * kn * kc / (den * den)); }
            else v -= (P.p_top - pc + h / 2.0) * F.Tbt[i] * lc;
            if (j > 0)      { double kn = K[q - nx], den = kc + kn;
                v -= (p[q - nx] - pc - h) * (lc - lam[q - nx]) * (t2h * kn * kn * kc / (den * den)); }
            else v -= (P.p_bot - pc - h / 2.0) * F.Tbb[i] * lc;
            g[q] -= v;
        }
        __syncthreads();
    }
};

template <typename TM>
__device__ __forceinline__ void init_levels(const FParams& P, char* slot, unsigned char* sm, Lv64* L64,
                                            Lv<TM>* LM) {
    constexpr bool SC = Scaled<TM>::value;
    const int nlev = P.nlev;
    if ((int)threadIdx.x < nlev) {
        const int l = threadIdx.x;
        Lv64& a = L64[l];
        a.nx = P.nx[l]; a.nz = P.nz[l]; a.nc = a.nx * a.nz; a.mnx = P.mnx[l];
        double** pp[N64] = {&a.Tx, &a.Tz, &a.Cdt, &a.D, &a.Tbt, &a.Tbb};
        for (int k = 0; k < N64; ++k)
            *pp[k] = P.s64[l][k] >= 0 ? (double*)(sm + P.s64[l][k]) : (double*)(slot + P.o64[l][k]);
        Lv<TM>& b = LM[l];
        b.nx = a.nx; b.nz = a.nz; b.hx = a.nx >> 1; b.nc = a.nc; b.mnx = P.mnx[l]; b.mhx = P.mhx[l];
        b.H = l < nlev - 1 ? b.hx * b.nz : 0;             // colour-split unless coarsest
        TM** qq[NMG] = {&b.c0, &b.c1, &b.c2, &b.c3, &b.q, &b.f, &b.dp, &b.D};
        for (int k = 0; k < NMG; ++k)
            *qq[k] = P.smg[l][k] >= 0 ? (TM*)(sm + P.smg[l][k])
                   : P.omg[l][k] >= 0 ? (TM*)(slot + P.omg[l][k]) : nullptr;
        if (P.osm[l] >= 0) b.dp = (TM*)(sm + P.osm[l]);   // corrections of small levels on chip
        if constexpr (!SC) { b.D = b.c3; b.c3 = nullptr; }   // FP32: D in the c3 slot
    }
    __syncthreads();
}

template <typename TM, int NT, bool WC, int CL>
__global__ void __launch_bounds__(NT, NT == 32 ? 32 : NT <= 128 ? 8 : NT <= 256 ? 4 : NT == 512 ? 2 : 1)
k_fused(const FParams P) {
    extern __shared__ unsigned char smraw[];
    __shared__ unsigned long long red[33];
    __shared__ int s_sample;
    __shared__ Lv64 L64[MAXL];
    __shared__ Lv<TM> LM[MAXL];
    char* slot = P.scratch + (size_t)blockIdx.x * P.slot_bytes;
    init_levels<TM>(P, slot, smraw, L64, LM);
    Cta<TM, WC, CL> C(P, slot, L64, LM, reinterpret_cast<TM*>(smraw), red);
    const int nc = C.nc, tid = C.tid, nt = C.nt;
    for (;;) {
        if (tid == 0) s_sample = atomicAdd(P.queue, 1);
        __syncthreads();
        const int s = s_sample;
        __syncthreads();
        if (s >= P.S) break;
        const unsigned long long t0 = globaltimer_ns();
        C.setup(s);
        int status = RICH_OK, maxpic = 0;
        bool alive = true;
        long long pic_tot = 0, mg_tot = 0;
        for (int step = 0; step < P.nsteps && alive; ++step)
            alive = C.time_step(pic_tot, mg_tot, maxpic, status);
        if (tid < 32) {
            const double q = C.qoi_warp0();
            if (tid == 0) {
                P.qoi[s] = alive ? q : __longlong_as_double(0x7FF8000000000000ll);
                if (P.status) P.status[s] = status;
                if (P.pic_total) P.pic_total[s] = pic_tot;
                if (P.mg_total) P.mg_total[s] = mg_tot;
                if (P.maxpic) P.maxpic[s] = maxpic;
                if (P.t_ns) P.t_ns[s] = (int64_t)(globaltimer_ns() - t0);
            }
        }
        if (P.p_final)
            for (int q = tid; q < nc; q += nt) P.p_final[(size_t)s * nc + q] = C.p[q];
        __syncthreads();
    }
}

}  // namespace

namespace {
// launch shapes of one (cycle precision, closure) pair: 128, 256, 512 or 1024
// threads, each with the V-cycle and the gamma >= 2 cycle instantiation
template <typename TM, int NT, bool WC, int CL>
int occ_one(const FParams& P, size_t smem, int* occ) {
    if (int e = allow_dyn_smem((const void*)k_fused<TM, NT, WC, CL>, smem)) return e;
    RICH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_fused<TM, NT, WC, CL>, NT, smem));
    if (*occ < 1) *occ = 1;
    return 0;
}

template <typename TM, int CL>
int occ_shapes(const FParams& P, size_t smem, int nt, int* occ) {
    const bool wc = P.gamma > 1;
    if (nt == 1024) return wc ? occ_one<TM, 1024, true, CL>(P, smem, occ) : occ_one<TM, 1024, false, CL>(P, smem, occ);
    if (nt == 256) return wc ? occ_one<TM, 256, true, CL>(P, smem, occ) : occ_one<TM, 256, false, CL>(P, smem, occ);
    if (nt == 128) return wc ? occ_one<TM, 128, true, CL>(P, smem, occ) : occ_one<TM, 128, false, CL>(P, smem, occ);
    if (nt == 32) return wc ? occ_one<TM, 32, true, CL>(P, smem, occ) : occ_one<TM, 32, false, CL>(P, smem, occ);
    return wc ? occ_one<TM, 512, true, CL>(P, smem, occ) : occ_one<TM, 512, false, CL>(P, smem, occ);
}

template <typename TM, int CL>
void launch_shapes(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st) {
    const bool wc = P.gamma > 1;
    if (nt == 1024) {
        if (wc) k_fused<TM, 1024, true, CL><<<grid, 1024, smem, st>>>(P);
        else k_fused<TM, 1024, false, CL><<<grid, 1024, smem, st>>>(P);
    } else if (nt == 256) {
        if (wc) k_fused<TM, 256, true, CL><<<grid, 256, smem, st>>>(P);
        else k_fused<TM, 256, false, CL><<<grid, 256, smem, st>>>(P);
    } else if (nt == 128) {
        if (wc) k_fused<TM, 128, true, CL><<<grid, 128, smem, st>>>(P);
        else k_fused<TM, 128, false, CL><<<grid, 128, smem, st>>>(P);
    } else if (nt == 32) {
        if (wc) k_fused<TM, 32, true, CL><<<grid, 32, smem, st>>>(P);
        else k_fused<TM, 32, false, CL><<<grid, 32, smem, st>>>(P);
    } else {
        if (wc) k_fused<TM, 512, true, CL><<<grid, 512, smem, st>>>(P);
        else k_fused<TM, 512, false, CL><<<grid, 512, smem, st>>>(P);
    }
}
}  // namespace
