// Batched modified-Picard / cell-centred-multigrid solve of the mixed-form
// Richards' equation (arXiv 1903.08741, Sec. 4), FP64 path and the FP32-in-FP64
// mixed-precision path.
//
// Layout: every per-cell quantity of level l is one array [S][nz_l][nx_l]
// (x fastest, row 0 at the bottom); a sample s of level l starts at s*nx_l*nz_l.
// Work is launched only for the samples still iterating: each kernel receives a
// compacted list of sample indices (Picard list, MG list) and a count, and is
// launched over (list slot, cell item) flattened, so converged samples cost
// nothing.  Per-sample norms are reduced in registers/shared memory and merged
// with one atomicMax per block on the IEEE bit pattern of |x| (for non-negative
// doubles the unsigned integer order is the numeric order, and NaN sorts above
// +Inf, so non-finite values surface as the maximum).
#include "rich_internal.cuh"
#include <math.h>
#include <string.h>
#include <stdio.h>
#include <chrono>
#include <vector>
#include <algorithm>
#include <stdlib.h>

namespace {

constexpr int TPB = 256;          // threads per block, flattened kernels
constexpr int RED_TPB = 256;      // threads per block, per-sample reduction kernels
constexpr int RED_CHUNK = 2048;   // cells per reduction block
constexpr unsigned long long ABS_MASK = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long INF_BITS = 0x7FF0000000000000ull;

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

// block-wide max, then one atomicMax into *dst (all threads must call)
__device__ __forceinline__ void block_max_atomic(unsigned long long v, unsigned long long* dst) {
    __shared__ unsigned long long sm[RED_TPB / 32];
    v = warp_max_u64(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ull;
        v = warp_max_u64(v);
        if (lane == 0 && v) atomicMax(dst, v);
    }
}

// flattened (slot, item) decomposition
__device__ __forceinline__ bool flat(const int32_t* list, int n, int W, int& s, int& item) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)n * W) return false;
    int slot = (int)(g / W);
    item = (int)(g - (long long)slot * W);
    s = list[slot];
    return true;
}

// ------------------------------------------------------------------ set-up
__global__ void k_setup(int S, int ncell, const double* __restrict__ lnKs,
                        const double* __restrict__ alpha, double alpha_scale, double p_init,
                        double* Ks, double* a, double* p) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)S * ncell) return;
    Ks[g] = exp(lnKs[g]);
    a[g] = alpha[g] * alpha_scale;
    p[g] = p_init;
}

__global__ void k_setup_samples(int S, int32_t* status, int32_t* alive, int64_t* pic_total,
                                int64_t* mg_total, int32_t* maxpic,
                                unsigned long long* n1, unsigned long long* n2,
                                unsigned long long* n3) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    status[s] = 0; alive[s] = 1; pic_total[s] = 0; mg_total[s] = 0; maxpic[s] = 0;
    n1[s] = 0; n2[s] = 0; n3[s] = 0;
}

// Dirichlet-face transmissibility Tb = 2 K(p_D) / h^2 with the adjacent cell's
// Ks and alpha (fixed for the whole solve).
__global__ void k_boundary_fine(int S, int nx, int nz, const double* __restrict__ Ks,
                                const double* __restrict__ a, double two_over_h2, double p_top,
                                double p_bot, double* Tbt, double* Tbb) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)S * nx) return;
    int s = (int)(g / nx), i = (int)(g - (long long)s * nx);
    size_t base = (size_t)s * nx * nz;
    size_t T = base + (size_t)(nz - 1) * nx + i, B = base + i;
    double kt = p_top < 0.0 ? Ks[T] * exp(a[T] * p_top) : Ks[T];
    double kb = p_bot < 0.0 ? Ks[B] * exp(a[B] * p_bot) : Ks[B];
    Tbt[g] = two_over_h2 * kt;
    Tbb[g] = two_over_h2 * kb;
}

__global__ void k_boundary_coarsen(int S, int nxc, const double* __restrict__ Tbt_f,
                                   const double* __restrict__ Tbb_f, double* Tbt_c, double* Tbb_c) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)S * nxc) return;
    int s = (int)(g / nxc), I = (int)(g - (long long)s * nxc);
    size_t f = (size_t)s * 2 * nxc + 2 * I;
    Tbt_c[g] = 0.25 * (0.5 * (Tbt_f[f] + Tbt_f[f + 1]));
    Tbb_c[g] = 0.25 * (0.5 * (Tbb_f[f] + Tbb_f[f + 1]));
}

__global__ void k_list_alive(int S, const int32_t* alive, int32_t* kpic, int32_t* list,
                             int32_t* count) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    kpic[s] = 0;
    if (alive[s]) list[atomicAdd(count, 1)] = s;
}

// ----------------------------------------------------------- Picard system
// Gardner closure: p < 0: E = exp(a p), K = Ks E, theta = tr + (ts - tr) E,
// C = (ts - tr) a E;  p >= 0: K = Ks, theta = ts, C = 0.
__global__ void k_theta_old(const int32_t* __restrict__ list, int n, int ncell,
                            const double* __restrict__ a, const double* __restrict__ p,
                            double tr, double ts, double* thold) {
    int s, q;
    if (!flat(list, n, ncell, s, q)) return;
    size_t P = (size_t)s * ncell + q;
    double pp = p[P];
    thold[P] = pp < 0.0 ? tr + (ts - tr) * exp(a[P] * pp) : ts;
}

__global__ void k_conductivity(const int32_t* __restrict__ list, int n, int ncell,
                               const double* __restrict__ Ks, const double* __restrict__ a,
                               const double* __restrict__ p, double tr, double ts, double dt,
                               double* K, double* th, double* Cdt) {
    int s, q;
    if (!flat(list, n, ncell, s, q)) return;
    size_t P = (size_t)s * ncell + q;
    double pp = p[P], ks = Ks[P];
    if (pp < 0.0) {
        double aa = a[P];
        double E = exp(aa * pp);
        K[P] = ks * E;
        th[P] = tr + (ts - tr) * E;
        Cdt[P] = ((ts - tr) * aa * E) / dt;
    } else {
        K[P] = ks;
        th[P] = ts;
        Cdt[P] = 0.0 / dt;
    }
}

// interior faces: T = (2/h^2) K_P K_N / (K_P + K_N)   (Eq. five_stencil)
__global__ void k_faces(const int32_t* __restrict__ list, int n, int nx, int nz,
                        const double* __restrict__ K, double two_over_h2, double* Tx, double* Tz) {
    int s, q;
    const int ncell = nx * nz;
    if (!flat(list, n, ncell, s, q)) return;
    int j = q / nx, i = q - j * nx;
    size_t P = (size_t)s * ncell + q;
    double kp = K[P];
    if (i < nx - 1) { double ke = K[P + 1]; Tx[P] = two_over_h2 * kp * ke / (kp + ke); }
    else Tx[P] = 0.0;
    if (j < nz - 1) { double kn = K[P + nx]; Tz[P] = two_over_h2 * kp * kn / (kp + kn); }
    else Tz[P] = 0.0;
}

// f = -R(p) (Eq. Mixed_based_3 right-hand side), diagonal D and 1/D, ||f||_inf.
__global__ void __launch_bounds__(RED_TPB)
k_rhs(const int32_t* __restrict__ list, int bps, int nx, int nz,
      const double* __restrict__ p, const double* __restrict__ th, const double* __restrict__ thold,
      const double* __restrict__ Tx, const double* __restrict__ Tz,
      const double* __restrict__ Tbt, const double* __restrict__ Tbb,
      const double* __restrict__ Cdt, double dt, double h, double p_top, double p_bot,
      double* f, double* D, double* invD, unsigned long long* nrm) {
    const int slot = blockIdx.x / bps, chunk = blockIdx.x - slot * bps;
    const int s = list[slot];
    const int ncell = nx * nz;
    const size_t base = (size_t)s * ncell;
    const int q0 = chunk * RED_CHUNK, q1 = min(ncell, q0 + RED_CHUNK);
    unsigned long long m = 0;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int j = q / nx, i = q - j * nx;
        size_t P = base + q;
        double pp = p[P];
        double R = (th[P] - thold[P]) / dt;
        double d = Cdt[P];
        if (i < nx - 1) { double t = Tx[P];     R += -t * (p[P + 1] - pp); d += t; }
        if (i > 0)      { double t = Tx[P - 1]; R += -t * (p[P - 1] - pp); d += t; }
        if (j < nz - 1) { double t = Tz[P];     R += -t * (p[P + nx] - pp) - t * h; d += t; }
        else { double t = Tbt[(size_t)s * nx + i]; R += -t * (p_top - pp) - t * h / 2.0; d += t; }
        if (j > 0)      { double t = Tz[P - nx]; R += -t * (p[P - nx] - pp) + t * h; d += t; }
        else { double t = Tbb[(size_t)s * nx + i]; R += t * (pp - p_bot) + t * h / 2.0; d += t; }
        f[P] = -R;
        D[P] = d;
        invD[P] = 1.0 / d;
        unsigned long long b = abs_bits(R);
        m = b > m ? b : m;
    }
    block_max_atomic(m, &nrm[s]);
}

// coarse operator by rediscretisation: mean of the two fine faces times 1/4,
// mean of the four fine mass terms (Fig. diffUpscale)
__global__ void k_coarsen(const int32_t* __restrict__ list, int n, int nxc, int nzc,
                          const double* __restrict__ Txf, const double* __restrict__ Tzf,
                          const double* __restrict__ Cdtf, const double* __restrict__ Tbtc,
                          const double* __restrict__ Tbbc, double* Tx, double* Tz, double* Cdt,
                          double* D, double* invD) {
    int s, q;
    const int ncell = nxc * nzc, fx = 2 * nxc;
    if (!flat(list, n, ncell, s, q)) return;
    int J = q / nxc, I = q - J * nxc;
    size_t fb = (size_t)s * 4 * ncell;
    size_t f00 = fb + (size_t)(2 * J) * fx + 2 * I, f01 = f00 + fx;
    size_t P = (size_t)s * ncell + q;
    double c = 0.25 * (Cdtf[f00] + Cdtf[f00 + 1] + Cdtf[f01] + Cdtf[f01 + 1]);
    double d = c;
    double te = 0.0, tn = 0.0;
    if (I < nxc - 1) { te = 0.25 * (0.5 * (Txf[f00 + 1] + Txf[f01 + 1])); d += te; }
    if (I > 0)       { d += 0.25 * (0.5 * (Txf[f00 - 1] + Txf[f01 - 1])); }
    if (J < nzc - 1) { tn = 0.25 * (0.5 * (Tzf[f01] + Tzf[f01 + 1])); d += tn; }
    else d += Tbtc[(size_t)s * nxc + I];
    if (J > 0)       { d += 0.25 * (0.5 * (Tzf[f00 - fx] + Tzf[f00 - fx + 1])); }
    else d += Tbbc[(size_t)s * nxc + I];
    Tx[P] = te; Tz[P] = tn; Cdt[P] = c; D[P] = d; invD[P] = 1.0 / d;
}

// --------------------------------------------------------------- multigrid
template <typename T>
__device__ __forceinline__ T offdiag(const T* __restrict__ Tx, const T* __restrict__ Tz,
                                     const T* x, size_t P, int i, int j, int nx, int nz) {
    T s = T(0);
    if (i < nx - 1) s += Tx[P] * x[P + 1];
    if (i > 0)      s += Tx[P - 1] * x[P - 1];
    if (j < nz - 1) s += Tz[P] * x[P + nx];
    if (j > 0)      s += Tz[P - nx] * x[P - nx];
    return s;
}

// one colour of red-black Gauss-Seidel (red: i + j even)
template <typename T>
__global__ void k_rbgs(const int32_t* __restrict__ list, int n, int nx, int nz, int colour,
                       const T* __restrict__ Tx, const T* __restrict__ Tz,
                       const T* __restrict__ invD, const T* __restrict__ f, T* dp) {
    int s, q;
    const int hx = nx >> 1;
    if (!flat(list, n, hx * nz, s, q)) return;
    int j = q / hx, c = q - j * hx;
    int i = 2 * c + ((j + colour) & 1);
    size_t P = (size_t)s * nx * nz + (size_t)j * nx + i;
    dp[P] = (f[P] + offdiag(Tx, Tz, dp, P, i, j, nx, nz)) * invD[P];
}

// r = f - A dp on the 2x2 children of each coarse cell, restricted by 1/4 sum
// (Eq. transfer); the coarse correction starts from zero
template <typename T>
__global__ void k_resid_restrict(const int32_t* __restrict__ list, int n, int nxc, int nzc,
                                 const T* __restrict__ Tx, const T* __restrict__ Tz,
                                 const T* __restrict__ D, const T* __restrict__ f,
                                 const T* __restrict__ dp, T* fc, T* dpc) {
    int s, q;
    const int ncc = nxc * nzc, nx = 2 * nxc, nz = 2 * nzc;
    if (!flat(list, n, ncc, s, q)) return;
    int J = q / nxc, I = q - J * nxc;
    size_t base = (size_t)s * 4 * ncc;
    T r[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int i = 2 * I + (k & 1), j = 2 * J + (k >> 1);
        size_t P = base + (size_t)j * nx + i;
        r[k] = f[P] - (D[P] * dp[P] - offdiag(Tx, Tz, dp, P, i, j, nx, nz));
    }
    size_t C = (size_t)s * ncc + q;
    fc[C] = T(0.25) * (r[0] + r[1] + r[2] + r[3]);
    dpc[C] = T(0);
}

// piecewise-constant prolongation and correction (Eq. transfer)
template <typename T>
__global__ void k_prolong(const int32_t* __restrict__ list, int n, int nxc, int nzc,
                          const T* __restrict__ dpc, T* dp) {
    int s, q;
    const int ncc = nxc * nzc, nx = 2 * nxc;
    if (!flat(list, n, ncc, s, q)) return;
    int J = q / nxc, I = q - J * nxc;
    T e = dpc[(size_t)s * ncc + q];
    size_t P = (size_t)s * 4 * ncc + (size_t)(2 * J) * nx + 2 * I;
    dp[P] += e; dp[P + 1] += e; dp[P + nx] += e; dp[P + nx + 1] += e;
}

// exact coarsest solve: one warp per sample, Gaussian elimination of the
// assembled five-point matrix (symmetric, diagonally dominant: no pivoting)
template <typename T>
__global__ void k_coarse_solve(const int32_t* __restrict__ list, int nx, int nz,
                               const T* __restrict__ Tx, const T* __restrict__ Tz,
                               const T* __restrict__ D, const T* __restrict__ f, T* dp) {
    extern __shared__ unsigned char smraw[];
    T* A = reinterpret_cast<T*>(smraw);
    const int nn = nx * nz, ld = nn + 1;
    const int s = list[blockIdx.x];
    const size_t base = (size_t)s * nn;
    const int lane = threadIdx.x;
    for (int r = lane; r < nn; r += 32) {
        for (int c = 0; c < nn; ++c) A[r * ld + c] = T(0);
        int j = r / nx, i = r - j * nx;
        A[r * ld + r] = D[base + r];
        if (i < nx - 1) A[r * ld + r + 1] = -Tx[base + r];
        if (i > 0)      A[r * ld + r - 1] = -Tx[base + r - 1];
        if (j < nz - 1) A[r * ld + r + nx] = -Tz[base + r];
        if (j > 0)      A[r * ld + r - nx] = -Tz[base + r - nx];
        A[r * ld + nn] = f[base + r];
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
    for (int r = lane; r < nn; r += 32) dp[base + r] = A[r * ld + nn];
}

// ||f - A dp||_inf per sample on the finest level
template <typename T>
__global__ void __launch_bounds__(RED_TPB)
k_resid_norm(const int32_t* __restrict__ list, int bps, int nx, int nz,
             const T* __restrict__ Tx, const T* __restrict__ Tz, const T* __restrict__ D,
             const T* __restrict__ f, const T* __restrict__ dp, unsigned long long* nrm) {
    const int slot = blockIdx.x / bps, chunk = blockIdx.x - slot * bps;
    const int s = list[slot];
    const int ncell = nx * nz;
    const size_t base = (size_t)s * ncell;
    const int q0 = chunk * RED_CHUNK, q1 = min(ncell, q0 + RED_CHUNK);
    unsigned long long m = 0;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int j = q / nx, i = q - j * nx;
        size_t P = base + q;
        T r = f[P] - (D[P] * dp[P] - offdiag(Tx, Tz, dp, P, i, j, nx, nz));
        unsigned long long b = abs_bits(r);
        m = b > m ? b : m;
    }
    block_max_atomic(m, &nrm[s]);
}

__global__ void k_zero(const int32_t* __restrict__ list, int n, int ncell, double* x) {
    int s, q;
    if (!flat(list, n, ncell, s, q)) return;
    x[(size_t)s * ncell + q] = 0.0;
}

// start of an MG solve: target = tol * max(1, ||f||); samples with
// ||f|| >= target enter the MG list
__global__ void k_mg_start(const int32_t* __restrict__ list, int n, double tol,
                           unsigned long long* nrm_f, double* target, int32_t* cyc,
                           int32_t* status, int32_t* alive, int32_t* out, int32_t* count) {
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n) return;
    int s = list[slot];
    unsigned long long b = nrm_f[s];
    nrm_f[s] = 0;
    cyc[s] = 0;
    if (b > INF_BITS - 1) {           // +Inf or NaN
        status[s] = max(status[s], (int)RICH_NONFINITE);
        alive[s] = 0;
        return;
    }
    double fn = __longlong_as_double((long long)b);
    double t = tol * (fn > 1.0 ? fn : 1.0);
    target[s] = t;
    if (fn >= t) out[atomicAdd(count, 1)] = s;
}

__global__ void k_mg_decide(const int32_t* __restrict__ list, int n, int maxit,
                            unsigned long long* nrm_r, const double* __restrict__ target,
                            int32_t* cyc, int64_t* mg_total, int32_t* status, int32_t* alive,
                            int32_t* out, int32_t* count) {
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n) return;
    int s = list[slot];
    unsigned long long b = nrm_r[s];
    nrm_r[s] = 0;
    int c = ++cyc[s];
    mg_total[s] += 1;
    if (b > INF_BITS - 1) {
        status[s] = max(status[s], (int)RICH_NONFINITE);
        alive[s] = 0;
        return;
    }
    double rn = __longlong_as_double((long long)b);
    if (rn < target[s]) return;                       // converged
    if (c >= maxit) { status[s] = max(status[s], (int)RICH_MG_MAXIT); return; }
    out[atomicAdd(count, 1)] = s;
}

__global__ void __launch_bounds__(RED_TPB)
k_update_p(const int32_t* __restrict__ list, int bps, int ncell, const int32_t* __restrict__ alive,
           const double* __restrict__ dp, double* p, unsigned long long* nrm) {
    const int slot = blockIdx.x / bps, chunk = blockIdx.x - slot * bps;
    const int s = list[slot];
    if (!alive[s]) return;                               // uniform per block
    const size_t base = (size_t)s * ncell;
    const int q0 = chunk * RED_CHUNK, q1 = min(ncell, q0 + RED_CHUNK);
    unsigned long long m = 0;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        double d = dp[base + q];
        p[base + q] += d;
        unsigned long long b = abs_bits(d);
        m = b > m ? b : m;
    }
    block_max_atomic(m, &nrm[s]);
}

__global__ void k_picard_decide(const int32_t* __restrict__ list, int n, int maxit, double tol,
                                unsigned long long* nrm_dp, int32_t* kpic, int64_t* pic_total,
                                int32_t* maxpic, int32_t* status, int32_t* alive, int32_t* out,
                                int32_t* count) {
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n) return;
    int s = list[slot];
    if (!alive[s]) return;                               // non-finite MG: already dead
    unsigned long long b = nrm_dp[s];
    nrm_dp[s] = 0;
    int k = ++kpic[s];
    pic_total[s] += 1;
    if (k > maxpic[s]) maxpic[s] = k;
    if (b > INF_BITS - 1) {
        status[s] = max(status[s], (int)RICH_NONFINITE);
        alive[s] = 0;
        return;
    }
    double dn = __longlong_as_double((long long)b);
    if (dn < tol) return;                                // converged this step
    if (k >= maxit) {
        status[s] = max(status[s], (int)RICH_PICARD_MAXIT);
        alive[s] = 0;
        return;
    }
    out[atomicAdd(count, 1)] = s;
}

// mean outward Darcy flux through the bottom faces: q.n = K_b (2 (p - p_bot)/h + 1)
__global__ void k_qoi(int S, int nx, int nz, const double* __restrict__ Ks,
                      const double* __restrict__ a, const double* __restrict__ p, double p_bot,
                      double h, const int32_t* __restrict__ alive, double* qoi) {
    const int s = blockIdx.x;
    const size_t base = (size_t)s * nx * nz;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nx; i += 32) {
        double kb = p_bot < 0.0 ? Ks[base + i] * exp(a[base + i] * p_bot) : Ks[base + i];
        acc += kb * (2.0 * (p[base + i] - p_bot) / h + 1.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) qoi[s] = alive[s] ? acc / nx : __longlong_as_double(0x7FF8000000000000ll);
}

// ---------------------------------------------------- mixed precision helpers
// FP32 copies of the operator on every level (Sec. 4.2 operator, stored once
// per Picard iteration for the FP32 V-cycles)
__global__ void k_to_f32_op(const int32_t* __restrict__ list, int n, int ncell,
                            const double* __restrict__ Tx, const double* __restrict__ Tz,
                            const double* __restrict__ D, float* Tx32, float* Tz32, float* D32,
                            float* invD32) {
    int s, q;
    if (!flat(list, n, ncell, s, q)) return;
    size_t P = (size_t)s * ncell + q;
    float d = (float)D[P];
    Tx32[P] = (float)Tx[P]; Tz32[P] = (float)Tz[P]; D32[P] = d; invD32[P] = 1.0f / d;
}

// FP64 defect r = f - A dp and its FP32 copy as the right-hand side of the
// FP32 V-cycle, with ||r||_inf per sample; the FP32 correction restarts at 0
__global__ void __launch_bounds__(RED_TPB)
k_defect(const int32_t* __restrict__ list, int bps, int nx, int nz,
         const double* __restrict__ Tx, const double* __restrict__ Tz, const double* __restrict__ D,
         const double* __restrict__ f, const double* __restrict__ dp, float* f32, float* e32,
         unsigned long long* nrm) {
    const int slot = blockIdx.x / bps, chunk = blockIdx.x - slot * bps;
    const int s = list[slot];
    const int ncell = nx * nz;
    const size_t base = (size_t)s * ncell;
    const int q0 = chunk * RED_CHUNK, q1 = min(ncell, q0 + RED_CHUNK);
    unsigned long long m = 0;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int j = q / nx, i = q - j * nx;
        size_t P = base + q;
        double r = f[P] - (D[P] * dp[P] - offdiag(Tx, Tz, dp, P, i, j, nx, nz));
        f32[P] = (float)r;
        e32[P] = 0.0f;
        unsigned long long b = abs_bits(r);
        m = b > m ? b : m;
    }
    block_max_atomic(m, &nrm[s]);
}

// dp += e (FP32 correction added in FP64)
__global__ void k_add_correction(const int32_t* __restrict__ list, int n, int ncell,
                                 const float* __restrict__ e, double* dp) {
    int s, q;
    if (!flat(list, n, ncell, s, q)) return;
    size_t P = (size_t)s * ncell + q;
    dp[P] += (double)e[P];
}

inline unsigned nblk(long long work, int tpb = TPB) { return (unsigned)((work + tpb - 1) / tpb); }

}  // namespace

// ============================================================== host side
int rich_count_levels(int nx, int nz) {
    if (nx < 1 || nz < 1) return -1;
    int n = 1;
    while (nx % 2 == 0 && nz % 2 == 0 && nx * nz > 4) { nx /= 2; nz /= 2; ++n; }
    if (n > RICH_MAX_LEVELS) return -1;
    return (nx * nz <= 64) ? n : -1;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int rich_ws_reserve(rich_ctx* ctx, int S, int nx, int nz, int mixed) {
    rich_ws& w = ctx->ws;
    if (w.base && w.S_cap >= S && w.nx == nx && w.nz == nz && w.mixed >= mixed) return 0;
    if (w.base) { cudaFree(w.base); w.base = nullptr; }
    if (w.h_counters) { cudaFreeHost(w.h_counters); w.h_counters = nullptr; }
    int nlev = rich_count_levels(nx, nz);
    if (nlev < 1) return RICH_ERR_INVALID;
    const size_t Sz = (size_t)std::max(S, 1);
    // plan
    size_t off = 0;
    std::vector<std::pair<void**, size_t>> plan;
    auto add = [&](void** ptr, size_t bytes) { plan.push_back({ptr, off}); off = align_up(off + bytes); };
    int lx = nx, lz = nz;
    for (int l = 0; l < nlev; ++l) {
        rich_level& L = w.lev[l];
        L = rich_level{};
        L.nx = lx; L.nz = lz;
        size_t nc = Sz * lx * lz * sizeof(double);
        add((void**)&L.Tx, nc); add((void**)&L.Tz, nc); add((void**)&L.Cdt, nc);
        add((void**)&L.D, nc); add((void**)&L.invD, nc); add((void**)&L.f, nc); add((void**)&L.dp, nc);
        add((void**)&L.Tbt, Sz * lx * sizeof(double)); add((void**)&L.Tbb, Sz * lx * sizeof(double));
        if (mixed) {
            size_t n4 = Sz * lx * lz * sizeof(float);
            add((void**)&L.Tx32, n4); add((void**)&L.Tz32, n4); add((void**)&L.D32, n4);
            add((void**)&L.invD32, n4); add((void**)&L.f32, n4); add((void**)&L.dp32, n4);
        }
        lx /= 2; lz /= 2;
    }
    size_t nc0 = Sz * nx * nz * sizeof(double);
    add((void**)&w.p, nc0); add((void**)&w.thold, nc0); add((void**)&w.Ks, nc0);
    add((void**)&w.a, nc0); add((void**)&w.K, nc0); add((void**)&w.th, nc0);
    add((void**)&w.h_in, 2 * nc0 + Sz * nx * nz * sizeof(double) + 2 * Sz * sizeof(double));
    add((void**)&w.status, Sz * 4); add((void**)&w.kpic, Sz * 4); add((void**)&w.cyc, Sz * 4);
    add((void**)&w.alive, Sz * 4); add((void**)&w.maxpic, Sz * 4);
    add((void**)&w.pic_total, Sz * 8); add((void**)&w.mg_total, Sz * 8);
    add((void**)&w.nrm_f, Sz * 8); add((void**)&w.nrm_r, Sz * 8); add((void**)&w.nrm_dp, Sz * 8);
    add((void**)&w.target, Sz * 8);
    add((void**)&w.list_pic, Sz * 4); add((void**)&w.list_mg, Sz * 4); add((void**)&w.list_tmp, Sz * 4);
    add((void**)&w.counters, 64);
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, off);
    if (e != cudaSuccess) { cudaGetLastError(); w.base = nullptr; w.S_cap = 0; return RICH_ERR_OOM; }
    for (auto& pr : plan) *pr.first = (char*)base + pr.second;
    w.base = base; w.bytes = off; w.S_cap = (int)Sz; w.nx = nx; w.nz = nz; w.nlev = nlev;
    w.mixed = mixed;
    RICH_CUDA(cudaMallocHost((void**)&w.h_counters, 64));
    return 0;
}

namespace {

#define KL(...) (rich_count_launch(), __VA_ARGS__)

struct Solver {
    rich_ctx* ctx;
    rich_ws& w;
    const rich_problem_t& pb;
    cudaStream_t st;
    int S;

    int read_counter(int k, int* out) {
        RICH_CUDA(cudaMemcpyAsync(w.h_counters + k, w.counters + k, sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, st));
        RICH_CUDA(cudaStreamSynchronize(st));
        *out = w.h_counters[k];
        return rich_prof_harvest(ctx);
    }
    int zero_counter(int k) {
        RICH_CUDA(cudaMemsetAsync(w.counters + k, 0, sizeof(int32_t), st));
        return 0;
    }

    // ---- V-cycle, generic in the working precision of the cycle
    template <typename T>
    void vcycle(int l, const int32_t* list, int n, bool mixed) {
        rich_level& L = w.lev[l];
        const T* Tx = mixed ? (const T*)L.Tx32 : (const T*)L.Tx;
        const T* Tz = mixed ? (const T*)L.Tz32 : (const T*)L.Tz;
        const T* D = mixed ? (const T*)L.D32 : (const T*)L.D;
        const T* invD = mixed ? (const T*)L.invD32 : (const T*)L.invD;
        T* f = mixed ? (T*)L.f32 : (T*)L.f;
        T* dp = mixed ? (T*)L.dp32 : (T*)L.dp;
        if (l == w.nlev - 1) {
            int nn = L.nx * L.nz;
            size_t sm = (size_t)nn * (nn + 1) * sizeof(T);
            KL(k_coarse_solve<T><<<n, 32, sm, st>>>(list, L.nx, L.nz, Tx, Tz, D, f, dp));
            return;
        }
        const long long wpair = (long long)n * (L.nx / 2) * L.nz;
        // algorithmic traffic of one colour pass: f, 1/D and the write of the
        // updated half, both face arrays, the other colour's dp once
        const double pb_bytes = (double)n * L.nx * L.nz * 4.0 * sizeof(T);
        const double pb_flops = (double)wpair * 9.0;
        auto smooth = [&](int nsweeps) {
            for (int it = 0; it < nsweeps; ++it)
                for (int c = 0; c < 2; ++c) {
                    if (l == 0) rich_prof_begin(ctx, st);
                    KL(k_rbgs<T><<<nblk(wpair), TPB, 0, st>>>(list, n, L.nx, L.nz, c, Tx, Tz, invD, f, dp));
                    if (l == 0) rich_prof_end(ctx, st, pb_bytes, pb_flops);
                }
        };
        smooth(pb.nu1);
        rich_level& Cl = w.lev[l + 1];
        T* fc = mixed ? (T*)Cl.f32 : (T*)Cl.f;
        T* dpc = mixed ? (T*)Cl.dp32 : (T*)Cl.dp;
        const long long wc = (long long)n * Cl.nx * Cl.nz;
        KL(k_resid_restrict<T><<<nblk(wc), TPB, 0, st>>>(list, n, Cl.nx, Cl.nz, Tx, Tz, D, f, dp, fc, dpc));
        vcycle<T>(l + 1, list, n, mixed);
        KL(k_prolong<T><<<nblk(wc), TPB, 0, st>>>(list, n, Cl.nx, Cl.nz, dpc, dp));
        smooth(pb.nu2);
    }

    int run(const double* lnKs, const double* alpha, double alpha_scale, double* qoi,
            double* p_final, int32_t* status_out) {
        const int nx = pb.nx, nz = pb.nz, ncell = nx * nz, nlev = w.nlev;
        const double h = 1.0 / nz, h2 = h * h, two_over_h2 = 2.0 / h2;
        const bool mixed = pb.precision == RICH_MIXED;
        const int bps = (ncell + RED_CHUNK - 1) / RED_CHUNK;
        KL(k_setup<<<nblk((long long)S * ncell), TPB, 0, st>>>(S, ncell, lnKs, alpha, alpha_scale,
                                                          pb.p_init, w.Ks, w.a, w.p));
        KL(k_setup_samples<<<nblk(S), TPB, 0, st>>>(S, w.status, w.alive, w.pic_total, w.mg_total,
                                                 w.maxpic, w.nrm_f, w.nrm_r, w.nrm_dp));
        KL(k_boundary_fine<<<nblk((long long)S * nx), TPB, 0, st>>>(S, nx, nz, w.Ks, w.a, two_over_h2,
                                                                pb.p_top, pb.p_bottom,
                                                                w.lev[0].Tbt, w.lev[0].Tbb));
        for (int l = 1; l < nlev; ++l)
            KL(k_boundary_coarsen<<<nblk((long long)S * w.lev[l].nx), TPB, 0, st>>>(
                S, w.lev[l].nx, w.lev[l - 1].Tbt, w.lev[l - 1].Tbb, w.lev[l].Tbt, w.lev[l].Tbb));
        RICH_CUDA(cudaGetLastError());
        rich_level& L0 = w.lev[0];
        for (int step = 0; step < pb.nsteps; ++step) {
            int np = 0;
            if (int e = zero_counter(0)) return e;
            KL(k_list_alive<<<nblk(S), TPB, 0, st>>>(S, w.alive, w.kpic, w.list_pic, w.counters + 0));
            if (int e = read_counter(0, &np)) return e;
            if (np == 0) break;
            KL(k_theta_old<<<nblk((long long)np * ncell), TPB, 0, st>>>(w.list_pic, np, ncell, w.a, w.p,
                                                                    pb.theta_r, pb.theta_s, w.thold));
            for (int it = 0; it < pb.picard_maxit && np > 0; ++it) {
                const long long wc = (long long)np * ncell;
                KL(k_conductivity<<<nblk(wc), TPB, 0, st>>>(w.list_pic, np, ncell, w.Ks, w.a, w.p,
                                                         pb.theta_r, pb.theta_s, pb.dt, w.K, w.th, L0.Cdt));
                KL(k_faces<<<nblk(wc), TPB, 0, st>>>(w.list_pic, np, nx, nz, w.K, two_over_h2, L0.Tx, L0.Tz));
                KL(k_rhs<<<(unsigned)np * bps, RED_TPB, 0, st>>>(w.list_pic, bps, nx, nz, w.p, w.th, w.thold,
                                                             L0.Tx, L0.Tz, L0.Tbt, L0.Tbb, L0.Cdt, pb.dt,
                                                             h, pb.p_top, pb.p_bottom, L0.f, L0.D,
                                                             L0.invD, w.nrm_f));
                for (int l = 1; l < nlev; ++l) {
                    rich_level& F = w.lev[l - 1];
                    rich_level& Cl = w.lev[l];
                    KL(k_coarsen<<<nblk((long long)np * Cl.nx * Cl.nz), TPB, 0, st>>>(
                        w.list_pic, np, Cl.nx, Cl.nz, F.Tx, F.Tz, F.Cdt, Cl.Tbt, Cl.Tbb, Cl.Tx, Cl.Tz,
                        Cl.Cdt, Cl.D, Cl.invD));
                }
                if (mixed)
                    for (int l = 0; l < nlev; ++l) {
                        rich_level& Lv = w.lev[l];
                        KL(k_to_f32_op<<<nblk((long long)np * Lv.nx * Lv.nz), TPB, 0, st>>>(
                            w.list_pic, np, Lv.nx * Lv.nz, Lv.Tx, Lv.Tz, Lv.D, Lv.Tx32, Lv.Tz32,
                            Lv.D32, Lv.invD32));
                    }
                KL(k_zero<<<nblk(wc), TPB, 0, st>>>(w.list_pic, np, ncell, L0.dp));
                int nm = 0;
                if (int e = zero_counter(1)) return e;
                KL(k_mg_start<<<nblk(np), TPB, 0, st>>>(w.list_pic, np, pb.mg_tol, w.nrm_f, w.target, w.cyc,
                                                     w.status, w.alive, w.list_mg, w.counters + 1));
                if (int e = read_counter(1, &nm)) return e;
                if (mixed && nm > 0)   // first FP32 right-hand side: the defect of dp = 0 is f
                    KL(k_defect<<<(unsigned)nm * bps, RED_TPB, 0, st>>>(
                        w.list_mg, bps, nx, nz, L0.Tx, L0.Tz, L0.D, L0.f, L0.dp, L0.f32, L0.dp32,
                        w.nrm_dp));
                for (int c = 0; c < pb.mg_maxit && nm > 0; ++c) {
                    if (!mixed) {
                        vcycle<double>(0, w.list_mg, nm, false);
                        KL(k_resid_norm<double><<<(unsigned)nm * bps, RED_TPB, 0, st>>>(
                            w.list_mg, bps, nx, nz, L0.Tx, L0.Tz, L0.D, L0.f, L0.dp, w.nrm_r));
                    } else {
                        // FP32 V-cycle on the FP32 defect, FP64 correction, then the FP64
                        // defect (stopping norm and the next FP32 right-hand side)
                        vcycle<float>(0, w.list_mg, nm, true);
                        KL(k_add_correction<<<nblk((long long)nm * ncell), TPB, 0, st>>>(
                            w.list_mg, nm, ncell, L0.dp32, L0.dp));
                        KL(k_defect<<<(unsigned)nm * bps, RED_TPB, 0, st>>>(
                            w.list_mg, bps, nx, nz, L0.Tx, L0.Tz, L0.D, L0.f, L0.dp, L0.f32, L0.dp32,
                            w.nrm_r));
                    }
                    if (int e = zero_counter(2)) return e;
                    KL(k_mg_decide<<<nblk(nm), TPB, 0, st>>>(w.list_mg, nm, pb.mg_maxit, w.nrm_r, w.target,
                                                          w.cyc, w.mg_total, w.status, w.alive,
                                                          w.list_tmp, w.counters + 2));
                    if (int e = read_counter(2, &nm)) return e;
                    std::swap(w.list_mg, w.list_tmp);
                }
                if (mixed) {   // the defect norm slot doubles as scratch in the mixed loop
                    RICH_CUDA(cudaMemsetAsync(w.nrm_dp, 0, sizeof(unsigned long long) * S, st));
                }
                KL(k_update_p<<<(unsigned)np * bps, RED_TPB, 0, st>>>(w.list_pic, bps, ncell, w.alive,
                                                                   L0.dp, w.p, w.nrm_dp));
                if (int e = zero_counter(2)) return e;
                KL(k_picard_decide<<<nblk(np), TPB, 0, st>>>(w.list_pic, np, pb.picard_maxit, pb.picard_tol,
                                                          w.nrm_dp, w.kpic, w.pic_total, w.maxpic,
                                                          w.status, w.alive, w.list_tmp, w.counters + 2));
                if (int e = read_counter(2, &np)) return e;
                std::swap(w.list_pic, w.list_tmp);
            }
        }
        KL(k_qoi<<<S, 32, 0, st>>>(S, nx, nz, w.Ks, w.a, w.p, pb.p_bottom, h, w.alive, qoi));
        if (p_final)
            RICH_CUDA(cudaMemcpyAsync(p_final, w.p, sizeof(double) * (size_t)S * ncell,
                                      cudaMemcpyDeviceToDevice, st));
        if (status_out)
            RICH_CUDA(cudaMemcpyAsync(status_out, w.status, sizeof(int32_t) * S,
                                      cudaMemcpyDeviceToDevice, st));
        RICH_CUDA(cudaGetLastError());
        return 0;
    }
};

}  // namespace

int rich_solve_device(rich_ctx* ctx, const rich_problem_t* pb, int S, const double* lnKs,
                      const double* alpha, double alpha_scale, double* qoi, double* p_final,
                      int32_t* status, rich_stats_t* stats, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    int e = rich_ws_reserve(ctx, S, pb->nx, pb->nz, pb->precision == RICH_MIXED);
    if (e) return e;
    rich_ws& w = ctx->ws;
    if (w.lev[w.nlev - 1].nx * w.lev[w.nlev - 1].nz > 64) return RICH_ERR_INVALID;
    static const char* which = getenv("RICH_SOLVER");
    const bool batched = which && strcmp(which, "batched") == 0;
    if (batched) {
        Solver sv{ctx, w, *pb, st, S};
        e = sv.run(lnKs, alpha, alpha_scale, qoi, p_final, status);
    } else {
        e = rich_solve_fused(ctx, pb, S, lnKs, alpha, alpha_scale, qoi, p_final, status, st);
    }
    if (e) return e;
    // worst status and counters (host)
    std::vector<int32_t> hs(S), hmax(S);
    std::vector<int64_t> hp(S), hm(S);
    RICH_CUDA(cudaMemcpyAsync(hs.data(), w.status, 4 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hmax.data(), w.maxpic, 4 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hp.data(), w.pic_total, 8 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaMemcpyAsync(hm.data(), w.mg_total, 8 * (size_t)S, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaStreamSynchronize(st));
    int worst = 0;
    rich_stats_t acc{};
    for (int s = 0; s < S; ++s) {
        worst = std::max(worst, (int)hs[s]);
        acc.picard_iters += hp[s];
        acc.mg_cycles += hm[s];
        acc.max_picard = std::max(acc.max_picard, hmax[s]);
        if (hs[s] == RICH_PICARD_MAXIT || hs[s] == RICH_NONFINITE) acc.failed++;
    }
    acc.cell_vcycles = acc.mg_cycles * (int64_t)pb->nx * pb->nz;
    if (!batched) {
        // algorithmic work of the fused launch: per fine cell and V-cycle 74 flops
        // and 16.7 words (two fused passes per level, hierarchy factor 4/3); per
        // Picard iteration 56 flops and 10 words per fine cell (assembly, coarse
        // operators, update)
        const double nc = (double)pb->nx * pb->nz;
        const double w8 = pb->precision == RICH_MIXED ? 4.0 : 8.0;
        const double flops = nc * (74.0 * acc.mg_cycles + 56.0 * acc.picard_iters);
        const double bytes = nc * (16.7 * w8 * acc.mg_cycles + 10.0 * 8.0 * acc.picard_iters);
        rich_prof_amend(ctx, bytes, flops);
    }
    acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = acc;
    return worst;
}
