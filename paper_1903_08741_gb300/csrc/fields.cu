// Random soil fields by FFT moving average (arXiv 1903.08741, Appendix A):
// white noise y on a periodic px x pz torus, z = F^-1( sqrt(F c) . F y ), keep
// the physical window, then ln Ks = z_0 and alpha = lo + span * Phi(z_1 / sigma).
//
// GPU design: the two real fields of a sample are packed into one complex
// transform (re = y_0, im = y_1); sqrt(F c) is real and even, so the filter maps
// real inputs to real outputs and the two fields come back in re / im.  The 2-D
// FFT is two passes of batched 1-D radix-2 transforms in shared memory (rows,
// then groups of adjacent columns so that global accesses stay coalesced).
// White noise: Philox4x32-10 (Salmon et al., SC'11) implemented from its
// definition, key = (seed low word, seed high word ^ level), counter = (cell
// pair, field, sample low, sample high), two uniforms -> Box-Muller.
#include "rich_internal.cuh"
#include <math.h>
#include <vector>
#include <algorithm>

namespace {

struct cplx { double re, im; };

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__device__ __forceinline__ double u01(uint32_t hi, uint32_t lo) {
    unsigned long long m = (((unsigned long long)hi << 32) | lo) >> 11;
    return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

// packed complex white noise: re = field fld0, im = field fld0 + 1, for
// samples first..first+S-1 on the torus (npts = px*pz, even)
// (first sample = *first_dev + first when first_dev is given: a captured CUDA
// graph can advance the sample range between replays)
__global__ void k_noise(int S, int npts, uint64_t seed, uint32_t level, int64_t first,
                        const int64_t* __restrict__ first_dev, cplx* out, uint32_t fld0 = 0) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (sample, pair)
    const int pairs = npts >> 1;
    if (g >= (long long)S * pairs) return;
    int s = (int)(g / pairs), q = (int)(g - (long long)s * pairs);
    uint64_t sample = (uint64_t)((first_dev ? *first_dev : 0) + first + s);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ level;
    double y[2][2];
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
        uint32_t c[4] = {(uint32_t)q, fld0 + (uint32_t)fld, (uint32_t)sample, (uint32_t)(sample >> 32)};
        philox10(c, k0, k1);
        double a = u01(c[0], c[1]), b = u01(c[2], c[3]);
        double r = sqrt(-2.0 * log(a));
        double sn, cs;
        sincos(6.283185307179586476925286766559 * b, &sn, &cs);
        y[fld][0] = r * cs; y[fld][1] = r * sn;
    }
    cplx* o = out + (size_t)s * npts + 2 * (size_t)q;
    o[0] = cplx{y[0][0], y[1][0]};
    o[1] = cplx{y[0][1], y[1][1]};
}

// twiddles w_k = exp(-2 pi i k / n), k < n/2
__global__ void k_twiddles(int n, cplx* tw) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n / 2) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    tw[k] = cplx{c, s};
}

// Batched radix-2 FFT of lines of length n (power of two) held in shared
// memory.  A block handles LPB lines; line l of sample b starts at
// b*sample_stride + l*line_stride, its elements are elem_stride apart.
// Bit-reversed load, log2(n) butterfly stages, 1/n on the inverse.
template <int LPB>
__global__ void k_fft_lines(cplx* data, int n, int logn, int lines, long long sample_stride,
                            int line_stride, int elem_stride, const cplx* __restrict__ tw,
                            int inverse) {
    // contiguous lines: consecutive threads take consecutive elements; strided
    // lines (columns): consecutive threads take adjacent lines
    const bool contig = elem_stride == 1;
    extern __shared__ cplx sh[];
    const int groups = lines / LPB;
    const int b = blockIdx.x / groups, g = blockIdx.x - b * groups;
    cplx* base = data + (size_t)b * sample_stride + (size_t)g * LPB * line_stride;
    const int tid = threadIdx.x, nt = blockDim.x;
    // load: element e of line l -> shared [l][rev(e)]; consecutive threads read
    // consecutive lines first so that column groups coalesce
    for (int t = tid; t < n * LPB; t += nt) {
        int l = contig ? t / n : t % LPB, e = contig ? t - (t / n) * n : t / LPB;
        int r = logn ? (int)(__brev((unsigned)e) >> (32 - logn)) : 0;
        sh[l * n + r] = base[(size_t)l * line_stride + (size_t)e * elem_stride];
    }
    __syncthreads();
    const double sgn = inverse ? -1.0 : 1.0;
    for (int m = 1, st = n >> 1; m < n; m <<= 1, st >>= 1) {
        for (int t = tid; t < (n >> 1) * LPB; t += nt) {
            int l = t / (n >> 1), bf = t - l * (n >> 1);
            int grp = bf / m, k = bf - grp * m;
            int a = grp * 2 * m + k, c = a + m;
            cplx w = tw[k * st];
            double wi = sgn * w.im;
            cplx x = sh[l * n + c], y = sh[l * n + a];
            double xr = x.re * w.re - x.im * wi;
            double xi = x.re * wi + x.im * w.re;
            sh[l * n + c] = cplx{y.re - xr, y.im - xi};
            sh[l * n + a] = cplx{y.re + xr, y.im + xi};
        }
        __syncthreads();
    }
    const double sc = inverse ? 1.0 / (double)n : 1.0;
    for (int t = tid; t < n * LPB; t += nt) {
        int l = contig ? t / n : t % LPB, e = contig ? t - (t / n) * n : t / LPB;
        cplx v = sh[l * n + e];
        if (inverse) { v.re *= sc; v.im *= sc; }
        base[(size_t)l * line_stride + (size_t)e * elem_stride] = v;
    }
}

__global__ void k_filter(int S, int npts, const double* __restrict__ sq, cplx* d) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)S * npts) return;
    double w = sq[g % npts];
    d[g].re *= w; d[g].im *= w;
}

// covariance model of one spectrum: nu = 0 exponential sigma2 exp(-r);
// nu > 0 the Matern function of Eq. nonIsotropic, norm = sigma2 2^(1-nu)/Gamma(nu)
struct CovModel {
    double sigma2, lx, lz, nu, norm;
};

// K_nu(x) for x > 0 from K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
// (DLMF 10.32.9): trapezoidal sum, geometrically convergent for this
// analytic, doubly exponentially decaying integrand; the step resolves the
// exp(-x t^2/2) peak at large x (min(1/16, 1/(2 sqrt x))), the sum ends past
// the integrand's maximum once a term adds less than 1e-18 (at most 4095 terms)
__device__ double bessel_k(double nu, double x) {
    const double dt = x > 64.0 ? 0.5 / sqrt(x) : 0.0625;
    double acc = 0.5 * exp(-x);
    for (int k = 1; k < 4096; ++k) {
        const double t = k * dt;
        const double f = exp(-x * cosh(t)) * cosh(nu * t);
        acc += f;
        if (f <= 1e-18 * acc && x * sinh(t) > nu) break;
    }
    return dt * acc;
}

// covariance on the torus at the periodic offset of point (a, b)
__global__ void k_cov(int px, int pz, double h, CovModel cm, cplx* c) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= px * pz) return;
    int b = g / px, a = g - b * px;
    int ia = min(a, px - a), ib = min(b, pz - b);
    double dx = ia * h, dz = ib * h;
    const double r = cm.lz == cm.lx ? sqrt(dx * dx + dz * dz) / cm.lx
                                    : sqrt((dx / cm.lx) * (dx / cm.lx) + (dz / cm.lz) * (dz / cm.lz));
    double v;
    if (cm.nu == 0.0) v = cm.sigma2 * exp(-r);
    else if (r == 0.0) v = cm.sigma2;
    else {
        const double x = 2.0 * sqrt(cm.nu) * r;
        v = cm.norm * pow(x, cm.nu) * bessel_k(cm.nu, x);
    }
    c[g] = cplx{v, 0.0};
}

__global__ void k_sqrt_spec(int npts, const cplx* __restrict__ lam, double* sq) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npts) return;
    double v = lam[g].re;
    sq[g] = v > 0.0 ? sqrt(v) : 0.0;
}

// marginal transforms of a packed pair: the re lane is Gaussian (shift + z,
// ln Ks) or uniform, the im lane uniform: lo + span Phi(z / sigma) with
// Phi(x) = erfc(-x/sqrt 2)/2 (Y = F_Y^-1(F_Z(Z)), Sec. 3.1)
struct PackTr {
    int re_uniform;
    double re_a, re_b;      // Gaussian: shift re_a; uniform: lo re_a, span re_b
    double im_lo, im_span;
};

__device__ __forceinline__ double uniform_of(double z, double inv_sigma, double lo, double span) {
    double gg = z * inv_sigma;
    return lo + span * 0.5 * erfc(-gg / sqrt(2.0));
}

// window of the torus -> the pair's two fields, in place into a compact
// [S][nz][nx] pair of real arrays (al may be null: the im lane is unused)
__global__ void k_window(int S, int nx, int nz, int px, int pz, const cplx* __restrict__ d,
                         double inv_sigma, PackTr tr, double* lk, double* al) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = nx * nz;
    if (g >= (long long)S * nc) return;
    int s = (int)(g / nc), q = (int)(g - (long long)s * nc);
    int j = q / nx, i = q - j * nx;
    cplx v = d[(size_t)s * px * pz + (size_t)j * px + i];
    lk[g] = tr.re_uniform ? uniform_of(v.re, inv_sigma, tr.re_a, tr.re_b) : v.re + tr.re_a;
    if (al) al[g] = uniform_of(v.im, inv_sigma, tr.im_lo, tr.im_span);
}

// one 2x2 averaging step of both fields
__global__ void k_avg2(int S, int nxc, int nzc, const double* __restrict__ lf,
                       const double* __restrict__ af, double* lc, double* ac) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = nxc * nzc, fx = 2 * nxc;
    if (g >= (long long)S * nc) return;
    int s = (int)(g / nc), q = (int)(g - (long long)s * nc);
    int J = q / nxc, I = q - J * nxc;
    size_t f00 = (size_t)s * 4 * nc + (size_t)(2 * J) * fx + 2 * I, f01 = f00 + fx;
    lc[g] = 0.25 * (lf[f00] + lf[f00 + 1] + lf[f01] + lf[f01 + 1]);
    if (ac) ac[g] = 0.25 * (af[f00] + af[f00 + 1] + af[f01] + af[f01 + 1]);
}

inline unsigned nb(long long w, int t = 256) { return (unsigned)((w + t - 1) / t); }
inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
inline bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

template <int L>
int fft_pass(cplx* d, int S, int n, int lines, long long sstride, int lstride, int estride,
             const cplx* tw, int inverse, cudaStream_t st) {
    size_t sm = (size_t)L * n * sizeof(cplx);
    RICH_CUDA(cudaFuncSetAttribute(k_fft_lines<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    rich_count_launch();
    k_fft_lines<L><<<(unsigned)S * (lines / L), 256, sm, st>>>(d, n, ilog2(n), lines, sstride, lstride,
                                                               estride, tw, inverse);
    return 0;
}

// lines per block: the largest of 8, 4, 2, 1 that divides the line count and
// keeps the block's lines within 128 KB of shared memory
int fft_dispatch(cplx* d, int S, int n, int lines, long long sstride, int lstride, int estride,
                 const cplx* tw, int inverse, cudaStream_t st) {
    for (int L = 8; L >= 1; L >>= 1) {
        if (lines % L || (size_t)L * n * sizeof(cplx) > (128u << 10)) continue;
        switch (L) {
            case 8: return fft_pass<8>(d, S, n, lines, sstride, lstride, estride, tw, inverse, st);
            case 4: return fft_pass<4>(d, S, n, lines, sstride, lstride, estride, tw, inverse, st);
            case 2: return fft_pass<2>(d, S, n, lines, sstride, lstride, estride, tw, inverse, st);
            default: return fft_pass<1>(d, S, n, lines, sstride, lstride, estride, tw, inverse, st);
        }
    }
    return RICH_ERR_INVALID;
}

int fft2(cplx* d, int S, int px, int pz, const cplx* twx, const cplx* twz, int inverse,
         cudaStream_t st) {
    const long long ss = (long long)px * pz;
    if (int e = fft_dispatch(d, S, px, pz, ss, px, 1, twx, inverse, st)) return e;   // rows (x)
    if (int e = fft_dispatch(d, S, pz, px, ss, 1, px, twz, inverse, st)) return e;   // columns (z)
    RICH_CUDA(cudaGetLastError());
    return 0;
}

}  // namespace

// ---------------------------------------------------------------- host side
// a field model outside the supported range: sigma2, corr_len > 0,
// corr_len_z >= 0 (0: isotropic), 0 <= nu <= 16
bool bad_field(const rich_field_t* fd) {
    return !(fd->sigma2 > 0) || !(fd->corr_len > 0) || !(fd->corr_len_z >= 0) || !(fd->nu >= 0) ||
           !(fd->nu <= 16);
}

// sqrt(F c) on a px x pz torus of spacing h, cached in the context
static int spectrum_on(rich_ctx* ctx, int px, int pz, double h, const rich_field_t* fd,
                       cudaStream_t st, const rich_spectrum** out, double* min_ratio) {
    const double sigma2 = fd->sigma2, corr_len = fd->corr_len, nu = fd->nu;
    const double lz = fd->corr_len_z > 0 ? fd->corr_len_z : fd->corr_len;
    for (const rich_spectrum& e : ctx->spectra)
        if (e.px == px && e.pz == pz && e.h == h && e.sigma2 == sigma2 && e.corr_len == corr_len &&
            e.corr_len_z == lz && e.nu == nu) {
            *out = &e;
            if (min_ratio) *min_ratio = e.min_ratio;
            return 0;
        }
    const int npts = px * pz;
    rich_spectrum e{};
    e.px = px; e.pz = pz; e.h = h; e.sigma2 = sigma2; e.corr_len = corr_len; e.corr_len_z = lz; e.nu = nu;
    const CovModel cm{sigma2, corr_len, lz, nu, nu > 0 ? sigma2 * pow(2.0, 1.0 - nu) / tgamma(nu) : 0.0};
    cplx* c = nullptr;
    RICH_CUDA(cudaMalloc(&c, sizeof(cplx) * npts));
    RICH_CUDA(cudaMalloc(&e.tw, sizeof(cplx) * (px / 2 + pz / 2 + 2)));
    cplx* tw = (cplx*)e.tw;
    rich_count_launch(); k_twiddles<<<nb(px / 2), 256, 0, st>>>(px, tw);
    rich_count_launch(); k_twiddles<<<nb(pz / 2), 256, 0, st>>>(pz, tw + px / 2 + 1);
    rich_count_launch(); k_cov<<<nb(npts), 256, 0, st>>>(px, pz, h, cm, c);
    if (int r = fft2(c, 1, px, pz, tw, tw + px / 2 + 1, 0, st)) { cudaFree(c); return r; }
    std::vector<cplx> hl(npts);
    RICH_CUDA(cudaMemcpyAsync(hl.data(), c, sizeof(cplx) * npts, cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaStreamSynchronize(st));
    double lmin = hl[0].re, lmax = hl[0].re;
    for (auto& v : hl) { lmin = std::min(lmin, v.re); lmax = std::max(lmax, v.re); }
    e.min_ratio = lmin / lmax;
    RICH_CUDA(cudaMalloc(&e.sq, sizeof(double) * npts));
    rich_count_launch(); k_sqrt_spec<<<nb(npts), 256, 0, st>>>(npts, c, e.sq);
    RICH_CUDA(cudaStreamSynchronize(st));
    cudaFree(c);
    if (ctx->spectra.size() >= 16) {               // bounded cache: drop the oldest
        cudaFree(ctx->spectra.front().sq); cudaFree(ctx->spectra.front().tw);
        ctx->spectra.erase(ctx->spectra.begin());
    }
    ctx->spectra.push_back(e);
    *out = &ctx->spectra.back();
    if (min_ratio) *min_ratio = e.min_ratio;
    return 0;
}

// smallest power-of-two torus of at least twice the grid per side whose
// circulant spectrum has no eigenvalue below -1e-12 max (doubled up to 3 times)
static int choose_torus(rich_ctx* ctx, int nx, int nz, const rich_field_t* fd, cudaStream_t st,
                        int* px, int* pz) {
    const double h = 1.0 / nz;
    int a = 1, b = 1;
    while (a < 2 * nx) a <<= 1;
    while (b < 2 * nz) b <<= 1;
    for (int tries = 0; tries < 4; ++tries) {
        const rich_spectrum* e = nullptr;
        double ratio = 0;
        if (int r = spectrum_on(ctx, a, b, h, fd, st, &e, &ratio)) return r;
        if (ratio >= -1e-12 || tries == 3) { *px = a; *pz = b; return 0; }
        a *= 2; b *= 2;
    }
    return RICH_ERR_INVALID;
}

static int ensure_work(rich_ctx* ctx, size_t bytes) {
    if (ctx->field_work && ctx->field_work_bytes >= bytes) return 0;
    if (ctx->field_work) cudaFree(ctx->field_work);
    ctx->field_work = nullptr; ctx->field_work_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->field_work, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return RICH_ERR_OOM; }
    ctx->field_work_bytes = bytes;
    return 0;
}

// FFT-MA of the packed noise in `work` ([cs][pz][px] complex) in place
static int fftma_inplace(cplx* work, int cs, const rich_spectrum* sp, cudaStream_t st) {
    const int px = sp->px, pz = sp->pz, npts = px * pz;
    const cplx* twx = (const cplx*)sp->tw;
    const cplx* twz = twx + px / 2 + 1;
    if (int e = fft2(work, cs, px, pz, twx, twz, 0, st)) return e;
    rich_count_launch();
    k_filter<<<nb((long long)cs * npts), 256, 0, st>>>(cs, npts, sp->sq, work);
    if (int e = fft2(work, cs, px, pz, twx, twz, 1, st)) return e;
    return 0;
}

constexpr size_t CHUNK_BYTES = 512ull << 20;

// one packed pair of fields: noise streams fld0, fld0 + 1, their marginal
// transforms and [S][nz>>c][nx>>c] outputs (out_im null: im lane unused)
struct Pack {
    uint32_t fld0;
    PackTr tr;
    double* out_re;
    double* out_im;
};

// FFT-MA draws of npk packed pairs per sample, chunked over samples so the
// complex work buffer stays within CHUNK_BYTES
static int packs_device(rich_ctx* ctx, const rich_field_t* fd, int nx, int nz, uint32_t level,
                        int64_t first, int S, int coarsen, int npk, const Pack* pk, cudaStream_t st,
                        const int64_t* first_dev) {
    if (!pow2(nx) || !pow2(nz) || coarsen < 0 || (nx >> coarsen) < 1 || (nz >> coarsen) < 1 ||
        bad_field(fd))
        return RICH_ERR_INVALID;
    if (S == 0) return 0;
    int px = 0, pz = 0;
    if (int e = choose_torus(ctx, nx, nz, fd, st, &px, &pz)) return e;
    const rich_spectrum* sp = nullptr;
    if (int e = spectrum_on(ctx, px, pz, 1.0 / nz, fd, st, &sp, nullptr)) return e;
    const int npts = px * pz;
    const size_t per = (size_t)npts * sizeof(cplx) + 32 * (size_t)nx * nz;
    const int chunk = (int)std::max<size_t>(1, CHUNK_BYTES / per);
    if (int e = ensure_work(ctx, per * std::min(chunk, S))) return e;
    cplx* work = (cplx*)ctx->field_work;
    const int cap = std::min(chunk, S);
    double* tmp = (double*)(work + (size_t)npts * cap);   // [cap][4][nz][nx] real scratch
    const int nxo = nx >> coarsen, nzo = nz >> coarsen;
    const double inv_sigma = 1.0 / sqrt(fd->sigma2);
    for (int s0 = 0; s0 < S; s0 += cap) {
        int cs = std::min(cap, S - s0);
        for (int k = 0; k < npk; ++k) {
            const Pack& P = pk[k];
            rich_count_launch();
            k_noise<<<nb((long long)cs * (npts / 2)), 256, 0, st>>>(cs, npts, fd->seed, level, first + s0,
                                                                     first_dev, work, P.fld0);
            if (int e = fftma_inplace(work, cs, sp, st)) return e;
            // real scratch: two ping-pong pairs of [cs][nz][nx] arrays
            const size_t blk = (size_t)cs * nx * nz;
            double* bl[2] = {tmp, tmp + 2 * blk};
            double* ba[2] = {tmp + blk, tmp + 3 * blk};
            const bool im = P.out_im != nullptr;
            double* wl = coarsen ? bl[0] : P.out_re + (size_t)s0 * nx * nz;
            double* wa = !im ? nullptr : coarsen ? ba[0] : P.out_im + (size_t)s0 * nx * nz;
            rich_count_launch();
            k_window<<<nb((long long)cs * nx * nz), 256, 0, st>>>(cs, nx, nz, px, pz, work, inv_sigma, P.tr,
                                                                wl, wa);
            int cx = nx, cz = nz, cur = 0;
            for (int c = 0; c < coarsen; ++c) {
                int ncx = cx / 2, ncz = cz / 2;
                bool last = c == coarsen - 1;
                double* ol = last ? P.out_re + (size_t)s0 * nxo * nzo : bl[1 - cur];
                double* oa = !im ? nullptr : last ? P.out_im + (size_t)s0 * nxo * nzo : ba[1 - cur];
                rich_count_launch();
                k_avg2<<<nb((long long)cs * ncx * ncz), 256, 0, st>>>(cs, ncx, ncz, bl[cur], im ? ba[cur] : nullptr,
                                                                       ol, oa);
                cur = 1 - cur;
                cx = ncx; cz = ncz;
            }
        }
    }
    RICH_CUDA(cudaGetLastError());
    return 0;
}

int rich_fields_device(rich_ctx* ctx, const rich_field_t* fd, int nx, int nz, uint32_t level,
                       int64_t first, int S, int coarsen, double* lnKs, double* alpha,
                       cudaStream_t st, const int64_t* first_dev) {
    const Pack pk{0u, PackTr{0, 0.0, 0.0, fd->alpha_lo, fd->alpha_span}, lnKs, alpha};
    return packs_device(ctx, fd, nx, nz, level, first, S, coarsen, 1, &pk, st, first_dev);
}

// The five soil fields (Table soilparams): streams 0/1 ln Ks (lnks_mean + Z)
// and alpha, 2/3 n and theta_s, 4 theta_r (the im lane of the last pack
// unused); theta fields are skipped when their outputs are null
int rich_soil_device(rich_ctx* ctx, const rich_field_t* fd, const rich_soil_model_t* sm, int nx, int nz,
                     uint32_t level, int64_t first, int S, int coarsen, const rich_soil_t* out,
                     cudaStream_t st) {
    if (!(sm->n_span >= 0) || !(sm->theta_s_span >= 0) || !(sm->theta_r_span >= 0) ||
        !(sm->lnks_mean > -700 && sm->lnks_mean < 700))
        return RICH_ERR_INVALID;
    Pack pk[3];
    int npk = 0;
    pk[npk++] = Pack{0u, PackTr{0, sm->lnks_mean, 0.0, fd->alpha_lo, fd->alpha_span}, out->lnKs, out->alpha};
    if (out->theta_s)
        pk[npk++] = Pack{2u, PackTr{1, sm->n_lo, sm->n_span, sm->theta_s_lo, sm->theta_s_span}, out->n, out->theta_s};
    else
        pk[npk++] = Pack{2u, PackTr{1, sm->n_lo, sm->n_span, 0.0, 0.0}, out->n, nullptr};
    if (out->theta_r)
        pk[npk++] = Pack{4u, PackTr{1, sm->theta_r_lo, sm->theta_r_span, 0.0, 0.0}, out->theta_r, nullptr};
    return packs_device(ctx, fd, nx, nz, level, first, S, coarsen, npk, pk, st, nullptr);
}

namespace {
// coarse white noise by 2x2 averaging on the torus, scaled by 1/2 so that it
// stays standard normal (Appendix A, Eq. averaging); both packed fields at once
__global__ void k_noise_upscale(int S, int pxc, int pzc, const cplx* __restrict__ y, cplx* yc) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = pxc * pzc, fx = 2 * pxc;
    if (g >= (long long)S * nc) return;
    int s = (int)(g / nc), q = (int)(g - (long long)s * nc);
    int J = q / pxc, I = q - J * pxc;
    const cplx* b = y + (size_t)s * 4 * nc + (size_t)(2 * J) * fx + 2 * I;
    cplx a = b[0], c = b[1], d = b[fx], e = b[fx + 1];
    yc[g] = cplx{0.5 * (a.re + c.re + d.re + e.re), 0.5 * (a.im + c.im + d.im + e.im)};
}
}

// one packed pair of fields drawn as a fine/coarse couple: outputs on the
// fine grid (f_*) and on the half grid (c_*); im outputs null: lane unused
struct PairPack {
    uint32_t fld0;
    PackTr tr;
    double *f_re, *f_im, *c_re, *c_im;
};

// Fine fields on nx x nz and coarse fields on (nx/2) x (nz/2) from one draw by
// covariance upscaling (Appendix A, Eqs. averaging, cov_upscale): the coarse
// white noise is half the 2x2 sums of the fine noise on the torus, filtered
// with the coarse grid's own spectrum on the half-size torus.
static int pair_packs_device(rich_ctx* ctx, const rich_field_t* fd, int nx, int nz, uint32_t level,
                             int64_t first, int S, int npk, const PairPack* pk, cudaStream_t st) {
    if (!pow2(nx) || !pow2(nz) || nx < 2 || nz < 2 || bad_field(fd))
        return RICH_ERR_INVALID;
    if (S == 0) return 0;
    int px = 0, pz = 0;
    if (int e = choose_torus(ctx, nx, nz, fd, st, &px, &pz)) return e;
    const rich_spectrum *spf = nullptr, *spc = nullptr;
    if (int e = spectrum_on(ctx, px, pz, 1.0 / nz, fd, st, &spf, nullptr)) return e;
    if (int e = spectrum_on(ctx, px / 2, pz / 2, 2.0 / nz, fd, st, &spc, nullptr)) return e;
    // spectrum_on may reallocate the cache vector: look both up again
    spectrum_on(ctx, px, pz, 1.0 / nz, fd, st, &spf, nullptr);
    spectrum_on(ctx, px / 2, pz / 2, 2.0 / nz, fd, st, &spc, nullptr);
    const int npf = px * pz, npc = npf / 4;
    const size_t per = (size_t)(npf + npc) * sizeof(cplx);
    const int cap = (int)std::min<size_t>((size_t)S, std::max<size_t>(1, CHUNK_BYTES / per));
    if (int e = ensure_work(ctx, per * cap)) return e;
    cplx* wf = (cplx*)ctx->field_work;
    cplx* wc = wf + (size_t)npf * cap;
    const double inv_sigma = 1.0 / sqrt(fd->sigma2);
    const int ncx = nx / 2, ncz = nz / 2;
    for (int s0 = 0; s0 < S; s0 += cap) {
        int cs = std::min(cap, S - s0);
        for (int k = 0; k < npk; ++k) {
            const PairPack& P = pk[k];
            rich_count_launch();
            k_noise<<<nb((long long)cs * (npf / 2)), 256, 0, st>>>(cs, npf, fd->seed, level, first + s0, nullptr,
                                                                    wf, P.fld0);
            rich_count_launch();
            k_noise_upscale<<<nb((long long)cs * npc), 256, 0, st>>>(cs, px / 2, pz / 2, wf, wc);
            if (int e = fftma_inplace(wf, cs, spf, st)) return e;
            if (int e = fftma_inplace(wc, cs, spc, st)) return e;
            rich_count_launch();
            k_window<<<nb((long long)cs * nx * nz), 256, 0, st>>>(
                cs, nx, nz, px, pz, wf, inv_sigma, P.tr, P.f_re + (size_t)s0 * nx * nz,
                P.f_im ? P.f_im + (size_t)s0 * nx * nz : nullptr);
            rich_count_launch();
            k_window<<<nb((long long)cs * ncx * ncz), 256, 0, st>>>(
                cs, ncx, ncz, px / 2, pz / 2, wc, inv_sigma, P.tr, P.c_re + (size_t)s0 * ncx * ncz,
                P.c_im ? P.c_im + (size_t)s0 * ncx * ncz : nullptr);
        }
    }
    RICH_CUDA(cudaGetLastError());
    return 0;
}

int rich_fields_pair_device(rich_ctx* ctx, const rich_field_t* fd, int nx, int nz, uint32_t level,
                            int64_t first, int S, double* lk_f, double* al_f, double* lk_c,
                            double* al_c, cudaStream_t st) {
    const PairPack pk{0u, PackTr{0, 0.0, 0.0, fd->alpha_lo, fd->alpha_span}, lk_f, al_f, lk_c, al_c};
    return pair_packs_device(ctx, fd, nx, nz, level, first, S, 1, &pk, st);
}

// the five soil fields as covariance-upscaled fine/coarse couples (theta
// outputs may be null: not drawn)
int rich_soil_pair_device(rich_ctx* ctx, const rich_field_t* fd, const rich_soil_model_t* sm, int nx, int nz,
                          uint32_t level, int64_t first, int S, const rich_soil_t* fine,
                          const rich_soil_t* coarse, cudaStream_t st) {
    PairPack pk[3];
    int npk = 0;
    pk[npk++] = PairPack{0u, PackTr{0, sm->lnks_mean, 0.0, fd->alpha_lo, fd->alpha_span}, fine->lnKs, fine->alpha,
                         coarse->lnKs, coarse->alpha};
    const bool ts = fine->theta_s && coarse->theta_s;
    pk[npk++] = PairPack{2u, PackTr{1, sm->n_lo, sm->n_span, ts ? sm->theta_s_lo : 0.0, ts ? sm->theta_s_span : 0.0},
                         fine->n, ts ? fine->theta_s : nullptr, coarse->n, ts ? coarse->theta_s : nullptr};
    if (fine->theta_r && coarse->theta_r)
        pk[npk++] = PairPack{4u, PackTr{1, sm->theta_r_lo, sm->theta_r_span, 0.0, 0.0}, fine->theta_r, nullptr,
                             coarse->theta_r, nullptr};
    return pair_packs_device(ctx, fd, nx, nz, level, first, S, npk, pk, st);
}

// 2x2 block means of both fields (the coarse member of an MLMC pair; al and
// alc may be null)
int rich_fields_average(rich_ctx* ctx, int S, int nx, int nz, const double* lk, const double* al,
                        double* lkc, double* alc, cudaStream_t st) {
    (void)ctx;
    if (nx % 2 || nz % 2) return RICH_ERR_INVALID;
    if (S == 0) return 0;
    const int ncx = nx / 2, ncz = nz / 2;
    rich_count_launch();
    k_avg2<<<nb((long long)S * ncx * ncz), 256, 0, st>>>(S, ncx, ncz, lk, al, lkc, alc);
    RICH_CUDA(cudaGetLastError());
    return 0;
}
