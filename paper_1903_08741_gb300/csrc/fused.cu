// Persistent fused solver: one kernel launch solves a whole batch (host
// side: slot layout, launch shapes, entry points; the kernels are in
// fused_kernel.cuh).
#include "fused_kernel.cuh"
#include <algorithm>
#include <mutex>

namespace {

unsigned magic(int d) { return d <= 1 ? 0u : (unsigned)((0x100000000ull / (unsigned)d) + 1); }
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Dynamic shared memory of a CTA (no device work): the coarsest level's dense
// matrix; then the arrays that the cycles read on the small coarse levels
// that warp 0 runs alone (levels l >= 1 with at most WARP_CELLS cells: the
// multigrid arrays, and for FP64 the coarsest level's faces and diagonal,
// which the direct solve assembles); then the corrections dp of as many of the other levels
// (coarsest first) as fit the budget of the launch shape (one 1024-thread CTA
// per SM may use ~220 KB, two 512-thread CTAs ~104 KB each, four 256-thread
// CTAs ~50 KB each, eight 128-thread CTAs ~24 KB each), so that the
// Gauss-Seidel neighbour reads of those levels
// stay on chip; levels that do not fit keep dp in the slot.  Results do not
// depend on where an array lives.
constexpr int WARP_CELLS = 256;

static void plan_smem(FParams& P, int nt) {
    const size_t w = P.mixed ? 4 : 8;
    const int c = P.nlev - 1;
    const size_t nnc = (size_t)P.nx[c] * P.nz[c];
    auto al16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    size_t off = al16(nnc * (nnc + 1) * w);
    const size_t budget = nt == 1024 ? 220 * 1024 : nt == 512 ? 104 * 1024 : nt == 256 ? 50 * 1024
                        : nt == 128 ? 24 * 1024 : 3 * 1024;
    for (int l = 0; l < MAXL; ++l) {
        P.osm[l] = -1;
        for (int k = 0; k < N64; ++k) P.s64[l][k] = -1;
        for (int k = 0; k < NMG; ++k) P.smg[l][k] = -1;
    }
    // small levels below the finest run on warp 0 with their arrays on chip;
    // a one-warp CTA (32 threads, 32 CTAs per SM) runs every level itself and
    // keeps them in its slot: on-chip copies would cost it its occupancy
    P.lw = P.nlev;
    for (int l = 1; l < P.nlev && nt > 32; ++l)
        if ((size_t)P.nx[l] * P.nz[l] <= (size_t)WARP_CELLS) { P.lw = l; break; }
    for (int l = P.lw; l < P.nlev; ++l) {
        const size_t nc = (size_t)P.nx[l] * P.nz[l];
        if (!P.mixed) {
            for (int k = 0; k < N64; ++k) {
                if (!(l == c && (k == A_TX || k == A_TZ || k == A_D))) continue;
                P.s64[l][k] = (long long)off;
                off = al16(off + nc * 8);
            }
        }
        for (int k = 0; k < NMG; ++k) {
            if (P.omg[l][k] < 0) continue;
            P.smg[l][k] = (long long)off;
            off = al16(off + nc * w);
        }
    }
    for (int l = P.lw - 1; l >= 0; --l) {
        const size_t bytes = al16((size_t)P.nx[l] * P.nz[l] * w);
        if (off + bytes > budget) break;
        P.osm[l] = (long long)off;
        off += bytes;
    }
    P.smem_bytes = (long long)off;
}

static int fused_setup(const rich_problem_t* pb, int S, FParams& P, int ckpt_every = 0) {
    P = FParams{};
    const int nlev = rich_count_levels(pb->nx, pb->nz);
    if (nlev < 1) return RICH_ERR_INVALID;
    const bool mixed = pb->precision == RICH_MIXED;
    // index arithmetic uses 32-bit magic division: cell index * row length < 2^32
    if ((unsigned long long)pb->nx * pb->nz * pb->nx >= (1ull << 32)) return RICH_ERR_INVALID;
    P.S = S; P.nlev = nlev; P.mixed = mixed;
    size_t off = 0;
    int lx = pb->nx, lz = pb->nz;
    const size_t w = mixed ? 4 : 8;
    for (int l = 0; l < nlev; ++l) {
        P.nx[l] = lx; P.nz[l] = lz; P.mnx[l] = magic(lx); P.mhx[l] = magic(lx / 2);
        const size_t nc = (size_t)lx * lz;
        for (int k = 0; k < N64; ++k) {
            size_t bytes = (k == A_TBT || k == A_TBB) ? (size_t)lx * 8 : nc * 8;
            P.o64[l][k] = (long long)off; off = al256(off + bytes);
        }
        for (int k = 0; k < NMG; ++k) {
            // FP64: wE wW wN wS q f dp D ; FP32: Tx Tz - D q f dp - (slots B_2, B_7 unused)
            if (mixed && (k == B_2 || k == B_7)) { P.omg[l][k] = -1; continue; }
            P.omg[l][k] = (long long)off; off = al256(off + nc * w);
        }
        lx /= 2; lz /= 2;
    }
    const size_t nc8 = (size_t)pb->nx * pb->nz * 8;
    P.o_f64 = off; off = al256(off + nc8);
    if (mixed) { P.o_dp64 = off; off = al256(off + nc8); } else P.o_dp64 = -1;
    P.o_p = off; off = al256(off + nc8);
    P.o_thold = off; off = al256(off + nc8);
    P.o_Ks = off; off = al256(off + nc8);
    P.o_a = off; off = al256(off + nc8);
    P.o_K = off; off = al256(off + nc8);
    P.o_th = off; off = al256(off + nc8);
    P.closure = pb->closure;
    if (pb->closure == RICH_VAN_GENUCHTEN) {
        long long* cl[] = {&P.o_n, &P.o_m, &P.o_trc, &P.o_tsc};
        for (long long* o : cl) { *o = (long long)off; off = al256(off + nc8); }
    } else {
        P.o_n = P.o_m = P.o_trc = P.o_tsc = -1;
    }
    if (ckpt_every > 0) {
        const int nck = (pb->nsteps + ckpt_every - 1) / ckpt_every;
        P.ckpt_every = ckpt_every;
        P.o_ckpt = off; off = al256(off + nc8 * std::max(nck, 1));
        P.o_seg = off; off = al256(off + nc8 * ckpt_every);
        long long* adj[] = {&P.o_lam, &P.o_rhs, &P.o_r, &P.o_dE, &P.o_dW, &P.o_dN, &P.o_dS, &P.o_dg, &P.o_g,
                            &P.o_rh, &P.o_pk, &P.o_v, &P.o_t, &P.o_ph, &P.o_sh};
        for (long long* o : adj) { *o = (long long)off; off = al256(off + nc8); }
        P.o_kry = (long long)off; off = al256(off + nc8 * (2 * ADJ_M + 1));
    }
    P.slot_bytes = (long long)off;
    P.nsteps = pb->nsteps; P.picard_maxit = pb->picard_maxit; P.mg_maxit = pb->mg_maxit;
    P.nu1 = pb->nu1; P.nu2 = pb->nu2; P.gamma = pb->cycle < 1 ? 1 : pb->cycle;
    P.inv_dt = 1.0 / pb->dt; P.tr = pb->theta_r; P.ts = pb->theta_s; P.p_top = pb->p_top;
    P.p_bot = pb->p_bottom; P.p_init = pb->p_init; P.picard_tol = pb->picard_tol; P.mg_tol = pb->mg_tol;
    P.h = 1.0 / pb->nz; P.two_over_h2 = 2.0 / (P.h * P.h);
    P.init_decay = pb->init_decay;
    return 0;
}

static size_t fused_smem(const FParams& P) { return (size_t)P.smem_bytes; }

// the fused kernel's instantiations live in one translation unit per (cycle
// precision, closure): fused_g64.cu, fused_g32.cu, fused_vg64.cu, fused_vg32.cu
static int fused_occupancy(const FParams& P, size_t smem, int nt, int* occ) {
    if (P.closure == RICH_VAN_GENUCHTEN)
        return P.mixed ? rich_occ_vg32(P, smem, nt, occ) : rich_occ_vg64(P, smem, nt, occ);
    return P.mixed ? rich_occ_g32(P, smem, nt, occ) : rich_occ_g64(P, smem, nt, occ);
}

static int fused_launch(const FParams& P, int grid, size_t smem, int nt, cudaStream_t st) {
    RICH_CUDA(cudaMemsetAsync(P.queue, 0, sizeof(int), st));
    rich_count_launch();
    if (P.closure == RICH_VAN_GENUCHTEN) {
        if (P.mixed) rich_launch_vg32(P, grid, smem, nt, st);
        else rich_launch_vg64(P, grid, smem, nt, st);
    } else if (P.mixed) {
        rich_launch_g32(P, grid, smem, nt, st);
    } else {
        rich_launch_g64(P, grid, smem, nt, st);
    }
    RICH_CUDA(cudaGetLastError());
    return 0;
}

// Fused persistent solve of S samples; stats arrays live in ctx->ws, the
// per-CTA slots and the queue counter in ctx->fused_scratch.
int rich_solve_fused(rich_ctx* ctx, const rich_problem_t* pb, int S, const double* lnKs,
                     const double* alpha, double alpha_scale, double* qoi, double* p_final,
                     int32_t* status, cudaStream_t st, const rich_soil_in* soil) {
    rich_samplebuf& w = ctx->sb;
    FParams P;
    if (pb->closure == RICH_VAN_GENUCHTEN && (!soil || !soil->n)) return RICH_ERR_INVALID;
    const int nt = (ctx->tune_threads == 1024 || ctx->tune_threads == 256 || ctx->tune_threads == 128 ||
                    ctx->tune_threads == 32)
                       ? ctx->tune_threads : 512;
    if (int e = fused_setup(pb, S, P)) return e;
    plan_smem(P, nt);
    if (soil) {
        P.n_in = soil->n; P.ts_in = soil->theta_s; P.tr_in = soil->theta_r;
        P.alpha_shift = soil->alpha_shift; P.n_shift = soil->n_shift;
    }
    const size_t off = (size_t)P.slot_bytes;
    const size_t smem = fused_smem(P);
    P.mixed_inner = ctx->tune_mixed_inner > 0 ? ctx->tune_mixed_inner : MIXED_INNER_DEFAULT;
    int occ = 0;
    if (int e = fused_occupancy(P, smem, nt, &occ)) return e;
    const int grid = std::max(1, std::min(S, ctx->sm_count * occ));
    const size_t need = (size_t)grid * off + 256;
    if (ctx->fused_bytes < need) {
        if (ctx->fused_scratch) cudaFree(ctx->fused_scratch);
        ctx->fused_scratch = nullptr; ctx->fused_bytes = 0;
        cudaError_t e = cudaMalloc(&ctx->fused_scratch, need);
        if (e != cudaSuccess) { cudaGetLastError(); return RICH_ERR_OOM; }
        ctx->fused_bytes = need;
    }
    P.scratch = (char*)ctx->fused_scratch + 256;
    P.queue = (int*)ctx->fused_scratch;
    P.lnKs = lnKs; P.alpha = alpha; P.alpha_scale = alpha_scale;
    P.qoi = qoi; P.p_final = p_final; P.status = w.status;
    P.pic_total = w.pic_total; P.mg_total = w.mg_total; P.maxpic = w.maxpic; P.t_ns = w.t_ns;
    // CTAs that share an SM during the solve: a grid smaller than the GPU's
    // resident capacity is spread over the SMs first
    w.last_occ = std::max(1, std::min(occ, (grid + ctx->sm_count - 1) / std::max(ctx->sm_count, 1)));
    rich_prof_begin(ctx, st);
    if (int e = fused_launch(P, grid, smem, nt, st)) return e;
    rich_prof_end(ctx, st, 0.0, 0.0);
    w.last = S;
    if (status)
        RICH_CUDA(cudaMemcpyAsync(status, w.status, sizeof(int32_t) * S, cudaMemcpyDeviceToDevice, st));
    return 0;
}

// Discrete adjoint of S samples: QoI and dQ/d ln Ks [S][nz][nx] (g_out).
int rich_adjoint_fused(rich_ctx* ctx, const rich_problem_t* pb, int S, const double* lnKs,
                       const double* alpha, double alpha_scale, int ckpt_every, double adj_tol,
                       int adj_maxit, int adj_method, double* qoi, double* g_out, cudaStream_t st) {
    rich_samplebuf& w = ctx->sb;
    FParams P;
    if (ckpt_every < 1 || pb->closure != RICH_GARDNER) return RICH_ERR_INVALID;
    if (int e = fused_setup(pb, S, P, ckpt_every)) return e;
    plan_smem(P, 512);
    P.adj_tol = adj_tol; P.adj_maxit = adj_maxit; P.adj_inner = pb->precision == RICH_MIXED ? 2 : 1;
    P.adj_method = adj_method;
    P.mixed_inner = ctx->tune_mixed_inner > 0 ? ctx->tune_mixed_inner : MIXED_INNER_DEFAULT;
    const size_t smem = fused_smem(P);
    int occ = 0;
    const void* kern = P.mixed ? rich_adjoint_kernel32(P.gamma > 1) : rich_adjoint_kernel64(P.gamma > 1);
    if (int e = allow_dyn_smem(kern, smem)) return e;
    RICH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 512, smem));
    occ = std::max(occ, 1);
    const int grid = std::max(1, std::min(S, ctx->sm_count * occ));
    const size_t need = (size_t)grid * (size_t)P.slot_bytes + 256;
    if (ctx->fused_bytes < need) {
        if (ctx->fused_scratch) cudaFree(ctx->fused_scratch);
        ctx->fused_scratch = nullptr; ctx->fused_bytes = 0;
        cudaError_t e = cudaMalloc(&ctx->fused_scratch, need);
        if (e != cudaSuccess) { cudaGetLastError(); return RICH_ERR_OOM; }
        ctx->fused_bytes = need;
    }
    P.scratch = (char*)ctx->fused_scratch + 256;
    P.queue = (int*)ctx->fused_scratch;
    P.lnKs = lnKs; P.alpha = alpha; P.alpha_scale = alpha_scale;
    P.qoi = qoi; P.p_final = nullptr; P.status = w.status; P.g_out = g_out;
    P.pic_total = w.pic_total; P.mg_total = w.mg_total; P.maxpic = w.maxpic;
    RICH_CUDA(cudaMemsetAsync(P.queue, 0, sizeof(int), st));
    rich_count_launch();
    rich_prof_begin(ctx, st);
    if (P.mixed) rich_adjoint_launch32(P, grid, smem, st);
    else rich_adjoint_launch64(P, grid, smem, st);
    rich_prof_end(ctx, st, 0.0, 0.0);
    RICH_CUDA(cudaGetLastError());
    return 0;
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  Its scratch (queue counter + per-CTA slots) is a
// file-scope device array of RICH_NOALLOC_SCRATCH_BYTES, created when the
// library is loaded and held by every GPU that loads it until the process
// exits.  Host code may not use the array's name as a device address (on the
// host it names a shadow object), so the address is looked up once per device
// with cudaGetSymbolAddress and cached; the look-up runs under a mutex, so
// first calls from several host threads resolve it once.  The cached address
// belongs to the device's primary context: after cudaDeviceReset on that
// device the array is gone and this entry point must not be called again in
// the process.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[RICH_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES];
int g_noalloc_sms[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;
}

extern "C" int rich_solve_batch_noalloc(const rich_problem_t* pb, int32_t nsamples,
                                        const double* lnKs, const double* alpha, double alpha_scale,
                                        double* qoi, int32_t* status, void* stream) {
    if (rich_check_problem(pb) || nsamples < 0) {
        rich_set_error("invalid problem or sample count", __FILE__, __LINE__);
        return RICH_ERR_INVALID;
    }
    if (pb->closure != RICH_GARDNER) {
        rich_set_error("the allocation-free entry point takes the Gardner closure only", __FILE__, __LINE__);
        return RICH_ERR_INVALID;
    }
    if (nsamples == 0) return 0;
    if (!lnKs || !alpha || !qoi) {
        rich_set_error("lnKs, alpha and qoi are required", __FILE__, __LINE__);
        return RICH_ERR_INVALID;
    }
    int dev = -1;
    RICH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        rich_set_error("device index beyond the allocation-free table", __FILE__, __LINE__);
        return RICH_ERR_INVALID;
    }
    char* base = nullptr;
    int dev_sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {      // first call on this device: resolve the symbol
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                rich_set_error(e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address", __FILE__,
                               __LINE__);
                return RICH_ERR_CUDA;
            }
            int sms = 0;
            RICH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            g_noalloc_sms[dev] = sms;
            g_noalloc_addr[dev] = ptr;
        }
        base = (char*)g_noalloc_addr[dev];
        dev_sms = g_noalloc_sms[dev];
    }
    FParams P;
    if (int e = fused_setup(pb, nsamples, P)) {
        rich_set_error("unsupported grid", __FILE__, __LINE__);
        return e;
    }
    plan_smem(P, 512);
    const size_t slot = (size_t)P.slot_bytes;
    const size_t slots = (RICH_NOALLOC_SCRATCH_BYTES - 256) / slot;
    if (slots < 1) {
        rich_set_error("grid needs more scratch per CTA than the allocation-free entry point holds "
                       "(RICH_NOALLOC_SCRATCH_BYTES)", __FILE__, __LINE__);
        return RICH_ERR_INVALID;
    }
    const size_t smem = fused_smem(P);
    P.mixed_inner = MIXED_INNER_DEFAULT;
    int occ = 0;
    if (int e = fused_occupancy(P, smem, 512, &occ)) return e;
    const int grid = (int)std::min<long long>({(long long)nsamples, (long long)dev_sms * occ, (long long)slots});
    P.queue = (int*)base;                 // cleared by fused_launch before the kernel
    P.scratch = base + 256;
    P.lnKs = lnKs; P.alpha = alpha; P.alpha_scale = alpha_scale;
    P.qoi = qoi; P.p_final = nullptr; P.status = status;
    P.pic_total = nullptr; P.mg_total = nullptr; P.maxpic = nullptr;
    return fused_launch(P, grid, smem, 512, (cudaStream_t)stream);
}
