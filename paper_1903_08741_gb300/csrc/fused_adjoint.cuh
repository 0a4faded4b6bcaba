// Device side of the discrete adjoint (kernel template), shared by the
// translation units that instantiate it; the Cta methods it calls (Jacobian
// pieces, J^T products and solvers, gradient update) live with the forward
// solver in fused_kernel.cuh.
#pragma once
#include "fused_kernel.cuh"

namespace {

// Discrete adjoint of the converged time-stepped solve (one sample per CTA):
// forward with a checkpoint of p every ckpt_every steps, then per segment
// (last first) recompute its states from the checkpoint and step backwards:
//   J_N^T lam_N = dQ/dp^N,  J_n^T lam_n = diag(C(p^n)/dt) lam_{n+1},
//   dQ/dm = dQ/dm|explicit - sum_n (dR_n/dm)^T lam_n     (m = ln Ks).
template <typename TM, bool WC>
__global__ void __maxnreg__(128)
k_adjoint(const FParams P) {
    extern __shared__ unsigned char smraw[];
    __shared__ unsigned long long red[33];
    __shared__ int s_sample;
    __shared__ Lv64 L64[MAXL];
    __shared__ Lv<TM> LM[MAXL];
    char* slot = P.scratch + (size_t)blockIdx.x * P.slot_bytes;
    init_levels<TM>(P, slot, smraw, L64, LM);
    Cta<TM, WC> C(P, slot, L64, LM, reinterpret_cast<TM*>(smraw), red);
    const int nc = C.nc, nx = C.nx, tid = C.tid, nt = C.nt;
    const int CK = P.ckpt_every;
    double* ckpt = (double*)(slot + P.o_ckpt);      // [nck][nc]
    double* seg = (double*)(slot + P.o_seg);        // [CK][nc]
    double* lam = (double*)(slot + P.o_lam);
    double* rhs = (double*)(slot + P.o_rhs);
    double* r = (double*)(slot + P.o_r);
    double* dE = (double*)(slot + P.o_dE);
    double* dW = (double*)(slot + P.o_dW);
    double* dN = (double*)(slot + P.o_dN);
    double* dS = (double*)(slot + P.o_dS);
    double* dg = (double*)(slot + P.o_dg);
    double* g = (double*)(slot + P.o_g);
    const double NaN = __longlong_as_double(0x7FF8000000000000ll);
    for (;;) {
        if (tid == 0) s_sample = atomicAdd(P.queue, 1);
        __syncthreads();
        const int s = s_sample;
        __syncthreads();
        if (s >= P.S) break;
        C.setup(s);
        int status = RICH_OK, maxpic = 0;
        bool alive = true;
        long long pic_tot = 0, mg_tot = 0, adj_its = 0;
        // ---- forward with checkpoints p^0, p^CK, p^2CK, ...
        for (int n = 1; n <= P.nsteps && alive; ++n) {
            if ((n - 1) % CK == 0) {
                double* dst = ckpt + (size_t)((n - 1) / CK) * nc;
                for (int q = tid; q < nc; q += nt) dst[q] = C.p[q];
                __syncthreads();
            }
            alive = C.time_step(pic_tot, mg_tot, maxpic, status);
        }
        double qv = 0.0;
        if (tid < 32) qv = C.qoi_warp0();
        if (alive) {
            // ---- dQ/dp^N (rhs) and the explicit dQ/dm (g), bottom cells
            for (int q = tid; q < nc; q += nt) {
                double gv = 0.0, rv = 0.0;
                if (q < nx) {
                    double kb = P.p_bot < 0.0 ? C.Ks[q] * exp(C.aa[q] * P.p_bot) : C.Ks[q];
                    rv = kb * (2.0 / C.h) / nx;
                    gv = kb * (2.0 * (C.p[q] - P.p_bot) / C.h + 1.0) / nx;
                }
                rhs[q] = rv;
                g[q] = gv;
            }
            __syncthreads();
            const int nck = (P.nsteps + CK - 1) / CK;
            for (int sg = nck - 1; sg >= 0 && alive; --sg) {
                const int n0 = sg * CK, n1 = min(n0 + CK, P.nsteps);
                // recompute p^{n0+1..n1} from the checkpoint
                for (int q = tid; q < nc; q += nt) C.p[q] = ckpt[(size_t)sg * nc + q];
                __syncthreads();
                long long dpic = 0, dmg = 0;
                int dmax = 0, dst = RICH_OK;
                for (int n = n0 + 1; n <= n1 && alive; ++n) {
                    alive = C.time_step(dpic, dmg, dmax, dst);
                    double* dstp = seg + (size_t)(n - n0 - 1) * nc;
                    for (int q = tid; q < nc; q += nt) dstp[q] = C.p[q];
                    __syncthreads();
                }
                if (!alive) { status = dst; break; }
                for (int n = n1; n > n0; --n) {
                    // state p^n, operator and Jacobian at p^n
                    const double* pn = seg + (size_t)(n - n0 - 1) * nc;
                    for (int q = tid; q < nc; q += nt) C.p[q] = pn[q];
                    __syncthreads();
                    C.assemble();
                    if (n < P.nsteps) {       // rhs = diag(C(p^n)/dt) lam_{n+1}
                        for (int q = tid; q < nc; q += nt) rhs[q] = L64[0].Cdt[q] * lam[q];
                        __syncthreads();
                    }
                    C.adj_prepare(dE, dW, dN, dS, dg);
                    const int its = P.adj_method == 2
                        ? C.adj_solve_gmres(dE, dW, dN, dS, dg, rhs, lam, (double*)(slot + P.o_kry))
                        : P.adj_method == 1
                        ? C.adj_solve_bicgstab(dE, dW, dN, dS, dg, rhs, lam, r, (double*)(slot + P.o_rh),
                                               (double*)(slot + P.o_pk), (double*)(slot + P.o_v),
                                               (double*)(slot + P.o_t), (double*)(slot + P.o_ph),
                                               (double*)(slot + P.o_sh))
                        : C.adj_solve(dE, dW, dN, dS, dg, rhs, lam, r);
                    adj_its += its;
                    // status is OK or MG_MAXIT here (the sample is alive);
                    // a J^T solve stopped at its cap outranks both
                    if (its > P.adj_maxit) status = RICH_ADJ_MAXIT;
                    C.adj_grad_update(lam, g);
                }
            }
        }
        if (tid == 0) {
            P.qoi[s] = alive ? qv : NaN;
            if (P.status) P.status[s] = status;
            if (P.pic_total) P.pic_total[s] = pic_tot;
            if (P.mg_total) P.mg_total[s] = adj_its;
            if (P.maxpic) P.maxpic[s] = maxpic;
        }
        for (int q = tid; q < nc; q += nt) P.g_out[(size_t)s * nc + q] = alive ? g[q] : NaN;
        __syncthreads();
    }
}

}  // namespace
