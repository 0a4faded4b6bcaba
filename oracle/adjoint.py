"""Discrete adjoint of the time-stepped mixed-form solve (oracle; test
infrastructure only).

For the converged states p^1..p^N of backward Euler (Sec. 4.1, Eq.
Mixed_based), R_n(p^n, p^{n-1}, m) = 0 with m = ln Ks.  The QoI is the mean
outward Darcy flux through the bottom faces at t_N.  With the Lagrangian
Q - sum_n lambda_n^T R_n the adjoint recursion is

    J_N^T lambda_N = dQ/dp^N
    J_n^T lambda_n = diag(C(p^n)/dt) lambda_{n+1}          (n < N)
    dQ/dm = dQ/dm|explicit - sum_n (dR_n/dm)^T lambda_n

where J_n = dR_n/dp^n is the full (Newton) Jacobian, including the derivative
of the harmonic-mean face conductivities through K(p) = Ks exp(alpha p), and
-diag(C(p^n)/dt) = dR_{n+1}/dp^n couples consecutive steps (C = d theta/dp).
Linear solves use a sparse direct factorisation (scipy SuperLU, a library
primitive).  The formulas are restated here from the residual of the C oracle
(face flux -T (p_nb - p_P + s h), s = +1 north, -1 south, 0 east/west;
Dirichlet faces -T_b (p_D - p_P +- h/2) with T_b = 2 Ks exp(alpha min(p_D,0))/h^2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import make_problem, solve_one


def _cell_K(p, lnks, a):
    """K, dK/dp, C/(theta_s - theta_r) per cell (Gardner closure, Eqs. Sw/Krw branches)."""
    ks = np.exp(lnks)
    neg = p < 0
    E = np.where(neg, np.exp(a * np.minimum(p, 0.0)), 1.0)
    K = ks * E
    dK = np.where(neg, a * K, 0.0)
    Cn = np.where(neg, a * E, 0.0)
    return K, dK, Cn


def _faces(nx, nz):
    """Interior faces as (cell, neighbour, s): s = +1 if the neighbour is above
    (north), -1 if below, 0 for east neighbours; each face listed once."""
    idx = np.arange(nx * nz).reshape(nz, nx)
    e = (idx[:, :-1].ravel(), idx[:, 1:].ravel(), np.zeros(nz * (nx - 1)))
    n = (idx[:-1, :].ravel(), idx[1:, :].ravel(), np.ones((nz - 1) * nx))
    return [np.concatenate(x) for x in zip(e, n)]


def residual_jacobians(p, lnks, a, pb, h):
    """Sparse J = dR/dp and G = dR/dm at state p (R per unit cell area)."""
    nz, nx = p.shape
    pf, mf, af = p.ravel(), lnks.ravel(), a.ravel()
    K, dK, Cn = _cell_K(pf, mf, af)
    n = nx * nz
    c, nb, s = _faces(nx, nz)
    Kc, Kn = K[c], K[nb]
    T = (2.0 / h ** 2) * Kc * Kn / (Kc + Kn)
    dT_dKc = (2.0 / h ** 2) * Kn ** 2 / (Kc + Kn) ** 2
    dT_dKn = (2.0 / h ** 2) * Kc ** 2 / (Kc + Kn) ** 2
    g = pf[nb] - pf[c] + s * h                       # flux of cell c through the face: -T g
    # dF_c/dp_c, dF_c/dp_nb (F_nb = -F_c)
    dFc_dpc = T - g * dT_dKc * dK[c]
    dFc_dpnb = -T - g * dT_dKn * dK[nb]
    rows = np.concatenate([c, c, nb, nb])
    cols = np.concatenate([c, nb, c, nb])
    vals = np.concatenate([dFc_dpc, dFc_dpnb, -dFc_dpc, -dFc_dpnb])
    # dF_c/dm_c = -g dT/dKc K_c, dF_c/dm_nb = -g dT/dKn K_nb
    gv = np.concatenate([-g * dT_dKc * Kc, -g * dT_dKn * Kn, g * dT_dKc * Kc, g * dT_dKn * Kn])
    # mass term and Dirichlet faces
    diag = (pb.theta_s - pb.theta_r) * Cn / pb.dt
    top = np.arange((nz - 1) * nx, n)
    bot = np.arange(nx)
    Tbt = (2.0 / h ** 2) * np.exp(mf[top]) * np.exp(af[top] * min(pb.p_top, 0.0))
    Tbb = (2.0 / h ** 2) * np.exp(mf[bot]) * np.exp(af[bot] * min(pb.p_bottom, 0.0))
    diag = diag.copy()
    diag[top] += Tbt
    diag[bot] += Tbb
    gdiag = np.zeros(n)
    gdiag[top] += -(pb.p_top - pf[top] + h / 2.0) * Tbt
    gdiag[bot] += -(pb.p_bottom - pf[bot] - h / 2.0) * Tbb
    ar = np.arange(n)
    J = sp.coo_matrix((np.concatenate([vals, diag]), (np.concatenate([rows, ar]),
                       np.concatenate([cols, ar]))), shape=(n, n)).tocsr()
    G = sp.coo_matrix((np.concatenate([gv, gdiag]), (np.concatenate([rows, ar]),
                       np.concatenate([cols, ar]))), shape=(n, n)).tocsr()
    return J, G, (pb.theta_s - pb.theta_r) * Cn / pb.dt


def qoi_grads(p, lnks, a, pb, h):
    """Q, dQ/dp, dQ/dm for the mean outward bottom flux (1/nx) sum K_b (2(p - p_bot)/h + 1)."""
    nz, nx = p.shape
    n = nx * nz
    kb = np.exp(lnks[0]) * np.exp(a[0] * min(pb.p_bottom, 0.0))
    q_i = kb * (2.0 * (p[0] - pb.p_bottom) / h + 1.0)
    dqdp = np.zeros(n)
    dqdm = np.zeros(n)
    dqdp[:nx] = kb * 2.0 / h / nx
    dqdm[:nx] = q_i / nx
    return q_i.mean(), dqdp, dqdm


def forward_states(pb, lnks, alpha, alpha_scale=1.0):
    """p^0..p^N by the oracle's Picard/CCMG solve, one step at a time."""
    nz, nx = lnks.shape
    one = make_problem(nsteps=1, dt=pb.dt, theta_r=pb.theta_r, theta_s=pb.theta_s, p_top=pb.p_top,
                       p_bottom=pb.p_bottom, p_init=pb.p_init, picard_tol=pb.picard_tol,
                       picard_maxit=pb.picard_maxit, mg_tol=pb.mg_tol, mg_maxit=pb.mg_maxit,
                       nu1=pb.nu1, nu2=pb.nu2, gamma=pb.gamma)
    states = [np.full((nz, nx), pb.p_init)]
    for n in range(pb.nsteps):
        p, q, rc, _ = solve_one(one, lnks, alpha, alpha_scale, p_init=states[-1])
        if rc not in (0, 2):
            raise RuntimeError(f"forward step {n} failed with status {rc}")
        states.append(p)
    return states


def gradient(pb, lnks, alpha, alpha_scale=1.0):
    """(Q, dQ/d ln Ks [nz, nx]) by the discrete adjoint of the converged solve."""
    nz, nx = lnks.shape
    h = 1.0 / nz
    a = alpha * alpha_scale
    states = forward_states(pb, lnks, alpha, alpha_scale)
    Q, dqdp, dqdm = qoi_grads(states[-1], lnks, a, pb, h)
    g = dqdm.copy()
    rhs = dqdp
    for n in range(pb.nsteps, 0, -1):
        J, G, cdt = residual_jacobians(states[n], lnks, a, pb, h)
        lam = spla.spsolve(J.T.tocsc(), rhs)
        g -= G.T @ lam
        # right-hand side of step n-1: -(dR_n/dp^{n-1})^T lam = diag(C(p^{n-1})/dt) lam
        _, _, cdt_prev = residual_jacobians(states[n - 1], lnks, a, pb, h)
        rhs = cdt_prev * lam
    return Q, g.reshape(nz, nx)
