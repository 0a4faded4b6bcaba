"""Pins of the oracle's discrete adjoint: its Jacobians against central finite
differences of the C oracle's residual, and its gradient against central finite
differences of the full time-stepped solve at tight tolerances."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from tests.inputs import PHYSICS, SOLVER


def problem(**kw):
    d = dict(PHYSICS)
    d.update(SOLVER)
    d.update(dict(nsteps=3, dt=0.01))
    d.update(kw)
    return O.make_problem(**d)


def residual(pb, lnks, alpha, p, p_old):
    return -O.picard_system(pb, lnks, alpha, p, p_old)[5].ravel()


@pytest.mark.parametrize("shape", [(8, 8), (6, 10)])
def test_jacobians_match_residual_differences(shape):
    nz, nx = shape
    rng = np.random.default_rng(5)
    lnks = 0.6 * rng.normal(size=shape)
    alpha = rng.uniform(0.5, 2.0, size=shape)
    p = -0.5 - 4.0 * rng.uniform(size=shape)
    p_old = p - 0.1 * rng.uniform(size=shape)
    pb = problem()
    h = 1.0 / nz
    J, G, _ = A.residual_jacobians(p, lnks, alpha, pb, h)
    for k in range(3):
        v = rng.normal(size=shape)
        eps = 1e-6
        fd = (residual(pb, lnks, alpha, p + eps * v, p_old) - residual(pb, lnks, alpha, p - eps * v, p_old)) / (2 * eps)
        assert np.abs(J @ v.ravel() - fd).max() <= 1e-6 * np.abs(fd).max()
        fdm = (residual(pb, lnks + eps * v, alpha, p, p_old) - residual(pb, lnks - eps * v, alpha, p, p_old)) / (2 * eps)
        assert np.abs(G @ v.ravel() - fdm).max() <= 1e-6 * np.abs(fdm).max()


def test_adjoint_gradient_matches_finite_differences():
    """8x8 grid, 3 steps; tight tolerances so that solver noise (tol/step) stays
    far below the finite-difference truncation error."""
    rng = np.random.default_rng(2)
    lnks, alpha = O.sample_fields(8, 8, 1, seed=9)
    lnks, alpha = lnks[0], alpha[0]
    pb = problem(picard_tol=1e-13, mg_tol=1e-14, picard_maxit=200, mg_maxit=400)
    Q, g = A.gradient(pb, lnks, alpha)
    for cell in [(0, 0), (0, 5), (3, 4), (7, 2)]:
        eps = 1e-6
        lp, lm = lnks.copy(), lnks.copy()
        lp[cell] += eps
        lm[cell] -= eps
        qp = A.qoi_grads(A.forward_states(pb, lp, alpha)[-1], lp, alpha, pb, 1 / 8)[0]
        qm = A.qoi_grads(A.forward_states(pb, lm, alpha)[-1], lm, alpha, pb, 1 / 8)[0]
        fd = (qp - qm) / (2 * eps)
        assert abs(g[cell] - fd) <= 1e-5 * max(abs(fd), 1e-3 * abs(g).max()), (cell, g[cell], fd)
    # the oracle's own QoI agrees with the forward solve's
    p, q, rc, _ = O.solve_one(pb, lnks, alpha)
    assert abs(q - Q) <= 1e-12 * abs(q)


@pytest.mark.parametrize("shape", [(4, 4), (8, 8)])
def test_newton_on_tiny_grids_reaches_the_picard_solution(shape):
    """Tiny-grid pin of the nonlinear solve: Newton's method with the analytic
    (finite-difference-free) Jacobian of the discrete residual, globalised by
    backtracking and started after five Picard iterations, converges quadratically to the exact discrete solution of
    one implicit step, and modified Picard + CCMG reaches the same state to
    within its tolerances."""
    nz, nx = shape
    lnks, alpha = O.sample_fields(nx, nz, 1, seed=21)
    lnks, alpha = lnks[0], alpha[0]
    pb = problem(nsteps=1, picard_tol=1e-13, picard_maxit=200, mg_tol=1e-14, mg_maxit=400)
    p_pic, q, rc, _ = O.solve_one(pb, lnks, alpha)
    assert rc == 0
    h = 1.0 / nz
    p_old = np.full(shape, PHYSICS["p_init"])
    # Newton is sensitive to its starting point (Sec. 4.2): start from the state
    # after 5 Picard iterations, still far from converged
    p, _, rc5, _ = O.solve_one(problem(nsteps=1, picard_tol=1e-13, picard_maxit=5, mg_tol=1e-14, mg_maxit=400),
                               lnks, alpha)
    assert rc5 == O.PICARD_MAXIT and np.abs(p - p_pic).max() > 1e-3
    steps = []
    for it in range(60):
        R = residual(pb, lnks, alpha, p, p_old)
        J, _, _ = A.residual_jacobians(p, lnks, alpha, pb, h)
        d = np.linalg.solve(J.toarray(), -R).reshape(shape)
        # backtracking on ||R||_inf (Newton from the old state overshoots on this
        # step); full steps near the root
        t, r0 = 1.0, np.abs(R).max()
        while t > 1e-6 and not np.abs(residual(pb, lnks, alpha, p + t * d, p_old)).max() < r0:
            t *= 0.5
        p = p + t * d
        steps.append(np.abs(t * d).max())
        if steps[-1] < 1e-14:
            break
    assert steps[-1] < 1e-14, steps
    # quadratic convergence once close: each step at most C times the square of the previous
    tail = [(b, a) for a, b in zip(steps[:-1], steps[1:]) if a < 1e-3 and b > 1e-15]
    assert tail and all(b <= 50.0 * a * a for b, a in tail), steps
    assert np.abs(p - p_pic).max() < 1e-10 * np.abs(p).max()
