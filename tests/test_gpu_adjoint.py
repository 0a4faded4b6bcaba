"""Discrete adjoint on the GPU: against the oracle's adjoint (sparse direct J^T
solves), against central finite differences of the GPU forward solve at tight
tolerances, invariance to the checkpoint interval, mixed vs FP64, and the
torch.autograd.Function wrapper."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as OA
from tests.inputs import PHYSICS, SOLVER

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIGHT = dict(picard_tol=1e-13, mg_tol=1e-14, picard_maxit=200, mg_maxit=400)


@pytest.fixture(scope="module")
def R():
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build
    build.build()
    return R


def setup_case(R, n, nkl, S, seed, lam=0.2):
    from paper_1903_08741_gb300.kl import kl_basis
    dev = torch.device("cuda:0")
    B, _ = kl_basis(n, n, nkl, 1.0, lam)
    rng = np.random.default_rng(seed)
    xi = rng.normal(size=(S, nkl))
    _, al = O.sample_fields(n, n, S, seed=seed + 1)
    return B, xi, al, (torch.from_numpy(B).to(dev), torch.from_numpy(xi).to(dev), torch.from_numpy(al).to(dev))


def gpu_pb(R, n, steps, dt, **kw):
    d = dict(PHYSICS)
    d.update(SOLVER)
    d.update(kw)
    return R.Problem(nx=n, nz=n, nsteps=steps, dt=dt, **d)


def test_adjoint_matches_oracle_adjoint(R):
    n, nkl, S, steps, dt = 16, 8, 3, 4, 0.005
    B, xi, al, (Bd, xid, ald) = setup_case(R, n, nkl, S, 3)
    q, dq, g, st, stats, rc = R.solve_batch_adjoint(gpu_pb(R, n, steps, dt, **TIGHT), Bd, xid, ald,
                                                    ckpt_every=2, want_dlnks=True)
    q, dq, g = q.cpu().numpy(), dq.cpu().numpy(), g.cpu().numpy()
    opb = O.make_problem(nsteps=steps, dt=dt, **PHYSICS, **TIGHT)
    for s in range(S):
        lnks = np.tensordot(xi[s], B, axes=1)
        Qo, go = OA.gradient(opb, lnks, al[s])
        assert abs(q[s] - Qo) <= 1e-10 * abs(Qo)
        assert np.abs(g[s] - go).max() <= 1e-7 * np.abs(go).max()
        dqo = np.tensordot(B, go, axes=([1, 2], [0, 1]))
        assert np.abs(dq[s] - dqo).max() <= 1e-7 * np.abs(dqo).max()


def test_adjoint_matches_gpu_finite_differences(R):
    """Central differences of the forward solve (tight tolerances), step 1e-6 on xi."""
    n, nkl, S, steps, dt = 32, 6, 2, 5, 0.004
    B, xi, al, (Bd, xid, ald) = setup_case(R, n, nkl, S, 5)
    pb = gpu_pb(R, n, steps, dt, **TIGHT)
    q, dq, _, st, _, _ = R.solve_batch_adjoint(pb, Bd, xid, ald, ckpt_every=3)
    dq = dq.cpu().numpy()
    eps = 1e-6
    for j in (0, 2, 5):
        xp, xm = xid.clone(), xid.clone()
        xp[:, j] += eps
        xm[:, j] -= eps
        qp = R.solve_batch(pb, R.kl_fields(Bd, xp), ald)[0].cpu().numpy()
        qm = R.solve_batch(pb, R.kl_fields(Bd, xm), ald)[0].cpu().numpy()
        fd = (qp - qm) / (2 * eps)
        for s in range(S):
            assert abs(dq[s, j] - fd[s]) <= 1e-5 * max(abs(fd[s]), 1e-3 * np.abs(dq[s]).max()), (s, j, dq[s, j], fd[s])


def test_checkpoint_interval_does_not_change_the_gradient(R):
    n, nkl, S, steps, dt = 16, 5, 3, 7, 0.005
    B, xi, al, (Bd, xid, ald) = setup_case(R, n, nkl, S, 7)
    pb = gpu_pb(R, n, steps, dt)
    ref = None
    for ck in (1, 3, 7, 10):
        q, dq, _, st, _, _ = R.solve_batch_adjoint(pb, Bd, xid, ald, ckpt_every=ck)
        if ref is None:
            ref = (q.cpu().numpy(), dq.cpu().numpy())
        else:
            assert np.array_equal(q.cpu().numpy(), ref[0])
            assert np.array_equal(dq.cpu().numpy(), ref[1])


def test_mixed_adjoint_close_to_fp64(R):
    n, nkl, S, steps, dt = 32, 6, 4, 4, 0.005
    B, xi, al, (Bd, xid, ald) = setup_case(R, n, nkl, S, 9)
    q64, dq64, _, s64, _, _ = R.solve_batch_adjoint(gpu_pb(R, n, steps, dt), Bd, xid, ald)
    q32, dq32, _, s32, _, _ = R.solve_batch_adjoint(gpu_pb(R, n, steps, dt, precision=R.MIXED), Bd, xid, ald)
    ok = (s64.cpu().numpy() == 0) & (s32.cpu().numpy() == 0)
    assert ok.sum() >= 3
    a, b = dq64.cpu().numpy()[ok], dq32.cpu().numpy()[ok]
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
    qa, qb = q64.cpu().numpy()[ok], q32.cpu().numpy()[ok]
    assert np.abs(qa - qb).max() <= 1e-6 * np.abs(qa).max()


def test_autograd_function(R):
    n, nkl, S, steps, dt = 16, 4, 2, 3, 0.005
    B, xi, al, (Bd, xid, ald) = setup_case(R, n, nkl, S, 11)
    pb = gpu_pb(R, n, steps, dt)
    x = xid.clone().requires_grad_(True)
    q = R.RichardsQoI.apply(x, ald, Bd, pb)
    (q * torch.tensor([2.0, -1.0], dtype=torch.float64, device=q.device)).sum().backward()
    _, dq, _, _, _, _ = R.solve_batch_adjoint(pb, Bd, xid, ald)
    expect = dq * torch.tensor([[2.0], [-1.0]], dtype=torch.float64, device=q.device)
    assert torch.allclose(x.grad, expect, rtol=0, atol=0)


def test_autograd_forward_only_without_grad(R):
    """Under torch.no_grad() (or with xi not requiring grad) the wrapper runs the
    forward solve alone: no adjoint launch, the same QoI as the adjoint's forward."""
    n, nkl, S, steps, dt = 16, 4, 3, 3, 0.005
    B, xi, al, (Bd, xid, ald) = setup_case(R, n, nkl, S, 12)
    pb = gpu_pb(R, n, steps, dt)
    q_adj, _, _, st, _, _ = R.solve_batch_adjoint(pb, Bd, xid, ald)
    l0 = R.launch_count()
    with torch.no_grad():
        q = R.RichardsQoI.apply(xid.clone().requires_grad_(True), ald, Bd, pb)
    l1 = R.launch_count()
    q2 = R.RichardsQoI.apply(xid, ald, Bd, pb)
    ok = st == 0
    assert torch.equal(q[ok], q_adj[ok]) and torch.equal(q2[ok], q_adj[ok])
    assert not q.requires_grad
    # the forward path launches the KL field kernel and the fused solve only
    assert l1 - l0 <= 2


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_krylov_solvers_and_defect_correction_agree(R, prec):
    """The three J^T solvers stop at a true relative residual of 1e-11, so their
    gradients agree to the 1e-7 the oracle comparison uses; BiCGStab and
    GMRES need fewer preconditioner applications than defect correction
    (rich_stats_t.mg_cycles counts them) and none hits the cap."""
    n, nkl, S, steps, dt = 64, 6, 4, 4, 0.002
    B, xi, al, (Bd, xid, ald) = setup_case(R, n, nkl, S, 13)
    kw = {} if prec == "fp64" else dict(precision=R.MIXED)
    pb = gpu_pb(R, n, steps, dt, **kw)
    out = {}
    try:
        for m in (R.DEFECT_CORRECTION, R.BICGSTAB, R.GMRES):
            R.set_adjoint_method(m)
            out[m] = R.solve_batch_adjoint(pb, Bd, xid, ald, ckpt_every=2)
    finally:
        R.set_adjoint_method(R.BICGSTAB)
    qd, dqd, _, sd, std, _ = out[R.DEFECT_CORRECTION]
    for m in (R.BICGSTAB, R.GMRES):
        qk, dqk, _, sk, stk, _ = out[m]
        ok = (sd.cpu().numpy() == 0) & (sk.cpu().numpy() == 0)
        assert ok.sum() >= 3
        assert torch.equal(qd[ok], qk[ok])
        a, b = dqd.cpu().numpy()[ok], dqk.cpu().numpy()[ok]
        assert np.abs(a - b).max() <= 1e-7 * np.abs(a).max(), m
        assert stk.mg_cycles < std.mg_cycles, m
        assert not (sk.cpu().numpy() == R.ADJ_MAXIT).any(), m


def test_adjoint_cap_sets_its_own_status(R):
    """A J^T solve stopped at the cap of rich_set_adjoint_limits flags its sample
    ADJ_MAXIT (not the forward solver's MG_MAXIT), the call returns that code,
    and the QoI (the forward solve) is unchanged; a tolerance the solver
    cannot reach in one application is forced by a cap of 1."""
    n, nkl, S, steps, dt = 32, 6, 4, 3, 0.002
    B, xi, al, (Bd, xid, ald) = setup_case(R, n, nkl, S, 17)
    pb = gpu_pb(R, n, steps, dt)
    q0, dq0, _, s0, st0, rc0 = R.solve_batch_adjoint(pb, Bd, xid, ald, ckpt_every=2)
    assert np.isin(s0.cpu().numpy(), (R.OK, R.MG_MAXIT)).all() and rc0 in (0, R.MG_MAXIT)
    assert not (s0.cpu().numpy() == R.ADJ_MAXIT).any()
    try:
        R.set_adjoint_limits(1e-11, 1)
        q1, dq1, _, s1, st1, rc1 = R.solve_batch_adjoint(pb, Bd, xid, ald, ckpt_every=2)
    finally:
        R.set_adjoint_limits()
    assert (s1.cpu().numpy() == R.ADJ_MAXIT).all() and rc1 == R.ADJ_MAXIT
    assert torch.equal(q0, q1)
    assert torch.isfinite(dq1).all()
    # every J^T solve (one per step) stops at the cap and counts cap + 1
    assert st1.mg_cycles == S * steps * 2
    with pytest.raises(R.RichError):
        R.set_adjoint_limits(0.0, 10)
    with pytest.raises(R.RichError):
        R.set_adjoint_limits(1e-11, 0)
