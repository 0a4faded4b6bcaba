"""GPU van Genuchten-Mualem path (Sec. 2.1; the infiltration problem of
Sec. 4.3; the soil fields of Table soilparams) against the FP64 oracle,
through the C ABI.

Fields drawn on the GPU match the oracle's to 1e-12.  Solves take identical
fields (drawn by the oracle and uploaded) and must agree to 1e-10 relative in
pressure head and QoI on the FP64 path (statuses equal, cycle counts within
rounding-order slack) and to 1e-6 relative in the QoI on the mixed path.
Tolerances here are tight (Picard 1e-10, MG 1e-12) so that both sides stop
on the same iteration; the paper's 1e-5 is what the workloads use.
"""
import os

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 1
TIGHT = dict(picard_tol=1e-10, mg_tol=1e-12, picard_maxit=60, mg_maxit=200)
PHI1 = dict(nu=1.0, corr_len=0.2, corr_len_z=0.2)


@pytest.fixture(scope="module")
def R():
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return R


def fields(n, S, a_bl, n_bl, seed=3, thetas=True):
    model = O.soil_model(a_bl, n_bl)
    f = O.sample_soil(n, n, S, model, seed=seed, **PHI1)
    return f if thetas else f[:3]


def compare_vg(R, n, S, steps, dt, a_bl=2.0, n_bl=1.6, cycle=2, thetas=True, alpha_shift=0.0, n_shift=0.0,
               rtol=1e-10, precision=0, **kw):
    f = fields(n, S, a_bl, n_bl, thetas=thetas)
    pb_o = O.infiltration_problem(nsteps=steps, dt=dt, gamma=cycle, **{**TIGHT, **kw})
    p_o, q_o, s_o, st_o = O.solve_batch_soil(pb_o, *f, alpha_shift=alpha_shift, n_shift=n_shift, nthreads=NTH)
    dev = torch.device("cuda:0")
    pb = R.Problem.infiltration(nx=n, nz=n, nsteps=steps, dt=dt, cycle=cycle, precision=precision,
                                **{**TIGHT, **kw})
    g = [torch.from_numpy(a).to(dev) for a in f]
    q, p, s, st, rc = R.solve_soil(pb, *g, alpha_shift=alpha_shift, n_shift=n_shift, want_p=True)
    q, p, s = q.cpu().numpy(), p.cpu().numpy(), s.cpu().numpy()
    assert np.array_equal(s, s_o), (s, s_o)
    ok = s_o == 0
    assert ok.sum() >= max(1, S // 2)
    rel_q = np.abs(q[ok] - q_o[ok]) / np.abs(q_o[ok])
    assert rel_q.max() <= rtol, rel_q.max()
    if precision == 0:
        rel_p = np.abs(p[ok] - p_o[ok]).max() / np.abs(p_o[ok]).max()
        assert rel_p <= rtol, rel_p
        assert abs(st.picard_iters - st_o.picard_iters) <= max(1, 0.01 * st_o.picard_iters)
        assert abs(st.mg_cycles - st_o.mg_cycles) <= max(2, 0.01 * st_o.mg_cycles)
    return q, q_o, s


@pytest.mark.parametrize("n,c", [(32, 0), (64, 0), (64, 2)])
def test_soil_fields_match_oracle(R, n, c):
    model = O.soil_model(3.0, 1.45)
    o = O.sample_soil(n, n, 4, model, seed=9, level=2, first_sample=5, coarsen_times=c, **PHI1)
    g = R.sample_soil(n, n, 4, R.soil_field_model(3.0, R.FieldModel(seed=9, **PHI1)), R.SoilModel(n_bl=1.45),
                      level=2, first_sample=5, coarsen_times=c)
    for a, b in zip(g, o):
        assert np.abs(a.cpu().numpy() - b).max() < 1e-12


@pytest.mark.parametrize("thetas", [True, False])
def test_soil_pair_matches_oracle(R, thetas):
    cov = dict(nu=0.5, corr_len=0.1, corr_len_z=0.01)
    fo, co = O.sample_soil_pair(64, 64, 3, O.soil_model(2.8, 1.55), seed=6, level=3, first_sample=4, **cov)
    fg, cg = R.sample_soil_pair(64, 64, 3, R.soil_field_model(2.8, R.FieldModel(seed=6, **cov)),
                                R.SoilModel(n_bl=1.55), level=3, first_sample=4, thetas=thetas)
    k = 5 if thetas else 3
    for a, b in list(zip(fg[:k], fo[:k])) + list(zip(cg[:k], co[:k])):
        assert np.abs(a.cpu().numpy() - b).max() < 1e-12


def test_soil_fields_without_thetas(R):
    g = R.sample_soil(32, 32, 3, R.soil_field_model(2.0, R.FieldModel.phi2()), R.SoilModel(n_bl=1.6),
                      thetas=False)
    assert g[3] is None and g[4] is None
    o = O.sample_soil(32, 32, 3, O.soil_model(2.0, 1.6), nu=0.5, corr_len=0.1, corr_len_z=0.01)
    for a, b in zip(g[:3], o[:3]):
        assert np.abs(a.cpu().numpy() - b).max() < 1e-12


@pytest.mark.parametrize("cycle", [1, 2])
def test_infiltration_fp64_matches_oracle(R, cycle):
    """32^2 x 12 samples, 6 steps of dt = 1/64 (h = 1/32, the cost study's
    coarsest setting), V and W(2,2) cycles."""
    compare_vg(R, 32, 12, 6, 1 / 64, cycle=cycle)


@pytest.mark.parametrize("n,S,steps", [(48, 5, 3), (16, 9, 4), (64, 4, 2)])
def test_infiltration_ragged_and_deep(R, n, S, steps):
    """Grids with odd coarsest levels (48 -> 3x3 coarsest), a shallow and a
    deeper hierarchy."""
    compare_vg(R, n, S, steps, 1 / 64)


def test_constant_thetas_and_continuation_shifts(R):
    """theta arrays absent (problem constants); alpha shifted by -0.1 and n by
    +0.2 (the (grad alpha, grad n) continuation of Sec. 5)."""
    compare_vg(R, 32, 8, 4, 1 / 64, thetas=False, alpha_shift=-0.1, n_shift=0.2)


def test_hard_parameters_statuses_match(R):
    """alpha 4, n 1.15 (the hard corner of Table alpha_n): whatever fails,
    fails on both sides; what converges agrees to 1e-10."""
    f = fields(32, 8, 4.0, 1.15)
    pb_o = O.infiltration_problem(nsteps=6, dt=1 / 64, picard_tol=1e-10, mg_tol=1e-12, picard_maxit=50,
                                  mg_maxit=200)
    _, q_o, s_o, _ = O.solve_batch_soil(pb_o, *f, nthreads=NTH)
    dev = torch.device("cuda:0")
    pb = R.Problem.infiltration(nx=32, nz=32, nsteps=6, dt=1 / 64, picard_tol=1e-10, mg_tol=1e-12,
                                picard_maxit=50, mg_maxit=200)
    q, _, s, _, _ = R.solve_soil(pb, *[torch.from_numpy(a).to(dev) for a in f])
    s = s.cpu().numpy()
    fail, fail_o = (s == 1) | (s == 3), (s_o == 1) | (s_o == 3)
    assert np.array_equal(fail, fail_o)
    ok = ~fail
    if ok.any():
        q = q.cpu().numpy()
        assert (np.abs(q[ok] - q_o[ok]) / np.abs(q_o[ok])).max() <= 1e-9


def test_infiltration_mixed_within_1e6(R):
    compare_vg(R, 64, 6, 3, 1 / 64, precision=1, rtol=1e-6)


def test_gardner_through_soil_entry_is_bitwise_solve_batch(R):
    """closure 0 through rich_solve_soil (no n, zero shift) is the same launch as
    rich_solve_batch: identical bits."""
    dev = torch.device("cuda:0")
    lk, al = O.sample_fields(32, 32, 6, seed=4)
    lk, al = torch.from_numpy(lk).to(dev), torch.from_numpy(al).to(dev)
    pb = R.Problem(nx=32, nz=32, nsteps=3, dt=0.01)
    q1, p1, s1, _, _ = R.solve_batch(pb, lk, al, 0.8, want_p=True)
    q2, p2, s2, _, _ = R.solve_soil(pb, lk, al, alpha_scale=0.8, want_p=True)
    assert torch.equal(q1.nan_to_num(7.0), q2.nan_to_num(7.0)) and torch.equal(p1, p2) and torch.equal(s1, s2)


def test_vg_invalid_calls(R):
    dev = torch.device("cuda:0")
    x = torch.zeros((1, 16, 16), dtype=torch.float64, device=dev)
    pb = R.Problem.infiltration(nx=16, nz=16, nsteps=1)
    with pytest.raises(R.RichError):
        R.solve_batch(pb, x, x)                      # the closure needs n
    with pytest.raises(R.RichError):
        R.solve_soil(pb, x, x)                       # n missing
    with pytest.raises(R.RichError):
        R.solve_soil(R.Problem.infiltration(nx=16, nz=16, closure=5), x, x, x)


def test_per_sample_counters_match_oracle(R):
    """rich_sample_counters: per-sample Picard iterations and W-cycles of the
    last solve equal the oracle's per-sample counts (cycle counts within the
    rounding-order slack of the parity tests)."""
    f = fields(32, 6, 2.0, 1.6, seed=8)
    pbo = O.infiltration_problem(nsteps=4, dt=1 / 64, **TIGHT)
    per = [O.solve_one_soil(pbo, *[a[s] for a in f])[3] for s in range(6)]
    dev = torch.device("cuda:0")
    pb = R.Problem.infiltration(nx=32, nz=32, nsteps=4, dt=1 / 64, **TIGHT)
    R.solve_soil(pb, *[torch.from_numpy(a).to(dev) for a in f])
    pic, mg = R.sample_counters(6)
    pic, mg = pic.cpu().numpy(), mg.cpu().numpy()
    for s in range(6):
        assert abs(pic[s] - per[s].picard_iters) <= 1
        assert abs(mg[s] - per[s].mg_cycles) <= max(2, 0.01 * per[s].mg_cycles)
    with pytest.raises(R.RichError):
        R.sample_counters(7)


def test_vg_w_cycle_block_shapes_bitwise(R):
    """The van Genuchten W-cycle kernels of all launch shapes agree bit for bit."""
    f = fields(32, 6, 2.0, 1.6, seed=11)
    dev = torch.device("cuda:0")
    g = [torch.from_numpy(x).to(dev) for x in f]
    pb = R.Problem.infiltration(nx=32, nz=32, nsteps=3, dt=1 / 64)
    out = {}
    try:
        for bt in (32, 128, 256, 512, 1024):
            R.set_tuning(bt, 0)
            out[bt] = R.solve_soil(pb, *g, want_p=True)
    finally:
        R.set_tuning(0, 0)
    for bt in (32, 128, 256, 1024):
        assert torch.equal(out[bt][1], out[512][1]) and torch.equal(out[bt][2], out[512][2])
