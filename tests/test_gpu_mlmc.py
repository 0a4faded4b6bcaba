"""MLMC with parametric continuation on the GPU vs the oracle's restatement of
Sec. 5, and the telescoping consistency of the coupled estimator."""
import numpy as np
import pytest

import oracle as O
from tests.inputs import PHYSICS, SOLVER

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build
    build.build()
    return R


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("coupling", [0, 1, 2])
def test_mlmc_matches_oracle(R, coupling):
    ns, n0, s0, T = (24, 12, 6), 8, 2, 0.04
    cfg = R.MlmcConfig(nsamples=ns, n0=n0, steps0=s0, t_final=T, coupling=coupling, eps=1e-3,
                       problem=R.Problem(**PHYSICS, **SOLVER))
    g = R.mlmc_estimate(cfg)
    o = O.mlmc_estimate(ns, n0, s0, T, coupling=coupling, **PHYSICS, **SOLVER)
    for l, lev in enumerate(o):
        y, qf, qc = lev["y"], lev["qf"], lev["qc"]
        assert g["n"][l] == y.size and g["failed"][l] == lev["failed"]
        assert rel(g["mean"][l], y.mean()) < 1e-9
        assert rel(g["var"][l], y.var(ddof=1)) < 1e-8
        assert rel(g["mean_f"][l], qf.mean()) < 1e-9
        assert rel(g["var_f"][l], qf.var(ddof=1)) < 1e-8
        if l > 0:
            assert rel(g["mean_c"][l], qc.mean()) < 1e-9
            assert rel(g["var_c"][l], qc.var(ddof=1)) < 1e-8
    est = sum(lev["y"].mean() for lev in o)
    rmse = np.sqrt(sum(lev["y"].var(ddof=1) / lev["y"].size for lev in o))
    assert rel(g["estimate"], est) < 1e-9 and rel(g["rmse"], rmse) < 1e-8
    # optimal allocation and cost from the GPU's own V_l and C_l (Eq. MLMCSAMP_ch6)
    s = sum(np.sqrt(v * c) for v, c in zip(g["var"], g["cost"]))
    assert rel(g["w_eps"], s * s / 1e-6) < 1e-12
    assert all(c > 0 for c in g["cost"])
    # full-occupancy cost: the solves' SM-seconds spread over the GPU; these
    # small batches leave most SMs idle, so it is below the wall-clock cost
    assert all(0 < cs <= 1.05 * c for cs, c in zip(g["cost_sm"], g["cost"]))
    s_sm = sum(np.sqrt(v * c) for v, c in zip(g["var"], g["cost_sm"]))
    assert rel(g["w_eps_sm"], s_sm * s_sm / 1e-6) < 1e-12


def test_level_variances_of_a_nearly_constant_qoi(R):
    """With sigma^2 = 1e-16 and a constant alpha every sample solves nearly the
    same problem: mean^2 / var of Y_l and Q_l is ~1e16, where a one-pass
    (sum Y^2 - n mean^2) variance is quantised in steps (~1e-15) larger than
    the variance itself (it returns 0, negative values or a multiple).  The
    estimator's shifted sums still give the oracle's two-pass variances;
    the 25 % bound covers the GPU/oracle difference of single QoIs (~1e-13
    relative) against a sample spread of ~2e-8."""
    ns, n0, s0, T = (24, 12, 6), 8, 2, 0.04
    cfg = R.MlmcConfig(nsamples=ns, n0=n0, steps0=s0, t_final=T, coupling=0, eps=1e-3,
                       model=R.FieldModel(sigma2=1e-16, alpha_span=0.0),
                       problem=R.Problem(**PHYSICS, **SOLVER))
    g = R.mlmc_estimate(cfg)
    o = O.mlmc_estimate(ns, n0, s0, T, coupling=0, sigma2=1e-16, alpha_span=0.0, **PHYSICS, **SOLVER)
    for l, lev in enumerate(o):
        y, qf = lev["y"], lev["qf"]
        assert g["n"][l] == y.size and g["failed"][l] == 0
        assert y.mean() ** 2 / y.var(ddof=1) > 1e14
        assert rel(g["mean"][l], y.mean()) < 1e-9 and rel(g["mean_f"][l], qf.mean()) < 1e-9
        assert g["var"][l] > 0 and g["var_f"][l] > 0
        if y.size >= 12:
            assert rel(g["var"][l], y.var(ddof=1)) < 0.25
            assert rel(g["var_f"][l], qf.var(ddof=1)) < 0.25


def close(a, b, tol):
    """Relative agreement; two NaNs (a level with fewer than two usable pairs
    has no variance) agree."""
    if np.isnan(a) or np.isnan(b):
        return np.isnan(a) and np.isnan(b)
    return rel(a, b) < tol


@pytest.mark.slow
def test_mlmc_configured_hierarchy_matches_oracle(R):
    """The configured five-level hierarchy (16^2 ... 256^2 with 5 2^l steps to
    T = 0.1, alpha_l = alpha (l+1)/5, covariance upscaling, Sec. 5 Eq.
    MLMCestimator_ch6) with N_l reduced to 16/8/4/2/2: the GPU's level
    statistics equal the oracle's restatement of the estimator."""
    ns, n0, s0, T = (16, 8, 4, 2, 2), 16, 5, 0.1
    cfg = R.MlmcConfig(nsamples=ns, n0=n0, steps0=s0, t_final=T, coupling=2, eps=1e-3,
                       problem=R.Problem(**PHYSICS, **SOLVER))
    g = R.mlmc_estimate(cfg)
    o = O.mlmc_estimate(ns, n0, s0, T, coupling=2, **PHYSICS, **SOLVER)
    for l, lev in enumerate(o):
        y, qf, qc = lev["y"], lev["qf"], lev["qc"]
        assert g["n"][l] == y.size and g["failed"][l] == lev["failed"]
        assert close(g["mean"][l], y.mean() if y.size else np.nan, 1e-9)
        assert close(g["var"][l], y.var(ddof=1) if y.size > 1 else np.nan, 1e-8)
        assert close(g["mean_f"][l], qf.mean() if y.size else np.nan, 1e-9)
        if l > 0:
            assert close(g["mean_c"][l], qc.mean() if y.size else np.nan, 1e-9)
    assert sum(g["n"]) >= sum(ns) // 2


@pytest.mark.parametrize("coupling", [0, 2])
def test_mlmc_grid_only_bias_matches_oracle(R, coupling):
    """Grid-only bias pairs (Eq. discErr): finest-level pairs with both members
    at the original alpha, from their own noise stream (level key 64); the
    bias |E[Q_L - Q_{L-1}]| and the total RMSE sqrt(bias^2 + sum V_l/N_l) (Eq.
    MSEMLMC_ch6) equal the oracle's restatement, and the level statistics do
    not change when the pairs are added."""
    ns, n0, s0, T, nb = (12, 6, 4), 8, 2, 0.04, 6
    base = dict(nsamples=ns, n0=n0, steps0=s0, t_final=T, coupling=coupling, eps=1e-3,
                problem=R.Problem(**PHYSICS, **SOLVER))
    g = R.mlmc_estimate(R.MlmcConfig(**base, bias_pairs=nb))
    g0 = R.mlmc_estimate(R.MlmcConfig(**base))
    assert g0["mean"] == g["mean"] and g0["var"] == g["var"] and g0["bias_pairs"] == 0
    L = len(ns) - 1
    M = n0 << L
    if coupling == 2:
        lk, al, lkc, alc = O.sample_fields_pair(M, M, nb, seed=0, level=64)
    else:
        lk, al = O.sample_fields(M, M, nb, seed=0, level=64)
        blk = lambda x: x.reshape(nb, M // 2, 2, M // 2, 2).mean(axis=(2, 4))
        lkc, alc = blk(lk), blk(al)
    pf = O.make_problem(nsteps=s0 << L, dt=T / (s0 << L), **PHYSICS, **SOLVER)
    pc = O.make_problem(nsteps=s0 << (L - 1), dt=T / (s0 << (L - 1)), **PHYSICS, **SOLVER)
    _, qf, sf, _ = O.solve_batch(pf, lk, al, 1.0, want_p=False)
    _, qc, sc, _ = O.solve_batch(pc, lkc, alc, 1.0, want_p=False)
    bad = np.isin(sf, (1, 3)) | np.isin(sc, (1, 3))
    y = (qf - qc)[~bad]
    assert g["bias_pairs"] == y.size >= nb // 2
    assert rel(g["bias_grid"], abs(y.mean())) < 1e-9
    assert rel(g["total_rmse"], np.sqrt(abs(y.mean()) ** 2 + g["rmse"] ** 2)) < 1e-9
    assert rel(g["bias_grid_se"], y.std(ddof=1) / np.sqrt(y.size)) < 1e-7
    extra = 0
    b = abs(y.mean())
    while b > 1e-3 / np.sqrt(2):
        b, extra = b / 2, extra + 1
    assert g["levels_for_eps"] == len(ns) + extra


def test_mixed_precision_mlmc_close_to_fp64(R):
    """The estimator with FP32 V-cycles inside FP64 defect correction: every
    level's pair counts equal the FP64 run's and its means of Q_l and of
    Y_l agree with them to 1e-6 of the QoI scale (the mixed path's QoI bar)."""
    base = dict(nsamples=(24, 12, 6), n0=8, steps0=2, t_final=0.04, coupling=2, eps=1e-3)
    g64 = R.mlmc_estimate(R.MlmcConfig(**base, problem=R.Problem(**PHYSICS, **SOLVER)))
    g32 = R.mlmc_estimate(R.MlmcConfig(**base, problem=R.Problem(precision=R.MIXED, **PHYSICS, **SOLVER)))
    scale = max(abs(v) for v in g64["mean_f"])
    assert g64["n"] == g32["n"] and g64["failed"] == g32["failed"]
    for l in range(3):
        assert abs(g32["mean"][l] - g64["mean"][l]) <= 1e-6 * scale, l
        assert abs(g32["mean_f"][l] - g64["mean_f"][l]) <= 1e-6 * scale, l


def test_mlmc_telescoping_consistency(R):
    """Exact coupling: the level-l fine member (pair l) and the level-l coarse
    member (pair l+1) have the same law, so their means agree within 4 sigma."""
    ns = (1200, 600, 300)
    cfg = R.MlmcConfig(nsamples=ns, n0=8, steps0=2, t_final=0.04, coupling=0,
                       problem=R.Problem(**PHYSICS, **SOLVER))
    g = R.mlmc_estimate(cfg)
    for l in range(len(ns) - 1):
        d = g["mean_f"][l] - g["mean_c"][l + 1]
        se = np.sqrt(g["var_f"][l] / g["n"][l] + g["var_c"][l + 1] / g["n"][l + 1])
        assert abs(d) < 4 * se, (l, d, se)


def test_adaptive_pc_mlmc(R):
    """Algorithm PC_MLMC: the final N_l (pairs with a defined QoI, the ones the
    variance counts) cover the optimal allocation computed from the final V_l
    and C_l, so the sampling RMSE is at most eps whatever the costs measured in
    this run (they set the allocation); since
    each level continues its own sample stream, the statistics equal a one-shot
    estimate with the final N_l."""
    eps = 0.02
    cfg = R.MlmcConfig(nsamples=(16, 8, 4), n0=8, steps0=2, t_final=0.04, coupling=2, eps=eps,
                       problem=R.Problem(**PHYSICS, **SOLVER))
    a = R.mlmc_adaptive(cfg, max_rounds=8)
    assert a["rounds"] >= 2
    n_final = [n + f for n, f in zip(a["n"], a["failed"])]
    assert all(n >= w for n, w in zip(n_final, (16, 8, 4)))
    assert all(n >= np.ceil(no) - 1e-9 for n, no in zip(a["n"], a["n_opt"])) or a["rounds"] == 8
    assert a["rmse"] <= eps * (1 + 1e-9) or a["rounds"] == 8
    one = R.mlmc_estimate(R.MlmcConfig(nsamples=tuple(n_final), n0=8, steps0=2, t_final=0.04, coupling=2,
                                       eps=eps, problem=R.Problem(**PHYSICS, **SOLVER)))
    for k in ("n", "failed"):
        assert one[k] == a[k]
    for l in range(3):
        assert rel(one["mean"][l], a["mean"][l]) < 1e-9 and rel(one["var"][l], a["var"][l]) < 1e-8


def test_per_level_tuning_keeps_fp64_statistics(R):
    base = dict(nsamples=(24, 12, 6), n0=8, steps0=2, t_final=0.04, coupling=2, eps=1e-3,
                problem=R.Problem(**PHYSICS, **SOLVER))
    g0 = R.mlmc_estimate(R.MlmcConfig(**base))
    g1 = R.mlmc_estimate(R.MlmcConfig(**base, tune_threads=(1024, 512, 1024)))
    assert g0["mean"] == g1["mean"] and g0["var"] == g1["var"]


VG_TIGHT = dict(picard_tol=1e-10, mg_tol=1e-12, picard_maxit=60, mg_maxit=200)
VG_PHYS = dict(theta_r=0.05, theta_s=0.5, p_top=-0.4, p_bottom=0.1, p_init=-0.4, closure=1, init_decay=80.0,
               nu1=2, nu2=2, gamma=2, **VG_TIGHT)


@pytest.mark.parametrize("coupling", [0, 1, 2])
def test_van_genuchten_mlmc_matches_oracle(R, coupling):
    """The paper's MLMC setting (Sec. 5.2): infiltration problem, five soil
    fields of Table soilparams with Matern Phi_1 covariance, W(2,2) cycles,
    h_l = dt_l, and the additive (d_alpha, d_n) continuation with the finest
    level fixed; level statistics equal the oracle's to 1e-9."""
    ns, n0, s0, T = (20, 10, 6), 8, 2, 0.25
    cov = dict(nu=1.0, corr_len=0.2, corr_len_z=0.2)
    cfg = R.MlmcConfig(nsamples=ns, n0=n0, steps0=s0, t_final=T, coupling=coupling, eps=1e-3,
                       problem=R.Problem.infiltration(**VG_TIGHT),
                       model=R.soil_field_model(2.0, R.FieldModel(seed=0, **cov)), soil=R.SoilModel(n_bl=1.6),
                       d_alpha=0.1, d_n=0.1, fixed_levels=1)
    g = R.mlmc_estimate(cfg)
    o = O.mlmc_estimate(ns, n0, s0, T, coupling=coupling, soil=O.soil_model(2.0, 1.6), d_alpha=0.1, d_n=0.1,
                        fixed_levels=1, **cov, **VG_PHYS)
    for l, lev in enumerate(o):
        y, qf, qc = lev["y"], lev["qf"], lev["qc"]
        assert g["n"][l] == y.size and g["failed"][l] == lev["failed"]
        assert y.size >= ns[l] // 2
        assert rel(g["mean"][l], y.mean()) < 1e-9
        assert rel(g["var"][l], y.var(ddof=1)) < 1e-8
        assert rel(g["mean_f"][l], qf.mean()) < 1e-9
        if l > 0:
            assert rel(g["mean_c"][l], qc.mean()) < 1e-9
