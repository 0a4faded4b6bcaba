"""Pins of the oracle's van Genuchten-Mualem physics (Sec. 2.1 and the
infiltration problem of Sec. 4.3) and of its five-field soil sampler
(Table soilparams), each against mathematics, not against a retyped formula:
the Mualem integral evaluated by quadrature, C as the derivative of theta,
the n = 2 closed form, the saturated limit against a dense direct solve,
discrete mass conservation, a manufactured solution and the field marginals.
"""
import numpy as np
import pytest

import oracle as O
from tests.test_oracle_pins import hydraulic_head_dense_solve

VG = O.VAN_GENUCHTEN


def vg(p, a, n, Ks=1.0, tr=0.05, ts=0.5):
    return O.closure(VG, Ks, a, n, tr, ts, p)


# ---------------------------------------------------------------- closure
@pytest.mark.parametrize("a,n", [(3.0, 1.45), (2.8, 1.55), (1.0, 2.5), (0.4, 1.15)])
def test_krw_is_the_mualem_integral(a, n):
    """Eq. Krw1: K_rw(S) = S^(1/2) [int_0^S dS/|p(S)| / int_0^1 dS/|p(S)|]^2 with
    p(S) the inverse of Eq. Sw, by adaptive quadrature (substituting S = u^k
    to tame the endpoint singularities) against the closed form of Eq. Krw."""
    from scipy.integrate import quad
    m = 1.0 - 1.0 / n

    def inv_abs_p(S):                      # 1/|p| = a / (S^(-1/m) - 1)^(1/n)
        return a / (S ** (-1.0 / m) - 1.0) ** (1.0 / n)

    def inv_abs_p_v(v):                    # the same in v = 1 - S, without cancellation
        return a / np.expm1(-np.log1p(-v) / m) ** (1.0 / n)

    def integral(S):
        # near S = 1, 1/|p| ~ v^(-1/n): the upper piece in v = w^4 (smooth in w)
        lo = quad(inv_abs_p, 0.0, min(S, 0.5), epsabs=0, epsrel=1e-13, limit=400)[0]
        if S <= 0.5:
            return lo
        k = 4.0
        g = lambda w: inv_abs_p_v(w ** k) * k * w ** (k - 1.0)
        return lo + quad(g, (1.0 - S) ** (1.0 / k), 0.5 ** (1.0 / k), epsabs=0, epsrel=1e-13, limit=400)[0]

    full = integral(1.0)
    for p in (-0.01, -0.1, -0.4, -1.0, -3.0):
        K, th, C = vg(p, a, n)
        S = (th - 0.05) / (0.5 - 0.05)
        ref = np.sqrt(S) * (integral(S) / full) ** 2
        assert abs(K / ref - 1.0) < 1e-8, (p, K, ref)


@pytest.mark.parametrize("a,n", [(3.0, 1.45), (1.0, 2.0), (0.5, 3.0)])
def test_capacity_is_dtheta_dp(a, n):
    """Eq. sc_van is the derivative of theta(p) of Eq. Sw: central differences
    with one Richardson step (truncation O(e^4), e = |p|/1000)."""
    th = lambda x: vg(x, a, n)[1]
    for p in (-1e-3, -0.05, -0.4, -2.0):
        e = 1e-3 * abs(p)
        d1 = (th(p + e) - th(p - e)) / (2 * e)
        d2 = (th(p + e / 2) - th(p - e / 2)) / e
        dth = (4 * d2 - d1) / 3
        C = vg(p, a, n)[2]
        assert abs(C - dth) < 1e-8 * abs(C) + 4e-16 / e, (p, C, dth)


def test_n2_closed_form_and_saturated_branch():
    """n = 2 (m = 1/2): S = (1 + (a p)^2)^(-1/2) and
    K_rw = S^(1/2) (1 - a|p| / sqrt(1 + a^2 p^2))^2; p >= 0 is saturated; theta
    and K are continuous at p = 0."""
    a, Ks, tr, ts = 1.7, 2.3, 0.07, 0.43
    for p in (-1e-4, -0.2, -1.0, -5.0):
        K, th, C = O.closure(VG, Ks, a, 2.0, tr, ts, p)
        S = (1 + (a * p) ** 2) ** -0.5
        assert abs(th - (tr + (ts - tr) * S)) < 1e-15
        x = a * abs(p) / np.sqrt(1 + (a * p) ** 2)
        assert abs(K - Ks * np.sqrt(S) * (1 - x) ** 2) < 1e-14 * Ks
    assert O.closure(VG, Ks, a, 2.0, tr, ts, 0.3) == (Ks, ts, 0.0)
    K0, th0, _ = O.closure(VG, Ks, a, 1.3, tr, ts, -1e-13)
    assert abs(K0 - Ks) < 1e-3 * Ks and abs(th0 - ts) < 1e-12


# ----------------------------------------------------------- discrete pins
def vg_problem(**kw):
    d = dict(nsteps=1, dt=0.01, picard_tol=1e-10, picard_maxit=100, mg_tol=1e-12, mg_maxit=200)
    d.update(kw)
    return O.infiltration_problem(**d)


@pytest.mark.parametrize("shape", [(8, 8), (16, 8)])
def test_saturated_limit_matches_dense_solve(shape):
    """Heads >= 0 everywhere (p_top = 0.3, p_bottom = 0.8): the van Genuchten
    closure reduces to K = Ks and the steady solve is the hydraulic-head system
    of an incidence-matrix construction, solved densely."""
    nz, nx = shape
    rng = np.random.default_rng(2)
    lnks = rng.normal(size=(1, nz, nx))
    n = np.full((1, nz, nx), 1.6)
    pb = vg_problem(dt=1e10, p_top=0.3, p_bottom=0.8, p_init=0.5, init_decay=0.0)
    p, q, st, _ = O.solve_batch_soil(pb, lnks, np.full((1, nz, nx), 2.0), n)
    assert st[0] == 0
    assert np.all(p >= 0)
    ref = hydraulic_head_dense_solve(lnks[0], p_top=0.3, p_bot=0.8)
    assert np.abs(p[0] - ref).max() < 1e-9


def test_mass_balance_with_soil_fields():
    """Mixed form conserves mass (Sec. 4.1) with per-cell theta_s, theta_r:
    the change of stored water over a step equals dt times the net boundary
    inflow at the new time, to the Picard tolerance."""
    nx = nz = 32
    model = O.soil_model(2.0, 1.6)
    lk, al, n, ts, tr = O.sample_soil(nx, nz, 1, model, seed=7, corr_len=0.2, corr_len_z=0.2, nu=1.0)
    pb = vg_problem(dt=0.005)
    h = 1.0 / nz

    def water(p):
        th = np.array([[vg(p[j, i], al[0, j, i], n[0, j, i], tr=tr[0, j, i], ts=ts[0, j, i])[1]
                        for i in range(nx)] for j in range(nz)])
        return h * h * th.sum()

    def outflow(p):
        kt = np.array([vg(pb.p_top, al[0, -1, i], n[0, -1, i], Ks=np.exp(lk[0, -1, i]))[0] for i in range(nx)])
        kb = np.array([vg(pb.p_bottom, al[0, 0, i], n[0, 0, i], Ks=np.exp(lk[0, 0, i]))[0] for i in range(nx)])
        q_top = -kt * ((pb.p_top - p[-1]) / (h / 2) + 1)
        q_bot = kb * ((p[0] - pb.p_bottom) / (h / 2) + 1)
        return h * (q_top.sum() + q_bot.sum())

    z = (np.arange(nz) + 0.5) * h
    p = np.repeat((-0.4 * (1 - np.exp(-80 * z)))[:, None], nx, axis=1)
    for step in range(3):
        p1, q, rc, _ = O.solve_one_soil(pb, lk[0], al[0], n[0], ts[0], tr[0], p_init=p)
        assert rc == 0
        dW = water(p1) - water(p)
        flux = pb.dt * outflow(p1)
        scale = pb.dt * h * np.exp(lk[0, 0]).sum()
        assert abs(dW + flux) < 1e-7 * scale, (step, dW, flux)
        p = p1


def _mms_vg(M):
    import sympy as sp
    x, z = sp.symbols("x z")
    pstar = -0.3 - 0.4 * z + 0.1 * sp.sin(sp.pi * z) * sp.cos(sp.pi * x)
    lnks = 0.3 * sp.cos(sp.pi * x) * sp.sin(sp.pi * z) + 0.1 * z
    al = 1.5 + 0.3 * sp.sin(sp.pi * x) * sp.cos(sp.pi * z)
    nn = 1.8 + 0.2 * sp.cos(sp.pi * x) * sp.cos(sp.pi * z)
    m = 1 - 1 / nn
    an = (-al * pstar) ** nn
    S = (1 + an) ** (-m)
    krw = sp.sqrt(S) * (1 - (an / (1 + an)) ** m) ** 2
    K = sp.exp(lnks) * krw
    src = sp.diff(-K * sp.diff(pstar, x), x) + sp.diff(-K * (sp.diff(pstar, z) + 1), z)
    fn = {k: sp.lambdify((x, z), e, "numpy") for k, e in dict(p=pstar, lnks=lnks, al=al, n=nn, src=src).items()}
    c = (np.arange(M) + 0.5) / M
    X, Z = np.meshgrid(c, c)
    return {k: np.broadcast_to(f(X, Z), X.shape).astype(np.float64) for k, f in fn.items()}


@pytest.mark.slow
def test_mms_second_order_van_genuchten():
    """Manufactured unsaturated steady solution p* < 0 with smooth Ks, alpha, n
    fields and the source f = -div(K(p*)(grad p* + e_z)) of the van
    Genuchten-Mualem conductivity: the discrete error is O(h^2)."""
    errs = []
    for M in (16, 32, 64, 128):
        d = _mms_vg(M)
        pb = vg_problem(dt=1e10, p_top=-0.7, p_bottom=-0.3, init_decay=0.0, picard_maxit=200)
        p, q, rc, _ = O.solve_one_soil(pb, d["lnks"], d["al"], d["n"], src=d["src"], p_init=d["p"])
        assert rc == 0
        errs.append(np.abs(p - d["p"]).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.85), (errs, orders)


def test_infiltration_initial_profile_and_boundary_flux_sign():
    """Eq. travellingwave: after zero steps the head is -0.4 (1 - exp(-80 z)) at
    the cell centres; after a few steps water enters through the wet bottom
    (p = 0.1), so the outward bottom flux is negative (inflow)."""
    nz = nx = 16
    model = O.soil_model(2.0, 1.6)
    f = O.sample_soil(nx, nz, 2, model, seed=1, corr_len=0.2, corr_len_z=0.2, nu=1.0)
    p0, q0, st0, _ = O.solve_batch_soil(vg_problem(nsteps=0), *f)
    z = (np.arange(nz) + 0.5) / nz
    assert np.abs(p0 - (-0.4 * (1 - np.exp(-80 * z)))[None, :, None]).max() < 1e-15
    p, q, st, _ = O.solve_batch_soil(vg_problem(nsteps=4, dt=1 / 64), *f)
    assert np.all(st == 0) and np.all(q < 0)


# ----------------------------------------------------------------- sampler
def test_soil_fields_marginals_and_shared_streams():
    """Table soilparams: alpha, n, theta_s, theta_r are uniform on baseline +-
    half-width (KS test), ln Ks = ln Ks_bl + Z; fields 0 and 1 are the same
    draws as the two-field sampler (noise streams 0 and 1)."""
    from scipy import stats
    nx = nz = 16
    model = O.soil_model(3.0, 1.45)
    lk, al, n, ts, tr = O.sample_soil(nx, nz, 2000, model, seed=5, corr_len=0.2, corr_len_z=0.2, nu=1.0)
    for arr, lo, w in ((al, 2.8, 0.4), (n, 1.40, 0.1), (ts, 0.45, 0.1), (tr, 0.045, 0.01)):
        assert arr.min() > lo and arr.max() < lo + w
        assert stats.kstest((arr[:, 3, 5] - lo) / w, "uniform").pvalue > 1e-3
    assert abs(lk.mean() - np.log(0.2)) < 0.05
    lk2, al2 = O.sample_fields(nx, nz, 2000, seed=5, corr_len=0.2, corr_len_z=0.2, nu=1.0,
                               alpha_lo=2.8, alpha_span=0.4)
    assert np.abs(lk - np.log(0.2) - lk2).max() < 1e-13
    assert np.array_equal(al, al2)
    # different streams: n is not a function of alpha
    assert abs(np.corrcoef(al[:, 3, 5], n[:, 3, 5])[0, 1]) < 0.1


def test_soil_pair_members():
    """Covariance-upscaled soil couples (Appendix A): the fine members are the
    plain soil draw, the coarse ln Ks / alpha are the two-field pair's coarse
    members, and the coarse n, theta_s, theta_r keep uniform marginals."""
    from scipy import stats
    model = O.soil_model(2.8, 1.55)
    cov = dict(nu=0.5, corr_len=0.1, corr_len_z=0.01)
    fine, coarse = O.sample_soil_pair(32, 32, 800, model, seed=2, level=1, **cov)
    plain = O.sample_soil(32, 32, 800, model, seed=2, level=1, **cov)
    for a, b in zip(fine, plain):
        assert np.array_equal(a, b)
    lkf, alf, lkc, alc = O.sample_fields_pair(32, 32, 800, seed=2, level=1, alpha_lo=model.alpha_lo,
                                              alpha_span=model.alpha_span, **cov)
    assert np.abs(coarse[0] - np.log(0.2) - lkc).max() < 1e-13 and np.array_equal(coarse[1], alc)
    for arr, lo, w in ((coarse[2], 1.50, 0.1), (coarse[3], 0.45, 0.1), (coarse[4], 0.045, 0.01)):
        assert arr.shape == (800, 16, 16) and arr.min() > lo and arr.max() < lo + w
        assert stats.kstest((arr[:, 5, 9] - lo) / w, "uniform").pvalue > 1e-3


# ------------------------------------------------------- van Genuchten MLMC
VG_MLMC = dict(theta_r=0.05, theta_s=0.5, p_top=-0.4, p_bottom=0.1, p_init=-0.4, closure=1, init_decay=80.0,
               gamma=2, picard_tol=1e-8, mg_tol=1e-10, nu=1.0, corr_len=0.2, corr_len_z=0.2)


def test_vg_mlmc_continuation_reading():
    """The additive continuation of Sec. 5.2 as read here: with every level
    fixed (fixed_levels = L + 1) it is the estimator without continuation,
    exactly; with it, the finest level still solves the original (alpha, n),
    so its fine members equal a plain solve of the same fields."""
    ns, n0, s0, T = (6, 4, 3), 8, 2, 0.25
    model = O.soil_model(2.0, 1.6)
    kw = dict(soil=model, d_alpha=0.1, d_n=0.1, coupling=0, **VG_MLMC)
    a = O.mlmc_estimate(ns, n0, s0, T, continuation=0, **kw)
    b = O.mlmc_estimate(ns, n0, s0, T, continuation=1, fixed_levels=3, **kw)
    c = O.mlmc_estimate(ns, n0, s0, T, continuation=1, fixed_levels=1, **kw)
    for la, lb in zip(a, b):
        assert np.array_equal(la["qf"], lb["qf"]) and np.array_equal(la["qc"], lb["qc"])
    assert np.array_equal(c[2]["qf"], a[2]["qf"])                  # finest: original parameters
    assert not np.array_equal(c[1]["qf"], a[1]["qf"])              # below it: shifted
    L = len(ns) - 1
    fine = O.sample_soil(n0 << L, n0 << L, ns[L], model, level=L, nu=1.0, corr_len=0.2, corr_len_z=0.2)
    pb = O.make_problem(nsteps=s0 << L, dt=T / (s0 << L), **{k: v for k, v in VG_MLMC.items()
                                                            if k not in ("nu", "corr_len", "corr_len_z")})
    _, q, st, _ = O.solve_batch_soil(pb, *fine, want_p=False)
    assert np.array_equal(q[st == 0], c[L]["qf"])


def test_vg_mlmc_telescoping_consistency():
    """Coupling 0 (finest-grid draws averaged down): the fine member of pair l
    and the coarse member of pair l+1 are the same grid, time step and shifted
    parameters on fields of the same law, so their means agree within 4
    standard errors (the telescoping sum of Eq. telescope_ch6 is exact)."""
    ns = (600, 300)
    out = O.mlmc_estimate(ns, 8, 2, 0.25, coupling=0, continuation=1, soil=O.soil_model(2.0, 1.6), d_alpha=0.2,
                          d_n=0.2, **VG_MLMC)
    f0, c1 = out[0]["qf"], out[1]["qc"]
    se = np.sqrt(f0.var(ddof=1) / f0.size + c1.var(ddof=1) / c1.size)
    assert abs(f0.mean() - c1.mean()) < 4 * se, (f0.mean(), c1.mean(), se)
