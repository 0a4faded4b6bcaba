"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these tests re-types an oracle formula and compares: each one checks a
closed form, an invariant, a brute-force or library computation, or a published
known-answer vector, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle as O
from tests.inputs import PHYSICS, SOLVER

HERE = os.path.dirname(os.path.abspath(__file__))


def problem(**kw):
    d = dict(PHYSICS)
    d.update(SOLVER)
    d.update(dict(nsteps=1, dt=0.01))
    d.update(kw)
    return O.make_problem(**d)


# ------------------------------------------------------------------ generator
def test_philox_known_answers():
    """Philox4x32-10 reproduces its published known-answer vectors (SC'11)."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = O.philox4x32_10(w[0:4], w[4:6])
        assert [int(v) for v in out] == w[6:10]


def test_white_noise_is_standard_normal():
    from scipy import stats
    y = np.concatenate([O.white_noise(0, 0, s, f, 4096) for s in range(8) for f in range(2)])
    assert abs(y.mean()) < 5 / np.sqrt(y.size)
    assert abs(y.var() - 1) < 5 * np.sqrt(2 / y.size)
    assert stats.kstest(y, "norm").pvalue > 1e-3
    # distinct (sample, field, level) streams are uncorrelated
    a, b = O.white_noise(0, 0, 1, 0, 8192), O.white_noise(0, 0, 1, 1, 8192)
    c = O.white_noise(0, 1, 1, 0, 8192)
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / np.sqrt(8192)
    assert abs(np.corrcoef(a, c)[0, 1]) < 5 / np.sqrt(8192)


# ------------------------------------------------------------------------ FFT
@pytest.mark.parametrize("shape", [(8, 8), (16, 32), (64, 4), (1, 16)])
def test_fft_matches_library(shape):
    rng = np.random.default_rng(1)
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    X = O.fft2(x)
    ref = np.fft.fft2(x)
    assert np.abs(X - ref).max() < 1e-12 * np.abs(ref).max()
    back = O.fft2(X, inverse=True)
    assert np.abs(back - x).max() < 1e-13 * np.abs(x).max()


# ------------------------------------------------------------- FFT-MA fields
@pytest.mark.parametrize("px,pz,h,lam", [(16, 16, 1 / 8, 0.3), (32, 16, 1 / 8, 0.2)])
def test_fftma_exact_covariance(px, pz, h, lam):
    """The circular autocorrelation of s = F^-1 sqrt(F c) equals the torus
    covariance c itself (Appendix A, Eqs. convol1, product1), computed here by
    brute force over all lags."""
    sq, ratio = O.fftma_sqrt_spectrum(px, pz, h, 1.0, lam)
    assert ratio >= -1e-12
    s = np.real(np.fft.ifft2(sq))
    for b in range(pz):
        for a in range(px):
            acorr = np.sum(s * np.roll(np.roll(s, -b, axis=0), -a, axis=1))
            dx, dz = min(a, px - a) * h, min(b, pz - b) * h
            assert abs(acorr - np.exp(-np.hypot(dx, dz) / lam)) < 1e-12


def test_fields_empirical_covariance_and_marginals():
    """4096 fields on 16x16: ln Ks is zero-mean with Cov(r) = exp(-r/0.3) at
    lags up to 8 cells (within 5 standard errors); alpha = 0.5 + 1.5 Phi(g) has
    a uniform marginal on (0.5, 2) (the configured bounded field)."""
    from scipy import stats
    n, S, lam = 16, 4096, 0.3
    lnks, alpha = O.sample_fields(n, n, S, seed=0)
    h = 1.0 / n
    assert abs(lnks.mean()) < 0.05
    for field in (lnks, None):
        z = lnks if field is not None else np.sqrt(2) * stats.norm.ppf((alpha - 0.5) / 1.5) / np.sqrt(2)
        for axis in (1, 2):
            for lag in range(0, 9):
                a = np.take(z, np.arange(0, n - lag), axis=axis)
                b = np.take(z, np.arange(lag, n), axis=axis)
                per_sample = (a * b).mean(axis=(1, 2))
                se = per_sample.std(ddof=1) / np.sqrt(S)
                target = np.exp(-lag * h / lam)
                assert abs(per_sample.mean() - target) < 5 * se + 1e-3, (axis, lag)
    assert alpha.min() > 0.5 and alpha.max() < 2.0
    u = (alpha[:, 5, 7] - 0.5) / 1.5
    assert stats.kstest(u, "uniform").pvalue > 1e-3


# ------------------------------------------------- Matern covariance (Eq. nonIsotropic)
def test_bessel_k_matches_library():
    """The oracle's K_nu (trapezoidal rule on its integral representation)
    against scipy's modified Bessel function of the second kind."""
    from scipy import special
    for nu in (0.5, 1.0, 1.5, 2.5, 0.3, 3.7):
        for x in np.geomspace(1e-4, 100.0, 300):
            assert abs(O.bessel_k(nu, x) / special.kv(nu, x) - 1.0) < 1e-13, (nu, x)


def test_matern_special_cases():
    """Eq. nonIsotropic at half-integer nu has closed forms in x = 2 sqrt(nu) r:
    nu = 1/2 the exponential exp(-x) (= exp(-sqrt 2 r)), nu = 3/2 (1 + x) exp(-x),
    nu = 5/2 (1 + x + x^2/3) exp(-x); nu = 1 is sigma2 x K_1(x); large nu tends
    to the squared exponential exp(-r^2) (nu <= 16 is supported).  Anisotropy scales each axis by its
    own length; r = 0 gives the variance; nu = 0 is the configured exp(-|d|/l)."""
    from scipy import special
    lx, lz, s2 = 0.1, 0.01, 1.7
    rng = np.random.default_rng(1)
    for dx, dz in rng.uniform(0, 0.2, size=(20, 2)) * np.array([1.0, 0.1]):
        r = np.hypot(dx / lx, dz / lz)
        forms = {0.5: lambda x: np.exp(-x), 1.5: lambda x: (1 + x) * np.exp(-x),
                 2.5: lambda x: (1 + x + x * x / 3) * np.exp(-x), 1.0: lambda x: x * special.kv(1, x)}
        for nu, f in forms.items():
            x = 2 * np.sqrt(nu) * r
            got = O.covariance(dx, dz, sigma2=s2, corr_len=lx, corr_len_z=lz, nu=nu)
            assert abs(got - s2 * f(x)) < 1e-13 * s2, (nu, dx, dz)
    # towards the squared exponential: the gap halves as nu doubles (O(1/nu))
    gaps = [max(abs(O.covariance(r * lx, 0.0, corr_len=lx, nu=nu) - np.exp(-r * r)) for r in np.linspace(0, 3, 61))
            for nu in (4.0, 8.0, 16.0)]
    assert gaps[2] < 0.016 and 0.4 < gaps[1] / gaps[0] < 0.6 and 0.4 < gaps[2] / gaps[1] < 0.6, gaps
    assert O.covariance(0.0, 0.0, sigma2=s2, corr_len=lx, corr_len_z=lz, nu=1.0) == s2
    assert O.covariance(0.05, 0.0, corr_len=0.2, nu=1.0) == O.covariance(0.0, 0.05, corr_len=0.2, nu=1.0)
    assert abs(O.covariance(0.3, 0.4, corr_len=0.3) - np.exp(-0.5 / 0.3)) < 1e-15


@pytest.mark.parametrize("px,pz,h,lx,lz,nu", [(32, 32, 1 / 16, 0.2, 0.2, 1.0), (32, 64, 1 / 32, 0.1, 0.01, 0.5)])
def test_fftma_exact_covariance_matern(px, pz, h, lx, lz, nu):
    """Phi_1 = (1, 0.2, 0.2, 1) and Phi_2 = (0.5, 0.1, 0.01, 1) of the paper's
    Matern table: the circular autocorrelation of s = F^-1 sqrt(F c) equals the
    torus covariance, by brute force over all lags (Appendix A)."""
    from scipy import special
    sq, ratio = O.fftma_sqrt_spectrum(px, pz, h, 1.0, lx, corr_len_z=lz, nu=nu)
    assert ratio >= -1e-12
    s = np.real(np.fft.ifft2(sq))
    F = np.fft.fft2(s)
    acorr = np.real(np.fft.ifft2(F * np.conj(F)))       # all lags at once
    for b in range(pz):
        for a in range(px):
            dx, dz = min(a, px - a) * h, min(b, pz - b) * h
            r = np.hypot(dx / lx, dz / lz)
            x = 2 * np.sqrt(nu) * r
            c = 1.0 if r == 0 else 2 ** (1 - nu) / special.gamma(nu) * x ** nu * special.kv(nu, x)
            assert abs(acorr[b, a] - c) < 1e-12, (a, b)


def test_fields_anisotropic_empirical_covariance():
    """4096 Phi_2 fields on 32x32 (h = 1/32, lz = 0.01 < h): the lag-1
    correlation along x is exp(-sqrt2 h/0.1) and along z exp(-sqrt2 h/0.01),
    within 5 standard errors."""
    n, S = 32, 4096
    lnks, _ = O.sample_fields(n, n, S, seed=4, corr_len=0.1, corr_len_z=0.01, nu=0.5)
    h = 1.0 / n
    for axis, lam in ((2, 0.1), (1, 0.01)):
        for lag in (0, 1, 2):
            a = np.take(lnks, np.arange(0, n - lag), axis=axis)
            b = np.take(lnks, np.arange(lag, n), axis=axis)
            per = (a * b).mean(axis=(1, 2))
            se = per.std(ddof=1) / np.sqrt(S)
            assert abs(per.mean() - np.exp(-np.sqrt(2) * lag * h / lam)) < 5 * se + 1e-3, (axis, lag)


@pytest.mark.parametrize("kw", [{}, dict(nu=1.0, corr_len=0.2, corr_len_z=0.2),
                                dict(nu=0.5, corr_len=0.1, corr_len_z=0.01), dict(nu=2.5, corr_len=0.15, corr_len_z=0.3)])
@pytest.mark.parametrize("n", [16, 32])
def test_torus_is_the_smallest_admissible(kw, n):
    """The FFT-MA torus (Appendix A): a power of two of at least twice the grid
    per side whose circulant spectrum has no eigenvalue below -1e-12 max; when
    it is larger than 2n, the torus of half its size has such an eigenvalue."""
    px, pz = O.torus_size(n, n, **kw)
    assert px == pz and px >= 2 * n and px & (px - 1) == 0
    _, ratio = O.fftma_sqrt_spectrum(px, pz, 1.0 / n, **kw)
    assert ratio >= -1e-12
    if px > 2 * n:
        _, half = O.fftma_sqrt_spectrum(px // 2, pz // 2, 1.0 / n, **kw)
        assert half < -1e-12


def test_fields_coarsening_is_2x2_mean():
    """coarsen_times = 1 returns the 2x2 block means of the fine draw."""
    lk, al = O.sample_fields(16, 16, 3, seed=5)
    lc, ac = O.sample_fields(16, 16, 3, seed=5, coarsen_times=1)
    blk = lambda x: x.reshape(3, 8, 2, 8, 2).mean(axis=(2, 4))
    assert np.abs(lc - blk(lk)).max() < 1e-14
    assert np.abs(ac - blk(al)).max() < 1e-14


# ---------------------------------------------------------- linear limits
def layered_head(ks_rows, p_top, p_bot):
    """Exact steady head in a horizontally layered column with uniform K per
    layer: Darcy flux q = -K d(p + z)/dz is constant, and the hydraulic head
    p + z drops across each half cell by q times its resistance (h/2)/K."""
    nz = ks_rows.size
    h = 1.0 / nz
    half = (h / 2) / ks_rows
    r_centre = np.concatenate([[half[0]], half[0] + np.cumsum(half[:-1] + half[1:])])
    r_total = r_centre[-1] + half[-1]
    phi_bot, phi_top = p_bot + 0.0, p_top + 1.0
    q = -(phi_top - phi_bot) / r_total
    phi = phi_bot - q * r_centre
    z = (np.arange(nz) + 0.5) * h
    return phi - z


@pytest.mark.parametrize("n", [8, 16, 32])
def test_saturated_limit_layered_closed_form(n):
    """alpha = 0 (K = Ks, C = 0): steady layered flow has a closed form that the
    harmonic face means, the half-cell Dirichlet faces and the gravity term
    reproduce exactly."""
    z = (np.arange(n) + 0.5) / n
    ks_rows = np.exp(0.8 * np.sin(2 * np.pi * z) + 0.5 * np.cos(5 * z) + 0.3 * z)
    lnks = np.repeat(np.log(ks_rows)[:, None], n, axis=1)
    alpha = np.zeros((n, n))
    pb = problem(nsteps=2)
    p, q, rc, st = O.solve_one(pb, lnks, alpha)
    assert rc == 0
    exact = layered_head(ks_rows, PHYSICS["p_top"], PHYSICS["p_bottom"])
    assert np.abs(p - exact[:, None]).max() < 1e-9
    # bottom-flux QoI equals the exact downward Darcy flux
    phi_drop = (PHYSICS["p_top"] + 1.0) - PHYSICS["p_bottom"]
    r_total = np.sum(1.0 / n / ks_rows)
    assert abs(q - phi_drop / r_total) < 1e-9 * max(1.0, abs(q))


def test_saturated_limit_columns_closed_form():
    """Ks varying only across x: every column carries its own vertical flux
    and the head is the same linear profile in each column (no lateral flow)."""
    n = 16
    rng = np.random.default_rng(3)
    lnks = np.repeat(rng.normal(size=n)[None, :], n, axis=0)
    p, q, rc, _ = O.solve_one(problem(), lnks, np.zeros((n, n)))
    z = (np.arange(n) + 0.5) / n
    exact = PHYSICS["p_bottom"] + (PHYSICS["p_top"] - PHYSICS["p_bottom"]) * z
    assert rc == 0 and np.abs(p - exact[:, None]).max() < 1e-9


def hydraulic_head_dense_solve(lnks, p_top=PHYSICS["p_top"], p_bot=PHYSICS["p_bottom"]):
    """Steady saturated flow solved for the hydraulic head phi = p + z with a
    dense direct solve of G^T diag(c) G phi = b phi_D, where G is the
    face-cell incidence matrix, c the face conductances (inverse of the sum of
    the two half-cell resistances) and b the Dirichlet half-cell conductances.
    Gravity never appears: it is absorbed into phi."""
    nz, nx = lnks.shape
    h = 1.0 / nz
    K = np.exp(lnks)
    rhalf = h * h / (2.0 * K)          # half-cell resistance per unit area
    idx = lambda i, j: j * nx + i
    rows, cond = [], []
    for j in range(nz):
        for i in range(nx):
            if i + 1 < nx:
                rows.append((idx(i, j), idx(i + 1, j)))
                cond.append(1.0 / (rhalf[j, i] + rhalf[j, i + 1]))
            if j + 1 < nz:
                rows.append((idx(i, j), idx(i, j + 1)))
                cond.append(1.0 / (rhalf[j, i] + rhalf[j + 1, i]))
    n = nx * nz
    G = np.zeros((len(rows), n))
    for k, (a, b) in enumerate(rows):
        G[k, a], G[k, b] = 1.0, -1.0
    A = G.T @ np.diag(cond) @ G
    rhs = np.zeros(n)
    for i in range(nx):
        bt, bb = 1.0 / rhalf[nz - 1, i], 1.0 / rhalf[0, i]
        A[idx(i, nz - 1), idx(i, nz - 1)] += bt
        A[idx(i, 0), idx(i, 0)] += bb
        rhs[idx(i, nz - 1)] += bt * (p_top + 1.0)
        rhs[idx(i, 0)] += bb * (p_bot + 0.0)
    phi = np.linalg.solve(A, rhs).reshape(nz, nx)
    z = (np.arange(nz) + 0.5) * h
    return phi - z[:, None]


@pytest.mark.parametrize("shape", [(8, 8), (8, 12), (16, 16)])
def test_saturated_limit_dense_direct_solve(shape):
    """8x8 (and two other shapes): heterogeneous saturated limit equals a dense
    direct solve of the hydraulic-head system built from an incidence matrix."""
    nz, nx = shape
    rng = np.random.default_rng(7)
    lnks = rng.normal(size=(nz, nx))
    p, q, rc, st = O.solve_one(problem(nsteps=1), lnks, np.zeros((nz, nx)))
    assert rc == 0
    assert np.abs(p - hydraulic_head_dense_solve(lnks)).max() < 1e-9
    # linear problem: the first Picard update is the solution, the second only
    # confirms it (||dp|| below the Picard tolerance)
    assert st.picard_iters == 2, st.picard_iters


# ------------------------------------------------------------ multigrid
@pytest.mark.parametrize("n", [8, 32, 64])
def test_mg_poisson_matches_dense_and_contracts(n):
    """Poisson special case (Ks = 1, alpha = 0, C = 0): CCMG converges to the
    dense solution; the residual decreases monotonically."""
    rng = np.random.default_rng(11)
    lnks = np.zeros((n, n))
    pb = problem()
    Tx, Tz, Tbt, Tbb, Cdt, f0 = O.picard_system(pb, lnks, np.zeros((n, n)), np.full((n, n), -1.0),
                                                np.full((n, n), -1.0))
    f = rng.normal(size=(n, n))
    dp, cyc, rc, hist = O.mg_solve(Tx, Tz, Tbt, Tbb, Cdt, f, tol=1e-13, maxit=200)
    assert rc == 0
    assert np.all(np.diff(hist) < 0)
    rho = (hist[-1] / hist[0]) ** (1.0 / cyc)
    assert rho < 0.2, rho              # V(2,2) with RB-GS: ~0.06-0.1 per cycle on these grids
    ref = np.linalg.solve(poisson_dense(n), f.reshape(-1)).reshape(n, n)
    assert np.abs(dp - ref).max() < 1e-10 * np.abs(ref).max()


def poisson_dense(n):
    """Dense 5-point operator of the unit-conductivity grid: neighbours at
    1/h^2, Dirichlet faces (top, bottom) at 2/h^2 through the half cell, no
    flow through the sides."""
    h = 1.0 / n
    A = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            P = j * n + i
            for (a, b, t) in ((i + 1, j, 1 / h ** 2), (i - 1, j, 1 / h ** 2),
                              (i, j + 1, 1 / h ** 2), (i, j - 1, 1 / h ** 2)):
                if 0 <= a < n and 0 <= b < n:
                    A[P, P] += t
                    A[P, b * n + a] -= t
                elif 0 <= a < n:      # beyond top/bottom: Dirichlet at h/2
                    A[P, P] += 2 / h ** 2
    return A


@pytest.mark.parametrize("n", [4, 16, 32, 64])
def test_w_cycle_converges_to_dense_and_beats_v(n):
    """Cycle index gamma = 2 (the W-cycle of Sec. 4.2): converges to the dense
    solution; with two levels (4^2 -> 2^2, the coarsest grid) it is the
    V-cycle exactly; with three or more levels it visits the coarse grids
    more often and contracts strictly faster than the V-cycle (and needs more
    coarse-grid work, so it is not the V-cycle under another name)."""
    rng = np.random.default_rng(5)
    z = np.zeros((n, n))
    Tx, Tz, Tbt, Tbb, Cdt, f0 = O.picard_system(problem(), z, z, np.full((n, n), -1.0),
                                                np.full((n, n), -1.0))
    f = rng.normal(size=(n, n))
    runs = {g: O.mg_solve(Tx, Tz, Tbt, Tbb, Cdt, f, tol=1e-13, maxit=200, gamma=g) for g in (1, 2, 3)}
    ref = np.linalg.solve(poisson_dense(n), f.reshape(-1)).reshape(n, n)
    rho = {}
    for g, (dp, cyc, rc, hist) in runs.items():
        assert rc == 0
        assert np.abs(dp - ref).max() < 1e-10 * np.abs(ref).max()
        rho[g] = (hist[min(4, cyc)] / hist[0]) ** (1.0 / min(4, cyc))
    if n == 4:
        assert np.array_equal(runs[1][0], runs[2][0]) and runs[1][1] == runs[2][1]
    else:
        assert rho[2] < 0.9 * rho[1], rho
        assert rho[3] <= rho[2] * 1.05, rho


# ------------------------------------------------------------ nonlinear pins
def _mms(M):
    import sympy as sp
    x, z = sp.symbols("x z")
    p_bot, p_top, A = PHYSICS["p_bottom"], PHYSICS["p_top"], 0.5
    pstar = p_bot + (p_top - p_bot) * z + A * sp.sin(sp.pi * z) * sp.cos(sp.pi * x)
    lnks = 0.4 * sp.cos(sp.pi * x) * sp.sin(sp.pi * z) + 0.2 * z
    al = 1.0 + 0.3 * sp.sin(sp.pi * x) * sp.cos(sp.pi * z)
    K = sp.exp(lnks) * sp.exp(al * pstar)
    qx = -K * sp.diff(pstar, x)
    qz = -K * (sp.diff(pstar, z) + 1)
    src = sp.diff(qx, x) + sp.diff(qz, z)       # steady: div q = f
    fn = {k: sp.lambdify((x, z), e, "numpy") for k, e in
          dict(p=pstar, lnks=lnks, al=al, src=src).items()}
    c = (np.arange(M) + 0.5) / M
    X, Z = np.meshgrid(c, c)
    return {k: np.broadcast_to(f(X, Z), X.shape).astype(np.float64) for k, f in fn.items()}


@pytest.mark.slow
def test_mms_second_order():
    """Manufactured steady solution p* with smooth Ks, alpha and the source
    f = -div(K(p*)(grad p* + e_z)): the discrete error is O(h^2)."""
    errs = []
    Ms = [16, 32, 64, 128]
    for M in Ms:
        d = _mms(M)
        pb = problem(nsteps=1, dt=1e10, picard_maxit=200)
        p, q, rc, st = O.solve_one(pb, d["lnks"], d["al"], src=d["src"], p_init=d["p"])
        assert rc == 0
        errs.append(np.abs(p - d["p"]).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.85), (errs, orders)


def test_mass_balance_per_step():
    """Mixed form conserves mass (Sec. 4.1): over one step the change of stored
    water equals dt times the net boundary inflow at t^{n+1}, up to the Picard
    residual; interior fluxes cancel in pairs."""
    n = 32
    lnks, alpha = O.sample_fields(n, n, 1, seed=3)
    lnks, alpha = lnks[0], alpha[0]
    pb = problem(nsteps=1, dt=0.01)
    h = 1.0 / n
    tr, ts = PHYSICS["theta_r"], PHYSICS["theta_s"]

    def water(p):
        E = np.where(p < 0, np.exp(alpha * np.minimum(p, 0)), 1.0)
        return h * h * np.sum(tr + (ts - tr) * E)

    def outflow(p):
        Ks = np.exp(lnks)
        kt = Ks[-1] * np.exp(alpha[-1] * min(PHYSICS["p_top"], 0))
        kb = Ks[0] * np.exp(alpha[0] * min(PHYSICS["p_bottom"], 0))
        q_top = -kt * ((PHYSICS["p_top"] - p[-1]) / (h / 2) + 1)      # outward +z
        q_bot = kb * ((p[0] - PHYSICS["p_bottom"]) / (h / 2) + 1)      # outward -z
        return h * (q_top.sum() + q_bot.sum())

    p = np.full((n, n), PHYSICS["p_init"])
    for step in range(4):
        p1, q, rc, st = O.solve_one(pb, lnks, alpha, p_init=p)
        if rc != 0:
            pytest.skip("sample did not converge")
        dW = water(p1) - water(p)
        flux = pb.dt * outflow(p1)
        scale = pb.dt * h * np.abs(np.exp(lnks[-1])).sum()
        assert abs(dW + flux) < 1e-6 * scale, (step, dW, flux)
        p = p1


def test_failure_statuses():
    n = 16
    lnks, alpha = O.sample_fields(n, n, 1, seed=0)
    p, q, rc, _ = O.solve_one(problem(picard_maxit=1), lnks[0], alpha[0])
    assert rc == O.PICARD_MAXIT and np.isnan(q)
    bad = lnks[0].copy()
    bad[3, 4] = np.nan
    p, q, rc, _ = O.solve_one(problem(), bad, alpha[0])
    assert rc == O.NONFINITE
    with pytest.raises(ValueError):
        O.solve_one(problem(), np.zeros((9, 9)), np.zeros((9, 9)))


# ------------------------------------------------------------------- MLMC
def test_optimal_sample_allocation_is_the_constrained_minimum():
    """Eq. MLMCSAMP_ch6 is the Lagrange minimiser of sum N_l W_l subject to
    sum V_l / N_l = eps^2 (Eq. MLMCopt_ch6): it meets the constraint, its cost
    is eps^-2 (sum sqrt(V W))^2, and random feasible reallocations cost more."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        L = rng.integers(2, 6)
        V = rng.uniform(1e-4, 1.0, L)
        W = rng.uniform(1e-3, 10.0, L)
        eps = 10 ** rng.uniform(-3, -1)
        levels = [O.LevelStats(10, 0.0, v, w) for v, w in zip(V, W)]
        n_opt, cost = O.optimal_samples(levels, eps)
        n_opt = np.array(n_opt)
        assert abs(np.sum(V / n_opt) - eps ** 2) < 1e-12 * eps ** 2
        assert abs(np.sum(n_opt * W) - cost) < 1e-9 * cost
        for _ in range(50):
            n_try = n_opt * np.exp(rng.normal(scale=0.3, size=L))
            n_try *= np.sum(V / n_try) / eps ** 2        # rescale onto the constraint
            assert np.sum(n_try * W) >= cost * (1 - 1e-12)


def test_mlmc_combine_telescopes():
    rng = np.random.default_rng(2)
    ys = [rng.normal(loc=m, scale=s, size=n) for m, s, n in ((1.0, 1.0, 400), (0.1, 0.2, 100))]
    levels = [O.level_stats(y, 1.0) for y in ys]
    est, rmse = O.mlmc_combine(levels)
    assert abs(est - (ys[0].mean() + ys[1].mean())) < 1e-14
    assert abs(rmse ** 2 - (ys[0].var(ddof=1) / 400 + ys[1].var(ddof=1) / 100)) < 1e-14


def test_oracle_mlmc_telescoping():
    """Coupled MLMC (Sec. 5, Eq. fine_coarse): with draws on the finest grid the
    level-0 fine member and the level-1 coarse member estimate the same mean."""
    o = O.mlmc_estimate((160, 160), 8, 2, 0.04, coupling=0, **PHYSICS, **SOLVER)
    a, b = o[0]["qf"], o[1]["qc"]
    se = np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    assert abs(a.mean() - b.mean()) < 4 * se


def test_oracle_mlmc_estimate_matches_plain_mc():
    """The telescoping MLMC estimate (Eq. MLMCestimator_ch6, coupling 0) and a
    plain MC estimate at the finest level with independent samples agree
    within 3 standard errors."""
    ns = (400, 120, 40)
    o = O.mlmc_estimate(ns, 8, 2, 0.04, coupling=0, **PHYSICS, **SOLVER)
    est = sum(lev["y"].mean() for lev in o)
    var = sum(lev["y"].var(ddof=1) / lev["y"].size for lev in o)
    lk, al = O.sample_fields(32, 32, 400, seed=0, level=77)
    pb = O.make_problem(nsteps=8, dt=0.04 / 8, **PHYSICS, **SOLVER)
    _, q, st, _ = O.solve_batch(pb, lk, al, want_p=False)
    q = q[(st == 0) | (st == 2)]
    se = np.sqrt(var + q.var(ddof=1) / q.size)
    assert abs(est - q.mean()) < 3 * se, (est, q.mean(), se)


def test_covariance_upscaling_pair_is_exact_on_both_grids():
    """Appendix A, Eqs. averaging / cov_upscale: the coarse member is an exact
    exp(-r/0.3) field on the 8x8 grid (empirical covariance within 5 s.e.),
    strongly correlated with the 2x2 means of the fine member."""
    S, n, lam = 4096, 16, 0.3
    lkf, alf, lkc, alc = O.sample_fields_pair(n, n, S, seed=3)
    h = 2.0 / n
    for axis in (1, 2):
        for lag in range(0, 5):
            a = np.take(lkc, np.arange(0, n // 2 - lag), axis=axis)
            b = np.take(lkc, np.arange(lag, n // 2), axis=axis)
            ps = (a * b).mean(axis=(1, 2))
            assert abs(ps.mean() - np.exp(-lag * h / lam)) < 5 * ps.std(ddof=1) / np.sqrt(S) + 1e-3
    blk = lkf.reshape(S, n // 2, 2, n // 2, 2).mean(axis=(2, 4))
    assert np.corrcoef(blk.reshape(-1), lkc.reshape(-1))[0, 1] > 0.8
    assert alc.min() > 0.5 and alc.max() < 2.0
    # the fine member is the plain draw of the same (seed, level, sample)
    lk1, al1 = O.sample_fields(n, n, 3, seed=3)
    assert np.abs(lk1 - lkf[:3]).max() < 1e-13 and np.abs(al1 - alf[:3]).max() < 1e-13
