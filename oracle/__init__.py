"""Plain FP64 CPU oracle for the stochastic Richards' equation solve.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this package.  It shares no code with the CUDA library.

The numerical core is ``richards_oracle.c`` (plain loops, -O2
-ffp-contract=off); this module compiles it with gcc on first use and wraps
it with ctypes.  The MLMC statistics of Sec. 5 (Eqs. MLMCestimator_ch6,
MC_var_ch6, eq:MLMCVar, MLMCSAMP_ch6) are written here in numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "richards_oracle.c")
_HDR = os.path.join(_HERE, "richards_oracle.h")
_LIB = os.path.join(_HERE, "liboracle_richards.so")

OK, PICARD_MAXIT, MG_MAXIT, NONFINITE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no multiply-add contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    _fields_ = [("nsteps", C.c_int32), ("dt", C.c_double), ("theta_r", C.c_double),
                ("theta_s", C.c_double), ("p_top", C.c_double), ("p_bottom", C.c_double),
                ("p_init", C.c_double), ("picard_tol", C.c_double), ("picard_maxit", C.c_int32),
                ("mg_tol", C.c_double), ("mg_maxit", C.c_int32), ("nu1", C.c_int32),
                ("nu2", C.c_int32), ("gamma", C.c_int32), ("closure", C.c_int32),
                ("init_decay", C.c_double)]


GARDNER, VAN_GENUCHTEN = 0, 1


class Soil(C.Structure):
    """Per-cell soil parameters of a batch (see orc_soil)."""
    _fields_ = [("lnKs", C.c_void_p), ("alpha", C.c_void_p), ("n", C.c_void_p),
                ("theta_s", C.c_void_p), ("theta_r", C.c_void_p), ("alpha_scale", C.c_double),
                ("alpha_shift", C.c_double), ("n_shift", C.c_double)]


class SoilModel(C.Structure):
    """Marginals of the five soil fields (see orc_soil_model)."""
    _fields_ = [("lnks_mean", C.c_double), ("alpha_lo", C.c_double), ("alpha_span", C.c_double),
                ("n_lo", C.c_double), ("n_span", C.c_double), ("theta_s_lo", C.c_double),
                ("theta_s_span", C.c_double), ("theta_r_lo", C.c_double), ("theta_r_span", C.c_double)]


def soil_model(alpha_bl, n_bl, ks_bl=0.2, theta_s_bl=0.5, theta_r_bl=0.05, d_alpha=0.2, d_n=0.05,
               d_theta_s=0.05, d_theta_r=0.005):
    """Table soilparams: ln Ks = ln Ks_bl + Z; every other parameter baseline +
    U(-d, d) (lo = baseline - d, span = 2 d)."""
    import math
    return SoilModel(math.log(ks_bl), alpha_bl - d_alpha, 2 * d_alpha, n_bl - d_n, 2 * d_n,
                     theta_s_bl - d_theta_s, 2 * d_theta_s, theta_r_bl - d_theta_r, 2 * d_theta_r)


class Cov(C.Structure):
    """Covariance of the Gaussian fields (nu = 0: exponential; nu > 0: Matern)."""
    _fields_ = [("sigma2", C.c_double), ("corr_len", C.c_double), ("corr_len_z", C.c_double),
                ("nu", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("picard_iters", C.c_int64), ("mg_cycles", C.c_int64),
                ("max_picard", C.c_int32), ("max_mg", C.c_int32)]


def make_problem(nsteps=10, dt=0.01, theta_r=0.1, theta_s=0.5, p_top=-0.5, p_bottom=-5.0,
                 p_init=-5.0, picard_tol=1e-8, picard_maxit=50, mg_tol=1e-10, mg_maxit=100,
                 nu1=2, nu2=2, gamma=1, closure=0, init_decay=0.0) -> Problem:
    """Physics and solver settings of the configured instance (Gardner closure);
    gamma = 1: V-cycles (configured), 2: W-cycles (the paper's choice, Sec. 4.2)."""
    return Problem(nsteps, dt, theta_r, theta_s, p_top, p_bottom, p_init, picard_tol,
                   picard_maxit, mg_tol, mg_maxit, nu1, nu2, gamma, closure, init_decay)


def infiltration_problem(nsteps=10, dt=0.01, picard_tol=1e-5, mg_tol=1e-5, gamma=2, **kw) -> Problem:
    """The infiltration problem of Sec. 4.3 (Eq. travellingwave) with the van
    Genuchten-Mualem closure: p(x,z,0) = -0.4 (1 - exp(-80 z)), p = -0.4 on the
    top, 0.1 on the bottom, theta_s = 0.5, theta_r = 0.05 (per-cell fields
    override them), W(2,2) cycles and tolerances 1e-5 as in the paper."""
    d = dict(nsteps=nsteps, dt=dt, theta_r=0.05, theta_s=0.5, p_top=-0.4, p_bottom=0.1, p_init=-0.4,
             picard_tol=picard_tol, picard_maxit=50, mg_tol=mg_tol, mg_maxit=100, nu1=2, nu2=2,
             gamma=gamma, closure=VAN_GENUCHTEN, init_decay=80.0)
    d.update(kw)
    return make_problem(**d)


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_white_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, C.c_int64, _dp]
        L.orc_fft2.argtypes = [_dp, _dp, C.c_int32, C.c_int32, C.c_int32]
        L.orc_fft2.restype = C.c_int
        L.orc_bessel_k.argtypes = [C.c_double, C.c_double]
        L.orc_bessel_k.restype = C.c_double
        L.orc_covariance.argtypes = [C.POINTER(Cov), C.c_double, C.c_double]
        L.orc_covariance.restype = C.c_double
        L.orc_fftma_spectrum.argtypes = [C.c_int32, C.c_int32, C.c_double, C.POINTER(Cov),
                                         _dp, C.POINTER(C.c_double)]
        L.orc_torus_size.argtypes = [C.c_int32, C.c_int32, C.c_double, C.POINTER(Cov),
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.orc_sample_fields.argtypes = [C.c_uint64, C.POINTER(Cov), C.c_double, C.c_double,
                                        C.c_int32, C.c_int32, C.c_uint32, C.c_int64, C.c_int32,
                                        C.c_int32, _dp, _dp, C.c_int32]
        L.orc_sample_fields_pair.argtypes = [C.c_uint64, C.POINTER(Cov), C.c_double, C.c_double,
                                             C.c_int32, C.c_int32, C.c_uint32, C.c_int64, C.c_int32,
                                             _dp, _dp, _dp, _dp]
        L.orc_solve_batch_soil.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32, C.c_int32,
                                           C.POINTER(Soil), C.c_void_p, _dp, _i32p, C.POINTER(Stats),
                                           C.c_int32]
        L.orc_solve_one_soil.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32, C.POINTER(Soil),
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                         C.POINTER(Stats)]
        L.orc_sample_soil_pair.argtypes = [C.c_uint64, C.POINTER(Cov), C.POINTER(SoilModel), C.c_int32,
                                           C.c_int32, C.c_uint32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]
        L.orc_closure.argtypes = [C.c_int32] + [C.c_double] * 6 + [C.POINTER(C.c_double)] * 3
        L.orc_sample_soil.argtypes = [C.c_uint64, C.POINTER(Cov), C.POINTER(SoilModel), C.c_int32,
                                      C.c_int32, C.c_uint32, C.c_int64, C.c_int32, C.c_int32,
                                      _dp, _dp, _dp, _dp, _dp, C.c_int32]
        L.orc_solve_one.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32, _dp, _dp, C.c_double,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                    C.POINTER(Stats)]
        L.orc_solve_batch.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32, C.c_int32, _dp, _dp,
                                      C.c_double, C.c_void_p, _dp, _i32p, C.POINTER(Stats), C.c_int32]
        L.orc_picard_system.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32, _dp, _dp, C.c_double,
                                        _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_mg_solve.argtypes = [C.c_int32, C.c_int32, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp,
                                   C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _dp,
                                   C.POINTER(C.c_int32), C.c_void_p]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- random fields
def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def white_noise(seed, level, sample, field, npts):
    y = np.empty(npts, np.float64)
    lib().orc_white_noise(seed, level, sample, field, npts, y)
    return y


def fft2(x, inverse=False):
    """2-D DFT of a complex [nz, nx] array with the oracle's own radix-2 FFT."""
    x = np.asarray(x, np.complex128)
    re, im = _f64(x.real.copy()), _f64(x.imag.copy())
    nz, nx = x.shape
    rc = lib().orc_fft2(re, im, nx, nz, int(inverse))
    if rc:
        raise ValueError("sizes must be powers of two")
    return re + 1j * im


def bessel_k(nu, x):
    """K_nu(x), x > 0, by the oracle's trapezoidal rule on its integral representation."""
    return lib().orc_bessel_k(nu, x)


def covariance(dx, dz, sigma2=1.0, corr_len=0.3, corr_len_z=0.0, nu=0.0):
    """Field covariance at offset (dx, dz): exponential (nu = 0) or Matern (Eq. nonIsotropic)."""
    return lib().orc_covariance(C.byref(Cov(sigma2, corr_len, corr_len_z, nu)), dx, dz)


def torus_size(nx, nz, sigma2=1.0, corr_len=0.3, corr_len_z=0.0, nu=0.0):
    px, pz = C.c_int32(), C.c_int32()
    lib().orc_torus_size(nx, nz, 1.0 / nz, C.byref(Cov(sigma2, corr_len, corr_len_z, nu)),
                         C.byref(px), C.byref(pz))
    return px.value, pz.value


def fftma_sqrt_spectrum(px, pz, h, sigma2=1.0, corr_len=0.3, corr_len_z=0.0, nu=0.0):
    s = np.empty(px * pz, np.float64)
    ratio = C.c_double()
    lib().orc_fftma_spectrum(px, pz, h, C.byref(Cov(sigma2, corr_len, corr_len_z, nu)), s,
                             C.byref(ratio))
    return s.reshape(pz, px), ratio.value


def sample_fields(nx, nz, nsamples, seed=0, level=0, first_sample=0, coarsen_times=0,
                  sigma2=1.0, corr_len=0.3, alpha_lo=0.5, alpha_span=1.5, nthreads=None,
                  corr_len_z=0.0, nu=0.0):
    """ln Ks and alpha fields [S, nz>>c, nx>>c] drawn by FFT-MA on the nx x nz grid."""
    nthreads = nthreads or os.cpu_count() or 1
    nxo, nzo = nx >> coarsen_times, nz >> coarsen_times
    lnKs = np.empty((nsamples, nzo, nxo), np.float64)
    alpha = np.empty((nsamples, nzo, nxo), np.float64)
    cv = Cov(sigma2, corr_len, corr_len_z, nu)
    rc = lib().orc_sample_fields(seed, C.byref(cv), alpha_lo, alpha_span, nx, nz, level,
                                 first_sample, nsamples, coarsen_times, lnKs.reshape(-1),
                                 alpha.reshape(-1), nthreads)
    if rc:
        raise ValueError("invalid field arguments")
    return lnKs, alpha


def sample_fields_pair(nx, nz, nsamples, seed=0, level=0, first_sample=0, sigma2=1.0, corr_len=0.3,
                       alpha_lo=0.5, alpha_span=1.5, corr_len_z=0.0, nu=0.0):
    """Fine [S, nz, nx] and coarse [S, nz/2, nx/2] fields by covariance upscaling."""
    f = [np.empty((nsamples, nz, nx)) for _ in range(2)]
    c = [np.empty((nsamples, nz // 2, nx // 2)) for _ in range(2)]
    cv = Cov(sigma2, corr_len, corr_len_z, nu)
    rc = lib().orc_sample_fields_pair(seed, C.byref(cv), alpha_lo, alpha_span, nx, nz, level,
                                      first_sample, nsamples, f[0].reshape(-1), f[1].reshape(-1),
                                      c[0].reshape(-1), c[1].reshape(-1))
    if rc:
        raise ValueError("invalid field arguments")
    return f[0], f[1], c[0], c[1]


# ---------------------------------------------------------------------- solver
def solve_one(pb, lnKs, alpha, alpha_scale=1.0, src=None, p_init=None):
    lnKs, alpha = _f64(lnKs), _f64(alpha)
    nz, nx = lnKs.shape
    src = None if src is None else _f64(src)
    p_init = None if p_init is None else _f64(p_init)
    p = np.empty((nz, nx), np.float64)
    q = C.c_double()
    st = Stats()
    rc = lib().orc_solve_one(C.byref(pb), nx, nz, lnKs.reshape(-1), alpha.reshape(-1), alpha_scale,
                             _ptr(src), _ptr(p_init), _ptr(p), C.byref(q), C.byref(st))
    if rc < 0:
        raise ValueError("invalid grid")
    return p, q.value, rc, st


def solve_batch(pb, lnKs, alpha, alpha_scale=1.0, want_p=True, nthreads=None):
    """Solve every sample of lnKs/alpha [S, nz, nx]; returns (p, qoi, status, stats)."""
    nthreads = nthreads or os.cpu_count() or 1
    lnKs, alpha = _f64(lnKs), _f64(alpha)
    S, nz, nx = lnKs.shape
    p = np.empty((S, nz, nx), np.float64) if want_p else None
    qoi = np.empty(S, np.float64)
    status = np.zeros(S, np.int32)
    st = Stats()
    rc = lib().orc_solve_batch(C.byref(pb), nx, nz, S, lnKs.reshape(-1), alpha.reshape(-1),
                               alpha_scale, _ptr(p), qoi, status, C.byref(st), nthreads)
    if rc < 0:
        raise ValueError("invalid grid")
    return p, qoi, status, st


def solve_batch_soil(pb, lnKs, alpha, n=None, theta_s=None, theta_r=None, alpha_scale=1.0,
                     alpha_shift=0.0, n_shift=0.0, want_p=True, nthreads=None):
    """Solve every sample with per-cell soil fields [S, nz, nx] (van
    Genuchten-Mualem needs n; theta fields optional); returns (p, qoi, status, stats)."""
    nthreads = nthreads or os.cpu_count() or 1
    arrs = [None if a is None else _f64(a) for a in (lnKs, alpha, n, theta_s, theta_r)]
    S, nz, nx = arrs[0].shape
    so = Soil(*[_ptr(a) for a in arrs], alpha_scale, alpha_shift, n_shift)
    p = np.empty((S, nz, nx), np.float64) if want_p else None
    qoi = np.empty(S, np.float64)
    status = np.zeros(S, np.int32)
    st = Stats()
    rc = lib().orc_solve_batch_soil(C.byref(pb), nx, nz, S, C.byref(so), _ptr(p), qoi, status,
                                    C.byref(st), nthreads)
    if rc < 0:
        raise ValueError("invalid grid or soil arrays")
    return p, qoi, status, st


def solve_one_soil(pb, lnKs, alpha, n=None, theta_s=None, theta_r=None, src=None, p_init=None,
                   alpha_scale=1.0, alpha_shift=0.0, n_shift=0.0):
    """One sample with per-cell soil fields [nz, nx], an optional source and
    initial head; returns (p, qoi, status, stats)."""
    arrs = [None if a is None else _f64(a) for a in (lnKs, alpha, n, theta_s, theta_r)]
    nz, nx = arrs[0].shape
    so = Soil(*[_ptr(a) for a in arrs], alpha_scale, alpha_shift, n_shift)
    src = None if src is None else _f64(src)
    p_init = None if p_init is None else _f64(p_init)
    p = np.empty((nz, nx))
    q = C.c_double()
    st = Stats()
    rc = lib().orc_solve_one_soil(C.byref(pb), nx, nz, C.byref(so), _ptr(src), _ptr(p_init), _ptr(p),
                                  C.byref(q), C.byref(st))
    if rc < 0:
        raise ValueError("invalid grid or soil arrays")
    return p, q.value, rc, st


def closure(kind, Ks, a, n, theta_r, theta_s, p):
    """(K, theta, C) of one cell at head p (kind 0 Gardner, 1 van Genuchten-Mualem)."""
    K, th, Cc = C.c_double(), C.c_double(), C.c_double()
    if lib().orc_closure(kind, Ks, a, n, theta_r, theta_s, p, C.byref(K), C.byref(th), C.byref(Cc)):
        raise ValueError("unknown closure")
    return K.value, th.value, Cc.value


def sample_soil(nx, nz, nsamples, model, seed=0, level=0, first_sample=0, coarsen_times=0, sigma2=1.0,
                corr_len=0.3, corr_len_z=0.0, nu=0.0, nthreads=None):
    """The five soil fields (ln Ks, alpha, n, theta_s, theta_r), each [S, nz>>c, nx>>c]."""
    nthreads = nthreads or os.cpu_count() or 1
    nxo, nzo = nx >> coarsen_times, nz >> coarsen_times
    out = [np.empty((nsamples, nzo, nxo)) for _ in range(5)]
    cv = Cov(sigma2, corr_len, corr_len_z, nu)
    rc = lib().orc_sample_soil(seed, C.byref(cv), C.byref(model), nx, nz, level, first_sample, nsamples,
                               coarsen_times, *[o.reshape(-1) for o in out], nthreads)
    if rc:
        raise ValueError("invalid field arguments")
    return tuple(out)


def sample_soil_pair(nx, nz, nsamples, model, seed=0, level=0, first_sample=0, sigma2=1.0, corr_len=0.3,
                     corr_len_z=0.0, nu=0.0):
    """The five soil fields as covariance-upscaled couples: (fine [5 arrays of
    S, nz, nx], coarse [5 arrays of S, nz/2, nx/2])."""
    fine = [np.empty((nsamples, nz, nx)) for _ in range(5)]
    coarse = [np.empty((nsamples, nz // 2, nx // 2)) for _ in range(5)]
    pf = (C.c_void_p * 5)(*[a.ctypes.data for a in fine])
    pc = (C.c_void_p * 5)(*[a.ctypes.data for a in coarse])
    cv = Cov(sigma2, corr_len, corr_len_z, nu)
    rc = lib().orc_sample_soil_pair(seed, C.byref(cv), C.byref(model), nx, nz, level, first_sample, nsamples,
                                    pf, pc)
    if rc:
        raise ValueError("invalid field arguments")
    return tuple(fine), tuple(coarse)


def picard_system(pb, lnKs, alpha, p, p_old, alpha_scale=1.0):
    """The Picard system at iterate p: (Tx, Tz, Tbt, Tbb, Cdt, f)."""
    lnKs, alpha, p, p_old = _f64(lnKs), _f64(alpha), _f64(p), _f64(p_old)
    nz, nx = lnKs.shape
    Tx, Tz, Cdt, f = (np.empty((nz, nx)) for _ in range(4))
    Tbt, Tbb = np.empty(nx), np.empty(nx)
    lib().orc_picard_system(C.byref(pb), nx, nz, lnKs.reshape(-1), alpha.reshape(-1), alpha_scale,
                            p.reshape(-1), p_old.reshape(-1), Tx.reshape(-1), Tz.reshape(-1),
                            Tbt, Tbb, Cdt.reshape(-1), f.reshape(-1))
    return Tx, Tz, Tbt, Tbb, Cdt, f


def mg_solve(Tx, Tz, Tbt, Tbb, Cdt, f, tol=1e-10, maxit=100, nu1=2, nu2=2, gamma=1):
    """CCMG V(nu1,nu2) solve from dp = 0; returns (dp, cycles, rc, residual history)."""
    Tx, Tz, Cdt, f = _f64(Tx), _f64(Tz), _f64(Cdt), _f64(f)
    nz, nx = f.shape
    dp = np.empty((nz, nx))
    cyc = C.c_int32()
    hist = np.zeros(maxit + 1)
    rc = lib().orc_mg_solve(nx, nz, 1.0 / nz, Tx.reshape(-1), Tz.reshape(-1), _f64(Tbt), _f64(Tbb),
                            Cdt.reshape(-1), f.reshape(-1), tol, maxit, nu1, nu2, gamma, dp.reshape(-1),
                            C.byref(cyc), _ptr(hist))
    return dp, cyc.value, rc, hist[: cyc.value + 1]


# ------------------------------------------------------------------------ MLMC
@dataclass
class LevelStats:
    n: int            # N_l samples
    mean: float       # E^MC_{N_l}[P_l - P_{l-1}]   (Eq. SMC_ch6)
    var: float        # V_l, unbiased 1/(N_l - 1)   (Eqs. MC_var_ch6, level_var_ch6)
    cost: float       # W_l, cost of one sample of the pair (seconds)


def level_stats(y, cost_per_sample):
    y = np.asarray(y, np.float64)
    n = y.size
    return LevelStats(n, float(y.mean()), float(y.var(ddof=1)) if n > 1 else float("nan"),
                      float(cost_per_sample))


def mlmc_combine(levels):
    """Telescoping estimate (Eq. MLMCestimator_ch6), sampling RMSE (Eq. eq:MLMCVar),
    optimal N_l (Eq. MLMCSAMP_ch6) and the cost W(eps) of the optimal allocation."""
    est = sum(L.mean for L in levels)
    rmse = float(np.sqrt(sum(L.var / L.n for L in levels)))
    return est, rmse


def optimal_samples(levels, eps):
    s = sum(np.sqrt(L.var * L.cost) for L in levels)
    n_opt = [eps ** -2 * s * np.sqrt(L.var / L.cost) for L in levels]
    w = eps ** -2 * s * s
    return n_opt, w


def mlmc_estimate(nsamples, n0, steps0, t_final, seed=0, coupling=0, continuation=1, key_offset=0,
                  sigma2=1.0, corr_len=0.3, alpha_lo=0.5, alpha_span=1.5, nthreads=None,
                  corr_len_z=0.0, nu=0.0, soil=None, d_alpha=0.05, d_n=0.1, fixed_levels=1,
                  with_thetas=True, **phys):
    """Parametric-continuation MLMC (Sec. 5) restated plainly: for level l draw
    N_l field pairs (coupling 0: on the finest grid, averaged down L-l times;
    coupling 1: on the level grid), solve the fine member on grid n0 2^l with
    steps0 2^l steps and alpha_l, the coarse member on the 2x2-averaged fields
    with the level-(l-1) grid, steps and alpha_{l-1}; Y_l = Q_l - Q_{l-1}.
    Returns per-level Y, Qf, Qc, statuses and the level statistics."""
    NL = len(nsamples)
    L = NL - 1
    nL = n0 << L
    vg = phys.get("closure", 0) == VAN_GENUCHTEN
    out = []

    def vg_steps(k):        # Sec. 5.2: the fixed_levels finest levels keep alpha and n
        return max(0, L + 1 - max(1, fixed_levels) - k) if continuation else 0

    def solve(pb, flds, k):
        if vg:
            kk = vg_steps(k)
            return solve_batch_soil(pb, *flds, alpha_shift=-kk * d_alpha, n_shift=kk * d_n, want_p=False,
                                    nthreads=nthreads)
        return solve_batch(pb, flds[0], flds[1], (k + 1) / NL if continuation else 1.0, want_p=False,
                           nthreads=nthreads)

    for l in range(NL):
        M = n0 << l
        fm = dict(seed=seed, level=l + key_offset, sigma2=sigma2, corr_len=corr_len, corr_len_z=corr_len_z, nu=nu)
        nf = 5 if with_thetas else 3
        if vg and coupling == 2 and l > 0:
            fine, crs = sample_soil_pair(M, M, nsamples[l], soil, **fm)
            fine, crs = fine[:nf], crs[:nf]
        elif vg:
            ndraw, ct = (nL, L - l) if coupling == 0 else (M, 0)
            fine = sample_soil(ndraw, ndraw, nsamples[l], soil, coarsen_times=ct, nthreads=nthreads, **fm)[:nf]
        elif coupling == 2 and l > 0:
            lk, al, lkc_up, alc_up = sample_fields_pair(M, M, nsamples[l], alpha_lo=alpha_lo,
                                                        alpha_span=alpha_span, **fm)
            fine, crs = (lk, al), (lkc_up, alc_up)
        elif coupling == 0:
            fine = sample_fields(nL, nL, nsamples[l], coarsen_times=L - l, nthreads=nthreads, alpha_lo=alpha_lo,
                                 alpha_span=alpha_span, **fm)
        else:
            fine = sample_fields(M, M, nsamples[l], nthreads=nthreads, alpha_lo=alpha_lo, alpha_span=alpha_span,
                                 **fm)
        pf = make_problem(nsteps=steps0 << l, dt=t_final / (steps0 << l), **phys)
        _, qf, sf, _ = solve(pf, fine, l)
        if l > 0:
            if coupling != 2:
                blk = lambda x: x.reshape(x.shape[0], M // 2, 2, M // 2, 2).mean(axis=(2, 4))
                crs = tuple(blk(x) for x in fine)
            pc = make_problem(nsteps=steps0 << (l - 1), dt=t_final / (steps0 << (l - 1)), **phys)
            _, qc, sc, _ = solve(pc, crs, l - 1)
        else:
            qc, sc = np.zeros_like(qf), np.zeros_like(sf)
        bad = np.isin(sf, (PICARD_MAXIT, NONFINITE)) | np.isin(sc, (PICARD_MAXIT, NONFINITE)) \
            | ~np.isfinite(qf) | ~np.isfinite(qc)
        y = (qf - qc)[~bad]
        out.append(dict(y=y, qf=qf[~bad], qc=qc[~bad], failed=int(bad.sum()), status_f=sf, status_c=sc))
    return out
