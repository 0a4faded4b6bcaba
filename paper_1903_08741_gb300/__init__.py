"""Python binding of librichards: batched stochastic Richards' solves on one GB300.

Thin ctypes marshalling over the C ABI declared in ``include/richards.h``:
torch tensors provide device memory and the current CUDA stream; every step of
the computation runs in the library's CUDA kernels.  There is no CPU fallback:
importing the binding without a built ``librichards.so`` raises, and so does
calling it without a CUDA device.

Entry points (same names as the C ABI): ``sample_fields``, ``sample_soil``,
``solve_batch``, ``solve_soil``, ``solve_batch_host``, ``mlmc_estimate`` and
the others listed by ``exported_symbols``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field, fields as dc_fields

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librichards.so")

OK, PICARD_MAXIT, MG_MAXIT, NONFINITE, ADJ_MAXIT = 0, 1, 2, 3, 4
FP64, MIXED = 0, 1
GARDNER, VAN_GENUCHTEN = 0, 1


class RichError(RuntimeError):
    pass


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32), ("nsteps", C.c_int32), ("dt", C.c_double),
                ("theta_r", C.c_double), ("theta_s", C.c_double), ("p_top", C.c_double),
                ("p_bottom", C.c_double), ("p_init", C.c_double), ("picard_tol", C.c_double),
                ("picard_maxit", C.c_int32), ("mg_tol", C.c_double), ("mg_maxit", C.c_int32),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("precision", C.c_int32), ("cycle", C.c_int32),
                ("closure", C.c_int32), ("init_decay", C.c_double)]


class _Soil(C.Structure):
    _fields_ = [("lnKs", C.c_void_p), ("alpha", C.c_void_p), ("n", C.c_void_p), ("theta_s", C.c_void_p),
                ("theta_r", C.c_void_p)]


class _SoilModel(C.Structure):
    _fields_ = [("lnks_mean", C.c_double), ("n_lo", C.c_double), ("n_span", C.c_double),
                ("theta_s_lo", C.c_double), ("theta_s_span", C.c_double), ("theta_r_lo", C.c_double),
                ("theta_r_span", C.c_double)]


class _Field(C.Structure):
    _fields_ = [("sigma2", C.c_double), ("corr_len", C.c_double), ("alpha_lo", C.c_double),
                ("alpha_span", C.c_double), ("seed", C.c_uint64), ("nu", C.c_double),
                ("corr_len_z", C.c_double)]


class _Fp64Rates(C.Structure):
    _fields_ = [("dfma_flops", C.c_double), ("div_per_s", C.c_double), ("exp_per_s", C.c_double),
                ("ms_total", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("picard_iters", C.c_int64), ("mg_cycles", C.c_int64), ("cell_vcycles", C.c_int64),
                ("max_picard", C.c_int32), ("failed", C.c_int32), ("seconds", C.c_double),
                ("sm_seconds", C.c_double)]


@dataclass
class Problem:
    """Physics and solver settings (Gardner closure; Picard Sec. 4.1; CCMG Sec. 4.2)."""
    nx: int = 32
    nz: int = 32
    nsteps: int = 10
    dt: float = 0.01
    theta_r: float = 0.1
    theta_s: float = 0.5
    p_top: float = -0.5
    p_bottom: float = -5.0
    p_init: float = -5.0
    picard_tol: float = 1e-8
    picard_maxit: int = 50
    mg_tol: float = 1e-10
    mg_maxit: int = 100
    nu1: int = 2
    nu2: int = 2
    precision: int = FP64
    cycle: int = 1           # 1: V-cycle (configured), 2: W-cycle (the paper's)
    closure: int = GARDNER   # or VAN_GENUCHTEN (Sec. 2.1; solve_soil with per-cell n)
    init_decay: float = 0.0  # > 0: p(x,z,0) = p_init (1 - exp(-init_decay z))

    def _c(self):
        return _Problem(*[getattr(self, f.name) for f in dc_fields(self)])

    @classmethod
    def infiltration(cls, **kw):
        """The infiltration problem of Sec. 4.3 (Eq. travellingwave) with the van
        Genuchten-Mualem closure: initial head -0.4 (1 - exp(-80 z)), top -0.4,
        bottom 0.1, theta_s 0.5, theta_r 0.05 (per-cell fields override them),
        W(2,2) cycles and Picard / MG tolerances 1e-5."""
        d = dict(theta_r=0.05, theta_s=0.5, p_top=-0.4, p_bottom=0.1, p_init=-0.4, picard_tol=1e-5,
                 mg_tol=1e-5, cycle=2, closure=VAN_GENUCHTEN, init_decay=80.0)
        d.update(kw)
        return cls(**d)


@dataclass
class SoilModel:
    """Marginals of the soil fields (Table soilparams): ln Ks = ln ks_bl + Z and
    baseline +- half-width uniform fields for n, theta_s, theta_r (alpha's range
    is the FieldModel's alpha_lo / alpha_span; see soil_field_model)."""
    ks_bl: float = 0.2
    n_bl: float = 1.45
    theta_s_bl: float = 0.5
    theta_r_bl: float = 0.05
    d_n: float = 0.05
    d_theta_s: float = 0.05
    d_theta_r: float = 0.005

    def _c(self):
        import math
        return _SoilModel(math.log(self.ks_bl), self.n_bl - self.d_n, 2 * self.d_n,
                          self.theta_s_bl - self.d_theta_s, 2 * self.d_theta_s,
                          self.theta_r_bl - self.d_theta_r, 2 * self.d_theta_r)


@dataclass
class FieldModel:
    """ln Ks ~ GRF(0, C); alpha = alpha_lo + alpha_span Phi(g).  C is the
    exponential sigma2 exp(-r/corr_len) for nu = 0, else the anisotropic Matern
    function (Eq. nonIsotropic) with lengths corr_len (x), corr_len_z (z; 0 =
    corr_len).  FieldModel.phi1() / phi2() give the paper's two parameter sets."""
    sigma2: float = 1.0
    corr_len: float = 0.3
    alpha_lo: float = 0.5
    alpha_span: float = 1.5
    seed: int = 0
    nu: float = 0.0
    corr_len_z: float = 0.0

    @classmethod
    def phi1(cls, **kw):
        """Isotropic Matern, (nu, lx, lz, sigma2) = (1, 0.2, 0.2, 1)."""
        return cls(**{**dict(sigma2=1.0, corr_len=0.2, corr_len_z=0.2, nu=1.0), **kw})

    @classmethod
    def phi2(cls, **kw):
        """Anisotropic Matern, (nu, lx, lz, sigma2) = (0.5, 0.1, 0.01, 1)."""
        return cls(**{**dict(sigma2=1.0, corr_len=0.1, corr_len_z=0.01, nu=0.5), **kw})

    def _c(self):
        return _Field(self.sigma2, self.corr_len, self.alpha_lo, self.alpha_span, self.seed, self.nu,
                      self.corr_len_z)


MLMC_MAX_LEVELS = 8


class _MlmcCfg(C.Structure):
    _fields_ = [("base", _Problem), ("field", _Field), ("nlevels", C.c_int32), ("n0", C.c_int32),
                ("steps0", C.c_int32), ("t_final", C.c_double),
                ("nsamples", C.c_int32 * MLMC_MAX_LEVELS), ("coupling", C.c_int32),
                ("continuation", C.c_int32), ("batch", C.c_int32), ("eps", C.c_double),
                ("key_offset", C.c_uint32), ("tune_threads", C.c_int32 * MLMC_MAX_LEVELS),
                ("tune_inner", C.c_int32 * MLMC_MAX_LEVELS), ("soil", _SoilModel), ("d_alpha", C.c_double),
                ("d_n", C.c_double), ("fixed_levels", C.c_int32), ("with_thetas", C.c_int32),
                ("bias_pairs", C.c_int32)]


_LV = C.c_double * MLMC_MAX_LEVELS
_LI = C.c_int64 * MLMC_MAX_LEVELS


class _MlmcResult(C.Structure):
    _fields_ = [("nlevels", C.c_int32), ("n", _LI), ("failed", _LI), ("mean", _LV), ("var", _LV),
                ("mean_f", _LV), ("var_f", _LV), ("mean_c", _LV), ("var_c", _LV), ("cost", _LV),
                ("cost_fine", _LV), ("n_opt", _LV), ("estimate", C.c_double), ("rmse", C.c_double),
                ("ml_variance", C.c_double), ("w_eps", C.c_double), ("w_mc_eps", C.c_double),
                ("bias_estimate", C.c_double), ("seconds", C.c_double), ("rounds", C.c_int32),
                ("bias_pairs", C.c_int64), ("bias_grid", C.c_double), ("bias_grid_se", C.c_double),
                ("total_rmse", C.c_double), ("levels_for_eps", C.c_int32), ("cost_sm", _LV),
                ("w_eps_sm", C.c_double)]


@dataclass
class MlmcConfig:
    """Levels l = 0..L: grid n0 2^l, steps0 2^l steps of t_final/(steps0 2^l),
    alpha_l = alpha (l+1)/(L+1) with continuation (Sec. 5)."""
    nsamples: tuple = (20000, 5000, 1200, 300, 80)
    n0: int = 16
    steps0: int = 5
    t_final: float = 0.1
    coupling: int = 0
    continuation: int = 1
    batch: int = 0
    eps: float = 1e-3
    key_offset: int = 0
    tune_threads: tuple = ()        # per level, 0 = the context's launch shape
    tune_inner: tuple = ()          # per level, 0 = the context's FP32 cycles per defect
    problem: Problem = field(default_factory=Problem)
    model: FieldModel = field(default_factory=FieldModel)
    # van Genuchten levels (problem.closure == VAN_GENUCHTEN): soil fields and
    # the additive (d_alpha, d_n) continuation of Sec. 5.2
    soil: SoilModel = field(default_factory=SoilModel)
    d_alpha: float = 0.05
    d_n: float = 0.1
    fixed_levels: int = 1
    with_thetas: int = 1
    # extra finest-level pairs at the original parameters for the grid-only
    # bias estimate (Eq. discErr) and the total RMSE; 0 = none
    bias_pairs: int = 0

    def _c(self):
        c = _MlmcCfg()
        c.base = self.problem._c()
        c.field = self.model._c()
        c.nlevels = len(self.nsamples)
        c.n0, c.steps0, c.t_final = self.n0, self.steps0, self.t_final
        for l, n in enumerate(self.nsamples):
            c.nsamples[l] = n
        c.coupling, c.continuation, c.batch, c.eps = self.coupling, self.continuation, self.batch, self.eps
        c.key_offset = self.key_offset
        for l, v in enumerate(self.tune_threads):
            c.tune_threads[l] = v
        for l, v in enumerate(self.tune_inner):
            c.tune_inner[l] = v
        c.soil = self.soil._c()
        c.d_alpha, c.d_n, c.fixed_levels, c.with_thetas = self.d_alpha, self.d_n, self.fixed_levels, self.with_thetas
        c.bias_pairs = self.bias_pairs
        return c


@dataclass
class Stats:
    picard_iters: int = 0
    mg_cycles: int = 0
    cell_vcycles: int = 0
    max_picard: int = 0
    failed: int = 0
    seconds: float = 0.0
    sm_seconds: float = 0.0


_lib = None


def lib():
    """Load librichards.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RichError(f"librichards.so not built ({LIB_PATH}); run paper_1903_08741_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u32, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
        L.rich_create.argtypes = [C.POINTER(vp), C.c_int]
        L.rich_destroy.argtypes = [vp]
        L.rich_status_str.argtypes = [C.c_int]
        L.rich_status_str.restype = C.c_char_p
        L.rich_last_error.restype = C.c_char_p
        L.rich_sample_fields.argtypes = [vp, C.POINTER(_Field), i32, i32, u32, i64, i32, i32, vp, vp, vp]
        L.rich_solve_batch.argtypes = [vp, C.POINTER(_Problem), i32, vp, vp, dbl, vp, vp, vp,
                                       C.POINTER(_Stats), vp]
        L.rich_solve_batch_host.argtypes = L.rich_solve_batch.argtypes
        L.rich_mlmc_accumulate.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp]
        L.rich_profile.argtypes = [vp, C.c_int]
        L.rich_profile_read.argtypes = [vp, C.POINTER(dbl), C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)]
        L.rich_launch_count.restype = i64
        L.rich_solve_batch_noalloc.argtypes = [C.POINTER(_Problem), i32, vp, vp, dbl, vp, vp, vp]
        L.rich_sample_fields_pair.argtypes = [vp, C.POINTER(_Field), i32, i32, u32, i64, i32, vp, vp, vp, vp, vp]
        L.rich_set_tuning.argtypes = [vp, i32, i32]
        L.rich_sample_fields_at.argtypes = [vp, C.POINTER(_Field), i32, i32, u32, vp, i32, i32, vp, vp, vp]
        L.rich_solve_batch_async.argtypes = [vp, C.POINTER(_Problem), i32, vp, vp, dbl, vp, vp, vp, vp]
        L.rich_kl_fields.argtypes = [vp, vp, i32, i32, vp, i32, vp, vp]
        L.rich_solve_batch_adjoint.argtypes = [vp, C.POINTER(_Problem), i32, vp, i32, vp, vp, dbl, i32, vp, vp,
                                               vp, vp, C.POINTER(_Stats), vp]
        L.rich_sample_soil.argtypes = [vp, C.POINTER(_Field), C.POINTER(_SoilModel), i32, i32, u32, i64, i32,
                                       i32, C.POINTER(_Soil), vp]
        L.rich_sample_soil_pair.argtypes = [vp, C.POINTER(_Field), C.POINTER(_SoilModel), i32, i32, u32, i64, i32,
                                            C.POINTER(_Soil), C.POINTER(_Soil), vp]
        L.rich_sample_counters.argtypes = [vp, i32, vp, vp, vp]
        L.rich_solve_soil.argtypes = [vp, C.POINTER(_Problem), i32, C.POINTER(_Soil), dbl, dbl, dbl, vp, vp, vp,
                                      C.POINTER(_Stats), vp]
        L.rich_mlmc_estimate.argtypes = [vp, C.POINTER(_MlmcCfg), C.POINTER(_MlmcResult)]
        L.rich_mlmc_adaptive.argtypes = [vp, C.POINTER(_MlmcCfg), i32, vp, C.POINTER(_MlmcResult)]
        L.rich_measure_fp64.argtypes = [vp, C.POINTER(_Fp64Rates)]
        L.rich_set_adjoint_method.argtypes = [vp, i32]
        L.rich_set_adjoint_limits.argtypes = [vp, dbl, i32]
        _lib = L
    return _lib


def exported_symbols():
    return ["rich_create", "rich_destroy", "rich_status_str", "rich_last_error",
            "rich_sample_fields", "rich_solve_batch", "rich_solve_batch_host",
            "rich_mlmc_accumulate", "rich_profile", "rich_profile_read", "rich_launch_count",
            "rich_solve_batch_noalloc", "rich_mlmc_estimate", "rich_sample_fields_pair",
            "rich_kl_fields", "rich_solve_batch_adjoint", "rich_set_tuning", "rich_sample_fields_at",
            "rich_solve_batch_async", "rich_mlmc_adaptive", "rich_sample_soil", "rich_solve_soil",
            "rich_sample_soil_pair", "rich_sample_counters", "rich_measure_fp64",
            "rich_set_adjoint_method", "rich_set_adjoint_limits"]


def _check(rc):
    if rc < 0:
        raise RichError(f"{lib().rich_status_str(rc).decode()}: {lib().rich_last_error().decode()}")
    return rc


_ctx = {}


def context(device: int = 0):
    """The library context of a CUDA device (created once per process)."""
    if device not in _ctx:
        h = C.c_void_p()
        _check(lib().rich_create(C.byref(h), device))
        _ctx[device] = h
    return _ctx[device]


def set_tuning(block_threads=0, mixed_inner=0, device=0):
    """Launch shape of the device's solves (see autotune.tune)."""
    _check(lib().rich_set_tuning(context(device), block_threads, mixed_inner))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RichError("librichards needs a CUDA device")
    return torch


def _stream(torch, device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_ptr(t, dtype, name):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise RichError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return C.c_void_p(t.data_ptr())


def sample_fields(nx, nz, nsamples, model: FieldModel | None = None, level=0, first_sample=0,
                  coarsen_times=0, device=0, out=None):
    """Draw (ln Ks, alpha) on device: [nsamples, nz >> c, nx >> c] float64 each."""
    torch = _torch()
    model = model or FieldModel()
    shape = (nsamples, nz >> coarsen_times, nx >> coarsen_times)
    if out is None:
        out = (torch.empty(shape, dtype=torch.float64, device=f"cuda:{device}"),
               torch.empty(shape, dtype=torch.float64, device=f"cuda:{device}"))
    lk, al = out
    _check(lib().rich_sample_fields(context(device), C.byref(model._c()), nx, nz, level, first_sample,
                                    nsamples, coarsen_times, _dev_ptr(lk, torch.float64, "lnKs"),
                                    _dev_ptr(al, torch.float64, "alpha"), _stream(torch, device)))
    return lk, al


def sample_fields_pair(nx, nz, nsamples, model: FieldModel | None = None, level=0, first_sample=0,
                       device=0):
    """Covariance-upscaled pair (Appendix A): fine [S, nz, nx] and coarse
    [S, nz/2, nx/2] ln Ks and alpha from one white-noise draw."""
    torch = _torch()
    model = model or FieldModel()
    d = f"cuda:{device}"
    f = [torch.empty((nsamples, nz, nx), dtype=torch.float64, device=d) for _ in range(2)]
    c = [torch.empty((nsamples, nz // 2, nx // 2), dtype=torch.float64, device=d) for _ in range(2)]
    _check(lib().rich_sample_fields_pair(context(device), C.byref(model._c()), nx, nz, level, first_sample,
                                         nsamples, *[_dev_ptr(t, torch.float64, "field") for t in (*f, *c)],
                                         _stream(torch, device)))
    return f[0], f[1], c[0], c[1]


def solve_batch(problem: Problem, lnKs, alpha, alpha_scale=1.0, want_p=False, device=None):
    """Solve every sample of lnKs/alpha ([S, nz, nx] float64 CUDA tensors).

    Returns (qoi [S], p_final [S, nz, nx] or None, status [S] int32, Stats, rc)."""
    torch = _torch()
    device = lnKs.device.index if device is None else device
    S = lnKs.shape[0]
    if tuple(lnKs.shape) != (S, problem.nz, problem.nx) or alpha.shape != lnKs.shape:
        raise RichError("lnKs/alpha must be [S, nz, nx]")
    qoi = torch.empty(S, dtype=torch.float64, device=lnKs.device)
    status = torch.empty(S, dtype=torch.int32, device=lnKs.device)
    p = torch.empty_like(lnKs) if want_p else None
    st = _Stats()
    rc = _check(lib().rich_solve_batch(context(device), C.byref(problem._c()), S,
                                       _dev_ptr(lnKs, torch.float64, "lnKs"),
                                       _dev_ptr(alpha, torch.float64, "alpha"), alpha_scale,
                                       _dev_ptr(qoi, torch.float64, "qoi"),
                                       None if p is None else _dev_ptr(p, torch.float64, "p"),
                                       _dev_ptr(status, torch.int32, "status"), C.byref(st),
                                       _stream(torch, device)))
    return qoi, p, status, Stats(*[getattr(st, f) for f, _ in _Stats._fields_]), rc


def soil_field_model(alpha_bl, model: FieldModel | None = None, d_alpha=0.2):
    """A FieldModel whose alpha marginal is alpha_bl +- d_alpha (Table soilparams)."""
    model = model or FieldModel.phi1()
    return FieldModel(**{**{f.name: getattr(model, f.name) for f in dc_fields(model)},
                         "alpha_lo": alpha_bl - d_alpha, "alpha_span": 2 * d_alpha})


def sample_soil(nx, nz, nsamples, model: FieldModel, soil: SoilModel, level=0, first_sample=0,
                coarsen_times=0, device=0, thetas=True):
    """The five soil fields (ln Ks, alpha, n, theta_s, theta_r) on device, each
    [nsamples, nz >> c, nx >> c] float64 (theta fields None when thetas=False)."""
    torch = _torch()
    shape = (nsamples, nz >> coarsen_times, nx >> coarsen_times)
    k = 5 if thetas else 3
    out = [torch.empty(shape, dtype=torch.float64, device=f"cuda:{device}") for _ in range(k)] + [None] * (5 - k)
    ptrs = _Soil(*[None if t is None else _dev_ptr(t, torch.float64, "soil field").value for t in out])
    _check(lib().rich_sample_soil(context(device), C.byref(model._c()), C.byref(soil._c()), nx, nz, level,
                                  first_sample, nsamples, coarsen_times, C.byref(ptrs), _stream(torch, device)))
    return tuple(out)


def sample_soil_pair(nx, nz, nsamples, model: FieldModel, soil: SoilModel, level=0, first_sample=0, device=0,
                     thetas=True):
    """The five soil fields as covariance-upscaled couples: (fine tuple of
    [S, nz, nx], coarse tuple of [S, nz/2, nx/2]); theta entries None when
    thetas=False."""
    torch = _torch()
    d = f"cuda:{device}"
    k = 5 if thetas else 3
    fine = [torch.empty((nsamples, nz, nx), dtype=torch.float64, device=d) for _ in range(k)] + [None] * (5 - k)
    coarse = [torch.empty((nsamples, nz // 2, nx // 2), dtype=torch.float64, device=d) for _ in range(k)]
    coarse += [None] * (5 - k)
    mk = lambda ts: _Soil(*[None if t is None else _dev_ptr(t, torch.float64, "soil field").value for t in ts])
    pf, pc = mk(fine), mk(coarse)
    _check(lib().rich_sample_soil_pair(context(device), C.byref(model._c()), C.byref(soil._c()), nx, nz, level,
                                       first_sample, nsamples, C.byref(pf), C.byref(pc), _stream(torch, device)))
    return tuple(fine), tuple(coarse)


def solve_soil(problem: Problem, lnKs, alpha, n=None, theta_s=None, theta_r=None, alpha_scale=1.0,
               alpha_shift=0.0, n_shift=0.0, want_p=False, device=None):
    """Solve with per-cell soil fields ([S, nz, nx] float64 CUDA tensors; the van
    Genuchten-Mualem closure needs n) and the additive continuation shifts of
    Sec. 5.  Returns (qoi, p_final or None, status, Stats, rc)."""
    torch = _torch()
    device = lnKs.device.index if device is None else device
    S = lnKs.shape[0]
    for t in (alpha, n, theta_s, theta_r):
        if t is not None and tuple(t.shape) != tuple(lnKs.shape):
            raise RichError("soil fields must share the shape [S, nz, nx]")
    if tuple(lnKs.shape) != (S, problem.nz, problem.nx):
        raise RichError("soil fields must be [S, nz, nx]")
    qoi = torch.empty(S, dtype=torch.float64, device=lnKs.device)
    status = torch.empty(S, dtype=torch.int32, device=lnKs.device)
    p = torch.empty_like(lnKs) if want_p else None
    ptrs = _Soil(*[None if t is None else _dev_ptr(t, torch.float64, "soil field").value
                   for t in (lnKs, alpha, n, theta_s, theta_r)])
    st = _Stats()
    rc = _check(lib().rich_solve_soil(context(device), C.byref(problem._c()), S, C.byref(ptrs), alpha_scale,
                                      alpha_shift, n_shift, _dev_ptr(qoi, torch.float64, "qoi"),
                                      None if p is None else _dev_ptr(p, torch.float64, "p"),
                                      _dev_ptr(status, torch.int32, "status"), C.byref(st),
                                      _stream(torch, device)))
    return qoi, p, status, Stats(*[getattr(st, f) for f, _ in _Stats._fields_]), rc


def sample_counters(nsamples, device=0):
    """Per-sample (Picard iterations, multigrid cycles) of the device's last
    solve, summed over its time steps: two int64 CUDA tensors [nsamples]."""
    torch = _torch()
    d = f"cuda:{device}"
    pic = torch.empty(nsamples, dtype=torch.int64, device=d)
    mg = torch.empty(nsamples, dtype=torch.int64, device=d)
    _check(lib().rich_sample_counters(context(device), nsamples, _dev_ptr(pic, torch.int64, "picard"),
                                      _dev_ptr(mg, torch.int64, "mg"), _stream(torch, device)))
    return pic, mg


def solve_batch_host(problem: Problem, lnKs: np.ndarray, alpha: np.ndarray, alpha_scale=1.0,
                     want_p=False, device=0):
    """As solve_batch with host (numpy) inputs and outputs; the library moves the data."""
    torch = _torch()
    lnKs = np.ascontiguousarray(lnKs, np.float64)
    alpha = np.ascontiguousarray(alpha, np.float64)
    S = lnKs.shape[0]
    qoi = np.empty(S, np.float64)
    status = np.empty(S, np.int32)
    p = np.empty_like(lnKs) if want_p else None
    st = _Stats()
    ptr = lambda a: None if a is None else C.c_void_p(a.ctypes.data)
    rc = _check(lib().rich_solve_batch_host(context(device), C.byref(problem._c()), S, ptr(lnKs),
                                            ptr(alpha), alpha_scale, ptr(qoi), ptr(p), ptr(status),
                                            C.byref(st), _stream(torch, device)))
    return qoi, p, status, Stats(*[getattr(st, f) for f, _ in _Stats._fields_]), rc


def mlmc_accumulate(acc, qoi_fine, status_fine=None, qoi_coarse=None, status_coarse=None):
    """Add one batch of level differences to the device FP64 accumulator acc[8]
    (sum Y, sum Y^2, count, failed, sum Qf, sum Qf^2, sum Qc, sum Qc^2)."""
    torch = _torch()
    dev = qoi_fine.device.index
    ptr = lambda t, dt, n: None if t is None else _dev_ptr(t, dt, n)
    _check(lib().rich_mlmc_accumulate(context(dev), ptr(qoi_fine, torch.float64, "qoi_fine"),
                                      ptr(qoi_coarse, torch.float64, "qoi_coarse"),
                                      ptr(status_fine, torch.int32, "status_fine"),
                                      ptr(status_coarse, torch.int32, "status_coarse"),
                                      qoi_fine.numel(), _dev_ptr(acc, torch.float64, "acc"),
                                      _stream(torch, dev)))
    return acc


def profile(enable=True, device=0):
    """Start (reset) or stop live event timing of the finest-level smoothing launches."""
    _check(lib().rich_profile(context(device), int(enable)))


def profile_read(device=0):
    """(milliseconds, launches, algorithmic bytes, algorithmic FLOPs) since profile(True)."""
    ms, n, b, f = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
    _check(lib().rich_profile_read(context(device), C.byref(ms), C.byref(n), C.byref(b), C.byref(f)))
    return ms.value, n.value, b.value, f.value


BICGSTAB, DEFECT_CORRECTION, GMRES = 1, 0, 2


def set_adjoint_method(method=BICGSTAB, device=0):
    """J^T solver of the device's adjoint solves: BICGSTAB (default), GMRES or DEFECT_CORRECTION."""
    _check(lib().rich_set_adjoint_method(context(device), method))


def set_adjoint_limits(rel_tol=1e-11, max_applications=400, device=0):
    """Stopping rule of the device's adjoint J^T solves: relative residual
    target and cap on preconditioner applications (then status ADJ_MAXIT)."""
    _check(lib().rich_set_adjoint_limits(context(device), float(rel_tol), int(max_applications)))


def measure_fp64(device=0):
    """FP64 FMA FLOP/s, divisions/s and exp/s of the device, measured by the
    library's microbenchmark kernels (the FP64 roofline denominator)."""
    _torch()
    r = _Fp64Rates()
    _check(lib().rich_measure_fp64(context(device), C.byref(r)))
    return {"dfma_flops": r.dfma_flops, "div_per_s": r.div_per_s, "exp_per_s": r.exp_per_s,
            "ms": r.ms_total}


def launch_count():
    """Kernels launched by librichards in this process so far."""
    return int(lib().rich_launch_count())


def _check_noalloc_args(problem: Problem, lnKs, alpha, qoi, status):
    """Shapes and devices of an allocation-free call, checked before anything
    reaches the library: the kernel reads S x nz x nx cells of each field and
    writes S entries of qoi and status, so a short or mis-shaped tensor would be
    read or written out of bounds on the device."""
    if lnKs.dim() != 3:
        raise RichError("lnKs must be [S, nz, nx]")
    S = lnKs.shape[0]
    if tuple(lnKs.shape) != (S, problem.nz, problem.nx) or tuple(alpha.shape) != tuple(lnKs.shape):
        raise RichError("lnKs/alpha must be [S, nz, nx] of the problem's grid")
    for name, t in (("qoi", qoi), ("status", status)):
        if t is not None and t.numel() < S:
            raise RichError(f"{name} must hold at least S = {S} entries")
    devs = {t.device for t in (lnKs, alpha, qoi, status) if t is not None}
    if len(devs) != 1:
        raise RichError("lnKs, alpha, qoi and status must be on one device")
    return S


def solve_batch_noalloc(problem: Problem, lnKs, alpha, alpha_scale=1.0, qoi=None, status=None):
    """Allocation-free solve (see include/richards.h): the library allocates
    nothing; the caller provides qoi [S] and status [S] (created here when not
    given).  Runs on lnKs's device, made current for the call; asynchronous on
    that device's current stream."""
    S = _check_noalloc_args(problem, lnKs, alpha, qoi, status)
    torch = _torch()
    if qoi is None:
        qoi = torch.empty(S, dtype=torch.float64, device=lnKs.device)
    if status is None:
        status = torch.empty(S, dtype=torch.int32, device=lnKs.device)
    with torch.cuda.device(lnKs.device):
        _check(lib().rich_solve_batch_noalloc(C.byref(problem._c()), S,
                                              _dev_ptr(lnKs, torch.float64, "lnKs"),
                                              _dev_ptr(alpha, torch.float64, "alpha"), alpha_scale,
                                              _dev_ptr(qoi, torch.float64, "qoi"),
                                              _dev_ptr(status, torch.int32, "status"),
                                              _stream(torch, lnKs.device.index)))
    return qoi, status


def _mlmc_result(r, rc):
    NL = r.nlevels
    out = {k: list(getattr(r, k))[:NL] for k in ("n", "failed", "mean", "var", "mean_f", "var_f", "mean_c",
                                                  "var_c", "cost", "cost_fine", "n_opt", "cost_sm")}
    out.update({k: getattr(r, k) for k in ("estimate", "rmse", "ml_variance", "w_eps", "w_mc_eps",
                                            "bias_estimate", "seconds", "rounds", "bias_pairs", "bias_grid",
                                            "bias_grid_se", "total_rmse", "levels_for_eps", "w_eps_sm")})
    out["nlevels"], out["rc"] = NL, rc
    return out


def mlmc_adaptive(cfg: MlmcConfig, max_rounds=10, nmax=None, device=0):
    """Algorithm PC_MLMC (Sec. 5.2): warm-up with cfg.nsamples, then optimal N_l for
    RMSE cfg.eps from measured V_l and C_l, repeated until no level needs more."""
    _torch()
    r = _MlmcResult()
    cap = None
    if nmax is not None:
        cap = (C.c_int64 * MLMC_MAX_LEVELS)(*[int(v) for v in nmax])
    rc = _check(lib().rich_mlmc_adaptive(context(device), C.byref(cfg._c()), max_rounds,
                                         None if cap is None else C.cast(cap, C.c_void_p), C.byref(r)))
    return _mlmc_result(r, rc)


def mlmc_estimate(cfg: MlmcConfig, device=0):
    """Multilevel Monte Carlo with parametric continuation on one GPU (host result)."""
    _torch()
    r = _MlmcResult()
    rc = _check(lib().rich_mlmc_estimate(context(device), C.byref(cfg._c()), C.byref(r)))
    return _mlmc_result(r, rc)


def kl_fields(basis, xi):
    """ln Ks [S, nz, nx] = sum_j xi[:, j] basis[j] (device tensors, float64)."""
    torch = _torch()
    nkl, nz, nx = basis.shape
    S = xi.shape[0]
    out = torch.empty((S, nz, nx), dtype=torch.float64, device=basis.device)
    dev = basis.device.index
    _check(lib().rich_kl_fields(context(dev), _dev_ptr(basis, torch.float64, "basis"), nkl, nz * nx,
                                _dev_ptr(xi, torch.float64, "xi"), S, _dev_ptr(out, torch.float64, "lnKs"),
                                _stream(torch, dev)))
    return out


def solve_batch_adjoint(problem: Problem, basis, xi, alpha, alpha_scale=1.0, ckpt_every=10, want_dlnks=False):
    """QoI [S] and dQ/dxi [S, n_kl] by the discrete adjoint (device tensors).
    Returns (qoi, dq_dxi, dq_dlnKs or None, status, Stats, rc)."""
    torch = _torch()
    nkl = basis.shape[0]
    S = xi.shape[0]
    dev = basis.device.index
    qoi = torch.empty(S, dtype=torch.float64, device=basis.device)
    dq = torch.empty((S, nkl), dtype=torch.float64, device=basis.device)
    status = torch.empty(S, dtype=torch.int32, device=basis.device)
    g = torch.empty((S, problem.nz, problem.nx), dtype=torch.float64, device=basis.device) if want_dlnks else None
    st = _Stats()
    rc = _check(lib().rich_solve_batch_adjoint(context(dev), C.byref(problem._c()), S,
                                               _dev_ptr(basis, torch.float64, "basis"), nkl,
                                               _dev_ptr(xi, torch.float64, "xi"),
                                               _dev_ptr(alpha, torch.float64, "alpha"), alpha_scale, ckpt_every,
                                               _dev_ptr(qoi, torch.float64, "qoi"), _dev_ptr(dq, torch.float64, "dq"),
                                               None if g is None else _dev_ptr(g, torch.float64, "g"),
                                               _dev_ptr(status, torch.int32, "status"), C.byref(st),
                                               _stream(torch, dev)))
    return qoi, dq, g, status, Stats(*[getattr(st, f) for f, _ in _Stats._fields_]), rc


def _autograd():
    import torch

    class RichardsQoI(torch.autograd.Function):
        """qoi = RichardsQoI.apply(xi, alpha, basis, problem[, alpha_scale, ckpt_every]):
        bottom-flux QoI of each sample with ln Ks = basis^T xi; backward returns
        grad_qoi[:, None] * dQ/dxi from the discrete adjoint."""

        @classmethod
        def apply(cls, xi, alpha, basis, problem, alpha_scale=1.0, ckpt_every=10):
            if not (torch.is_grad_enabled() and xi.requires_grad):
                # no gradient can flow (torch.no_grad(), or xi without
                # requires_grad): the forward solve alone, no adjoint sweep
                return solve_batch(problem, kl_fields(basis, xi.detach().contiguous()), alpha, alpha_scale)[0]
            return super().apply(xi, alpha, basis, problem, alpha_scale, ckpt_every)

        @staticmethod
        def forward(ctx, xi, alpha, basis, problem, alpha_scale=1.0, ckpt_every=10):
            if not ctx.needs_input_grad[0]:
                ctx.save_for_backward(None)
                return solve_batch(problem, kl_fields(basis, xi.detach().contiguous()), alpha, alpha_scale)[0]
            qoi, dq, _, status, _, _ = solve_batch_adjoint(problem, basis, xi.detach().contiguous(),
                                                           alpha, alpha_scale, ckpt_every)
            ctx.save_for_backward(dq)
            return qoi

        @staticmethod
        def backward(ctx, grad_qoi):
            (dq,) = ctx.saved_tensors
            if dq is None:
                return None, None, None, None, None, None
            return grad_qoi[:, None] * dq, None, None, None, None, None

    return RichardsQoI


def __getattr__(name):
    if name == "RichardsQoI":
        return _autograd()
    raise AttributeError(name)


def sample_fields_at(nx, nz, nsamples, first_sample_dev, out, model: FieldModel | None = None, level=0,
                     coarsen_times=0):
    """sample_fields with the first sample index read from a device int64 tensor
    (graph-capturable once the grid has been used outside the capture)."""
    torch = _torch()
    model = model or FieldModel()
    lk, al = out
    dev = lk.device.index
    if first_sample_dev.dtype != torch.int64 or not first_sample_dev.is_cuda:
        raise RichError("first_sample_dev must be a CUDA int64 tensor")
    _check(lib().rich_sample_fields_at(context(dev), C.byref(model._c()), nx, nz, level,
                                       C.c_void_p(first_sample_dev.data_ptr()), nsamples, coarsen_times,
                                       _dev_ptr(lk, torch.float64, "lnKs"), _dev_ptr(al, torch.float64, "alpha"),
                                       _stream(torch, dev)))
    return lk, al


def solve_batch_async(problem: Problem, lnKs, alpha, qoi, status, alpha_scale=1.0, p_final=None):
    """Enqueue the fused solve on the current stream (no host synchronisation;
    capturable in a CUDA graph after a first uncaptured call)."""
    torch = _torch()
    dev = lnKs.device.index
    _check(lib().rich_solve_batch_async(context(dev), C.byref(problem._c()), lnKs.shape[0],
                                        _dev_ptr(lnKs, torch.float64, "lnKs"), _dev_ptr(alpha, torch.float64, "alpha"),
                                        alpha_scale, _dev_ptr(qoi, torch.float64, "qoi"),
                                        None if p_final is None else _dev_ptr(p_final, torch.float64, "p_final"),
                                        _dev_ptr(status, torch.int32, "status"), _stream(torch, dev)))
