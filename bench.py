"""Benchmark: batched Monte Carlo Picard/CCMG solves of the stochastic Richards'
equation on GB300 (one JSON line on rank 0).

Default workload (N = 1): 4096 samples on a 128 x 128 grid, 20 implicit-Euler
steps of dt = 0.005, FP64, fields by FFT-MA from seed 0 (ln Ks: exp. covariance,
sigma^2 = 1, corr. length 0.3; alpha = 0.5 + 1.5 Phi(g)).  One bench step =
sample the batch's fields on the GPU + solve every sample + accumulate the MC
sums of the QoI (mean bottom flux) in FP64 on the GPU.  Inputs (~1.07 GB of
fields per step) exceed L2, and every step draws fresh samples.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload mc128|mc32] [--precision fp64|mixed]

Under torchrun (N > 1) every rank solves its own batch (weak scaling) and the
per-step MC sums are all-reduced (8 doubles, the estimator's one exchange).
``--impl reference`` times the FP64 CPU oracle on the host cores instead
(rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (grid side, samples per GPU, steps, dt)
    "mc128": (128, 4096, 20, 0.005),
    "mc32": (32, 64, 10, 0.01),
}
PHYS = dict(theta_r=0.1, theta_s=0.5, p_top=-0.5, p_bottom=-5.0, p_init=-5.0,
            picard_tol=1e-8, picard_maxit=50, mg_tol=1e-10, mg_maxit=100, nu1=2, nu2=2)
FP64_TFLOPS_NOMINAL = 1.25      # GB300 FP64 (non-tensor) nominal: 152 SMs x 2 FMA/clk x 2070 MHz x 2

# DRAM traffic of the fused solver per algorithmic byte: (dram__bytes_read.sum +
# dram__bytes_write.sum) of one launch of a reduced case of the workload (304
# samples, 2 time steps; ncu, see profiles/), divided by that launch's
# algorithmic bytes (the library's count).  The bench scales it by the timed
# launch's algorithmic bytes.  Valid only while the kernel sources are the
# ones captured (fused_sha()).
TRAFFIC = {
    # (precision, block_threads): (fused_sha() of the captured sources, DRAM bytes per algorithmic byte)
    ("fp64", 512): ("7f22827adec5c407e87fd507ed3f6a2f0b5fd91a9c973c9aa6fea8a4846256e6", 1.9240),
    ("mixed", 512): ("7f22827adec5c407e87fd507ed3f6a2f0b5fd91a9c973c9aa6fea8a4846256e6", 0.7142),
}


def fused_sha():
    """sha256 over the fused solver's sources (kernel header, then host code)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("fused_kernel.cuh", "fused.cu"):
        with open(os.path.join(ROOT, "paper_1903_08741_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def captured_traffic(prec_name, block_threads, alg_bytes_per_launch):
    ent = TRAFFIC.get((prec_name, block_threads))
    if ent is None or ent[0] != fused_sha():
        return None
    return ent[1] * alg_bytes_per_launch


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 9
                          for k in range(4) if r[5 + k].lower() == "active"})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def merge_step_sums(pg, step_acc, acc):
    """The estimator's one exchange: all-reduce (sum) the 8 FP64 MC sums of
    this step over the ranks and add them to the running total."""
    if pg is not None:
        pg.all_reduce(step_acc)
    acc += step_acc
    return acc


def max_over_ranks(pg, value, device):
    """Slowest rank's time (the bench reports whole-job throughput)."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# covariance of the Gaussian fields: the configured exponential exp(-r/0.3) and
# the paper's Matern sets Phi_1, Phi_2 (Eq. nonIsotropic and its table)
FIELDS = {"exp": {}, "phi1": dict(nu=1.0, corr_len=0.2, corr_len_z=0.2),
          "phi2": dict(nu=0.5, corr_len=0.1, corr_len_z=0.01)}
FIELD_TEXT = {"exp": "exp. cov. 0.3", "phi1": "Matern Phi_1 (nu 1, 0.2, 0.2)",
              "phi2": "Matern Phi_2 (nu 0.5, 0.1, 0.01)"}


def cpu_baseline(n, nsamples, steps, dt, seed=0, field="exp", cycle=1):
    """The FP64 oracle as it stands, on every host core: fields + solves of a
    bounded sample of the workload.  Returns (solves/s, cores, seconds)."""
    import oracle as O
    cores = os.cpu_count() or 1
    O.build()
    t0 = time.perf_counter()
    lk, al = O.sample_fields(n, n, nsamples, seed=seed, first_sample=10_000_000, nthreads=cores,
                             **FIELDS[field])
    pb = O.make_problem(nsteps=steps, dt=dt, gamma=cycle, **PHYS)
    O.solve_batch(pb, lk, al, nthreads=cores, want_p=False)
    dt_s = time.perf_counter() - t0
    return nsamples / dt_s, cores, dt_s


# The (alpha, n) values of the robustness study (Sec. 4.3, Table alpha_n).
MAP_ALPHAS = [0.2 * k for k in range(1, 21)]
MAP_NS = [1.1, 1.2, 1.3, 1.4, 1.5, 1.6, 1.7, 1.8, 1.9, 2.0, 2.2, 2.4, 2.6, 2.8, 3.0, 3.2, 3.4, 3.6, 3.8, 4.0]


def run_vgmap(args):
    """The solver-robustness study of Sec. 4.3: the infiltration problem (van
    Genuchten-Mualem, Eq. travellingwave) on h = 1/32 with dt = 1/64 to T = 0.1
    (6 steps), W(2,2) cycles, Picard and MG tolerances 1e-5, Ks = 0.2 exp(Z)
    with 64 Matern fields (Phi_1 unless --field phi2), for each of the 400
    (alpha, n) pairs of Table alpha_n: all 25,600 solves in one batched launch.
    Reports solves/s, and per pair the mean W-cycles per solve and the number
    of failed samples (the paper's cost and failure maps)."""
    import math
    import numpy as np
    import torch
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    field = args.field if args.field != "exp" else "phi1"
    n, reps = 32, args.samples or 64
    dt = 1.0 / 64
    steps = args.time_steps or round(0.1 / dt)
    prec = R.MIXED if args.precision == "mixed" else R.FP64
    na, nn = len(MAP_ALPHAS), len(MAP_NS)
    S = na * nn * reps
    lk, _ = R.sample_fields(n, n, reps, R.FieldModel(seed=0, **FIELDS[field]))
    lk = (lk + math.log(0.2)).repeat(na * nn, 1, 1).contiguous()          # pair-major, 64 fields each
    pa = torch.tensor(MAP_ALPHAS, dtype=torch.float64, device=dev).repeat_interleave(nn * reps)
    pn = torch.tensor(MAP_NS, dtype=torch.float64, device=dev).repeat(na).repeat_interleave(reps)
    al = pa[:, None, None].expand(S, n, n).contiguous()
    nf = pn[:, None, None].expand(S, n, n).contiguous()
    pb = R.Problem.infiltration(nx=n, nz=n, nsteps=steps, dt=dt, precision=prec, cycle=args.cycle)
    from paper_1903_08741_gb300 import autotune
    if args.launch:
        block_threads, mixed_inner = (int(x) for x in args.launch.split("/"))
        R.set_tuning(block_threads, mixed_inner)
    else:
        block_threads, mixed_inner = autotune.tune(pb, S)
    for _ in range(args.warmup):
        R.solve_soil(pb, lk[:1024], al[:1024], nf[:1024])
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = R.launch_count()
    R.profile(True)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        q, _, st, stats, _ = R.solve_soil(pb, lk, al, nf)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    kms, klaunch, kbytes, kflops = R.profile_read()
    R.profile(False)
    launches = R.launch_count() - l0
    clk = clocks.stop()
    pic, mg = R.sample_counters(S)
    stv = st.cpu().numpy().reshape(na, nn, reps)
    mgv = mg.cpu().numpy().reshape(na, nn, reps).astype(np.float64)
    fail = ((stv == 1) | (stv == 3)).sum(axis=2)
    okm = np.where((stv == 0) | (stv == 2), mgv, np.nan)
    with np.errstate(invalid="ignore"):
        mean_cyc = np.nanmean(okm, axis=2)
    value = S * args.steps / (ms / 1e3)
    k_tflops = kflops / (kms / 1e3) / 1e12 if kms > 0 else 0.0
    out = {
        "metric": "Picard-MG solves/s", "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == R.FP64 else "f32-in-f64", "data": "synthetic",
        "config": {"workload": f"vgmap: infiltration problem, van Genuchten-Mualem, {n}x{n} grid, {steps} steps "
                               f"dt=1/64, {na}x{nn} (alpha, n) pairs x {reps} Ks fields ({FIELD_TEXT[field]}), "
                               f"cycle index {pb.cycle}, tolerances 1e-5",
                   "global_batch": S, "launch": {"block_threads": block_threads, "mixed_inner": mixed_inner},
                   "l2": "inputs larger than L2 (3 x %.0f MB soil fields)" % (S * n * n * 8 / 1e6)},
        "clocks": clk, "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": k_tflops, "peak": FP64_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                     "frac": k_tflops / FP64_TFLOPS_NOMINAL, "traffic": None,
                     "peak_kind": "FP64 nominal (152 SMs x 2 FMA/clk x 2.07 GHz)",
                     "note": "multigrid and Picard-assembly FLOPs only; the van Genuchten closure's "
                             "transcendentals are not counted"},
        "failed_samples": int(fail.sum()), "mean_wcycles_per_solve": float(np.nanmean(okm)),
        "map": {"alpha": [round(a, 10) for a in MAP_ALPHAS], "n": MAP_NS,
                "mean_cycles": [[None if not np.isfinite(v) else round(float(v), 1) for v in row] for row in mean_cyc],
                "failures": fail.tolist()},
    }
    if not args.no_cpu:
        import oracle as O
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        ns = args.cpu_samples or 2 * cores
        sel = np.arange(ns) * (S // ns)
        pbo = O.infiltration_problem(nsteps=steps, dt=dt, gamma=pb.cycle)
        O.solve_batch_soil(pbo, lk[sel].cpu().numpy(), al[sel].cpu().numpy(), nf[sel].cpu().numpy(),
                           want_p=False, nthreads=cores)
        secs = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": ns / secs, "unit": "solves/s", "cores": cores, "kind": "oracle",
                               "sample": f"{ns} solves spread over the map, {secs:.1f} s"}
    print(json.dumps(out))


def workload_suffix(args):
    """Non-default field model / cycle, appended to the workload name."""
    out = ""
    if args.field != "exp":
        out += ", " + FIELD_TEXT[args.field]
    if args.cycle != 1:
        out += f", cycle index {args.cycle}"
    return out


def run_reference(args):
    ws, rank, local, pg = dist_setup(args)
    n, S, steps, dt = WORKLOADS[args.workload]
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    per_step = max(cores, args.ref_samples or cores)
    for _ in range(args.warmup):
        cpu_baseline(n, per_step, steps, dt, field=args.field, cycle=args.cycle)
    t = 0.0
    for _ in range(args.steps):
        _, _, s = cpu_baseline(n, per_step, steps, dt, field=args.field, cycle=args.cycle)
        t += s
    value = per_step * args.steps / t
    sample = f"{per_step} samples per step of the {n}x{n}, {steps}-step workload"
    print(json.dumps({
        "impl": "reference", "metric": "Picard-MG solves/s", "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"mc{n}: {n}x{n} grid, {S} samples, {steps} steps dt={dt}, FP64"
                               + workload_suffix(args), "sample": sample},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


MLMC_LEVELS = dict(nsamples=(20000, 5000, 1200, 300, 80), n0=16, steps0=5, t_final=0.1)


def mlmc_launch_batch(levels, nl, level=None):
    """Pairs per solver launch of an MLMC level: the estimator (rich_mlmc_estimate
    with cfg.batch = 0) holds B = 2^31 / (16 n_L^2) finest-level fields, n_L the
    finest grid, and solves level l (grid m) in launches of B (n_L / m)^2
    pairs, so each level is tuned for that launch size."""
    L = len(levels["nsamples"]) - 1
    nL = levels["n0"] << L
    B = max(1, (1 << 31) // (16 * nL * nL))
    if level is None:
        level = list(levels["nsamples"]).index(nl)
    r = nL // (levels["n0"] << level)
    return min(nl, B * r * r)


def mlmc_tuning(R, prec, cycle=1):
    """Per-level launch shapes of the five-level hierarchy from the autotuner."""
    from paper_1903_08741_gb300 import autotune
    tt, ti = [], []
    for l, nl in enumerate(MLMC_LEVELS["nsamples"]):
        m = MLMC_LEVELS["n0"] << l
        st_l = MLMC_LEVELS["steps0"] << l
        bt, mi = autotune.tune(R.Problem(nx=m, nz=m, nsteps=st_l, dt=MLMC_LEVELS["t_final"] / st_l,
                                         precision=prec, cycle=cycle, **PHYS), mlmc_launch_batch(MLMC_LEVELS, nl, l))
        tt.append(bt)
        ti.append(mi)
    R.set_tuning(0, 0)
    return tt, ti


def mlmc_config(R, prec, coupling, field="exp", cycle=1, bias_pairs=0, key_offset=0):
    tt, ti = mlmc_tuning(R, prec, cycle)
    return R.MlmcConfig(**MLMC_LEVELS, coupling=coupling, eps=1e-3, tune_threads=tuple(tt), tune_inner=tuple(ti),
                        problem=R.Problem(precision=prec, cycle=cycle, **PHYS),
                        model=R.FieldModel(seed=0, **FIELDS[field]), bias_pairs=bias_pairs, key_offset=key_offset)


def mlmc_warmup(R, cfg, k=0):
    small = R.MlmcConfig(nsamples=(64, 32, 16, 8, 4), n0=16, steps0=5, t_final=0.1, coupling=cfg.coupling,
                         key_offset=100 + k, problem=cfg.problem, model=cfg.model,
                         tune_threads=cfg.tune_threads, tune_inner=cfg.tune_inner)
    R.mlmc_estimate(small)


def mlmc_report(r, cfg):
    """The estimator's figures: level statistics, W(eps) (Eq. MLMCSAMP_ch6),
    sampling RMSE, grid-only bias and total RMSE (Eqs. discErr, MSEMLMC_ch6)."""
    out = {"w_eps_s": r["w_eps"], "eps": 1e-3,
           "w_eps_full_gpu_s": r["w_eps_sm"],
           "levels": {k: r[k] for k in ("n", "failed", "mean", "var", "cost", "cost_sm", "cost_fine", "n_opt",
                                        "mean_f", "var_f")},
           "cost_note": "cost: wall seconds per pair of this run's batches; cost_sm: GPU-seconds per pair on a "
                        "fully occupied GPU (field time + the solves' SM-seconds / SMs), the per-pair cost that "
                        "W(eps) assumes once N_l fills the GPU",
           "estimate": r["estimate"], "sampling_rmse": r["rmse"], "ml_variance": r["ml_variance"],
           "w_mc_eps_s": r["w_mc_eps"], "mc_over_mlmc": r["w_mc_eps"] / r["w_eps"],
           "bias_with_continuation_jump": r["bias_estimate"], "run_seconds": r["seconds"],
           "launch": {"block_threads": list(cfg.tune_threads), "mixed_inner": list(cfg.tune_inner),
                      "from": "autotuner, per level"}}
    if r["bias_pairs"] > 0:
        out.update({"bias_grid_only": r["bias_grid"], "bias_grid_only_se": r["bias_grid_se"],
                    "bias_pairs": r["bias_pairs"], "total_rmse": r["total_rmse"],
                    "levels_for_eps": r["levels_for_eps"]})
    return out


def mlmc_batch1(R, cfg):
    """The hierarchy with one sample per launch (batch 1) on N_l = 200/50/12/3/2:
    per-level costs of unbatched GPU solves; the level variances are the
    batched run's, which these few samples cannot estimate."""
    c1 = R.MlmcConfig(**{**MLMC_LEVELS, "nsamples": (200, 50, 12, 3, 2)}, coupling=cfg.coupling, eps=1e-3,
                      batch=1, key_offset=500, tune_threads=(1024,) * 5, tune_inner=cfg.tune_inner,
                      problem=cfg.problem, model=cfg.model)
    R.mlmc_estimate(R.MlmcConfig(nsamples=(2, 2), n0=16, steps0=5, t_final=0.1, batch=1, coupling=cfg.coupling,
                                 key_offset=600, problem=cfg.problem, model=cfg.model))
    return R.mlmc_estimate(c1)


def w_eps(var, cost, eps=1e-3):
    import math
    return sum(math.sqrt(max(v, 0.0) * c) for v, c in zip(var, cost)) ** 2 / eps ** 2


def run_mlmc(args):
    """Parametric-continuation MLMC over 16^2..256^2 (5 levels, N_l = 20000, 5000,
    1200, 300, 80; 5 2^l steps to T = 0.1): reports V_l, C_l and the cost W(eps)
    to RMSE 1e-3 from the measured V_l and C_l (Eq. MLMCSAMP_ch6)."""
    import torch
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    prec = R.MIXED if args.precision == "mixed" else R.FP64
    cfg = mlmc_config(R, prec, args.coupling, args.field, args.cycle, bias_pairs=args.bias_pairs)
    if args.batch1:
        return run_mlmc_batch1(args, R, cfg, prec)
    for k in range(args.warmup):
        mlmc_warmup(R, cfg, k)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = R.launch_count()
    res = []
    for k in range(args.steps):
        cfg.key_offset = 10 * k
        res.append(R.mlmc_estimate(cfg))
    launches = R.launch_count() - l0
    clk = clocks.stop()
    r = res[-1]
    secs = sum(x["seconds"] for x in res) / len(res)
    out = {
        "metric": "MLMC cost to RMSE 1e-3 (s)", "value": r["w_eps"], "unit": "s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == R.FP64 else "f32-in-f64", "data": "synthetic",
        "config": {"workload": "mlmc5: 16^2..256^2, N_l = 20000/5000/1200/300/80, 5*2^l steps to T=0.1, "
                               f"alpha_l = alpha (l+1)/5, {FIELD_TEXT[args.field]}, seed 0"
                               + (f", cycle index {args.cycle}" if args.cycle > 1 else ""),
                   "coupling": COUPLING_TEXT[args.coupling]},
        "clocks": clk, "gpu_launches": launches,
    }
    out.update(mlmc_report(r, cfg))
    if args.adaptive_eps > 0:
        acfg = R.MlmcConfig(**{**MLMC_LEVELS, "nsamples": (512, 128, 32, 16, 8)}, coupling=args.coupling,
                            eps=args.adaptive_eps, key_offset=1000, tune_threads=cfg.tune_threads,
                            tune_inner=cfg.tune_inner, problem=cfg.problem, model=cfg.model)
        a = R.mlmc_adaptive(acfg, max_rounds=10)
        out["adaptive"] = {"eps": args.adaptive_eps, "rounds": a["rounds"], "n": a["n"], "failed": a["failed"],
                           "rmse": a["rmse"], "estimate": a["estimate"], "seconds": a["seconds"],
                           "var": a["var"], "cost": a["cost"], "w_eps_predicted": a["w_eps"]}
    print(json.dumps(out))


COUPLING_TEXT = {0: "finest-grid draw, 2x2 averages of ln Ks and alpha",
                 1: "level-grid draw, 2x2 averages of ln Ks and alpha",
                 2: "covariance upscaling (2x2-averaged white noise)"}


MLMC_VG_LEVELS = dict(nsamples=(20000, 5000, 1200, 300, 80), n0=16, steps0=3, t_final=0.2)


def run_mlmc_vg(args):
    """The paper's MLMC experiment (Sec. 5.2): the infiltration problem with the
    van Genuchten-Mualem closure and five soil fields (Table soilparams, Matern
    Phi_1 unless --field phi2) on 16^2..256^2 with 3 2^l steps to T = 0.2
    (dt_l close to h_l), target parameters alpha_L = 3.0, n_L = 1.45 (Phi_2:
    2.8, 1.55) on the finest level, additive continuation d_alpha = 0.05,
    d_n = 0.1 below it, W(2,2) cycles, tolerances 1e-5, N_l = 20000/5000/
    1200/300/80, coupling by covariance upscaling.  Reports V_l, C_l and
    W(eps = 1e-3), with the continuation and without it."""
    import torch
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    prec = R.MIXED if args.precision == "mixed" else R.FP64
    field = args.field if args.field != "exp" else "phi1"
    a_l, n_l = (3.0, 1.45) if field == "phi1" else (2.8, 1.55)
    base = R.Problem.infiltration(precision=prec, cycle=args.cycle)
    model = R.soil_field_model(a_l, R.FieldModel(seed=0, **FIELDS[field]))
    soil = R.SoilModel(n_bl=n_l)
    from paper_1903_08741_gb300 import autotune
    tt, ti = [], []
    for l, nl in enumerate(MLMC_VG_LEVELS["nsamples"]):
        m = MLMC_VG_LEVELS["n0"] << l
        st_l = MLMC_VG_LEVELS["steps0"] << l
        bt, mi = autotune.tune(R.Problem.infiltration(nx=m, nz=m, nsteps=st_l, dt=MLMC_VG_LEVELS["t_final"] / st_l,
                                                      precision=prec, cycle=base.cycle),
                               mlmc_launch_batch(MLMC_VG_LEVELS, nl, l))
        tt.append(bt)
        ti.append(mi)
    R.set_tuning(0, 0)
    common = dict(coupling=2, eps=1e-3, tune_threads=tuple(tt), tune_inner=tuple(ti), problem=base,
                  model=model, soil=soil, d_alpha=0.05, d_n=0.1, fixed_levels=args.fixed_levels)
    for k in range(args.warmup):
        R.mlmc_estimate(R.MlmcConfig(nsamples=(64, 32, 16, 8, 4), n0=16, steps0=3, t_final=0.2,
                                     key_offset=100 + k, **common))
    clocks = ClockSampler(0)
    clocks.start()
    l0 = R.launch_count()
    res = {}
    for cont in (1, 0):
        for k in range(args.steps):
            res[cont] = R.mlmc_estimate(R.MlmcConfig(**MLMC_VG_LEVELS, key_offset=10 * k, continuation=cont,
                                                     **common))
    launches = R.launch_count() - l0
    clk = clocks.stop()
    r = res[1]
    lev = lambda x: {k: x[k] for k in ("n", "failed", "mean", "var", "cost", "n_opt", "mean_f", "var_f")}
    out = {
        "metric": "MLMC cost to RMSE 1e-3 (s)", "value": r["w_eps"], "unit": "s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["seconds"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == R.FP64 else "f32-in-f64", "data": "synthetic",
        "config": {"workload": f"mlmc5vg: infiltration problem, van Genuchten-Mualem, five soil fields "
                               f"({FIELD_TEXT[field]}), 16^2..256^2, 3*2^l steps to T=0.2, alpha_L={a_l}, "
                               f"n_L={n_l}, d_alpha=0.05, d_n=0.1, {args.fixed_levels} finest level(s) unperturbed, "
                               f"cycle index {base.cycle}, tolerances 1e-5, "
                               f"N_l = 20000/5000/1200/300/80, covariance upscaling"},
        "clocks": clk, "gpu_launches": launches,
        "levels": lev(r), "estimate": r["estimate"], "rmse": r["rmse"],
        "w_mc_eps_s": r["w_mc_eps"], "mc_over_mlmc": r["w_mc_eps"] / r["w_eps"],
        "no_continuation": {"w_eps": res[0]["w_eps"], "levels": lev(res[0]), "estimate": res[0]["estimate"]},
        "launch": {"block_threads": tt, "mixed_inner": ti, "from": "autotuner, per level"},
    }
    print(json.dumps(out))


def run_mlmc_batch1(args, R, cfg, prec):
    """Per-level costs with one sample per launch (see mlmc_batch1)."""
    clocks = ClockSampler(0)
    clocks.start()
    l0 = R.launch_count()
    r = mlmc_batch1(R, cfg)
    launches = R.launch_count() - l0
    clk = clocks.stop()
    print(json.dumps({
        "metric": "MLMC cost per pair, batch 1 (s)", "value": r["cost"][-1], "unit": "s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": 1e3 * r["seconds"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == R.FP64 else "f32-in-f64",
        "data": "synthetic",
        "config": {"workload": "mlmc5 hierarchy with batch 1 (one sample per launch), N_l = 200/50/12/3/2, "
                               f"coupling {cfg.coupling}"},
        "clocks": clk, "gpu_launches": launches,
        "levels": {k: r[k] for k in ("n", "failed", "cost", "cost_fine")},
    }))


def run_adjoint(args):
    """Discrete adjoint (256^2 grid, 256 samples, 50 steps of dt = 0.002, ln Ks
    from a 128-mode KL expansion of exp(-r/0.2), xi ~ N(0,1) seed 0, alpha as
    in the 32^2 workload): gradients of the bottom-flux QoI w.r.t. the KL
    coefficients per second.  --check adds central finite differences (step
    1e-6, tight tolerances) on 2 samples x 2 coefficients."""
    import numpy as np
    import torch
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build as B
    from paper_1903_08741_gb300.kl import kl_basis
    B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    n, S, steps, dt, nkl = 256, args.samples or 256, args.time_steps or 50, 0.002, 128
    prec = R.MIXED if args.precision == "mixed" else R.FP64
    basis, lam = kl_basis(n, n, nkl, 1.0, 0.2)
    Bd = torch.from_numpy(basis).to(dev)
    xi = torch.from_numpy(np.random.default_rng(0).normal(size=(S, nkl))).to(dev)
    _, al = R.sample_fields(n, n, S, R.FieldModel(seed=0))
    pb = R.Problem(nx=n, nz=n, nsteps=steps, dt=dt, precision=prec, **PHYS)
    method = {"bicgstab": R.BICGSTAB, "gmres": R.GMRES, "dc": R.DEFECT_CORRECTION}[args.adjoint_method]
    R.set_adjoint_method(method)
    for k in range(args.warmup):
        small = R.Problem(nx=n, nz=n, nsteps=2, dt=dt, precision=prec, **PHYS)
        R.solve_batch_adjoint(small, Bd, xi[:8].contiguous(), al[:8].contiguous(), ckpt_every=10)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = R.launch_count()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        q, dq, _, st, stats, rc = R.solve_batch_adjoint(pb, Bd, xi, al, ckpt_every=10)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    launches = R.launch_count() - l0
    clk = clocks.stop()
    stv = st.cpu().numpy()
    out = {
        "metric": "adjoint gradients/s", "value": S * args.steps / (ms / 1e3), "unit": "gradients/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == R.FP64 else "f32-in-f64", "data": "synthetic",
        "config": {"workload": f"adjoint{n}: {n}x{n} grid, {S} samples, {steps} steps dt={dt}, "
                               f"ln Ks = 128-mode KL (exp. cov. 0.2), checkpoint every 10 steps",
                   "jt_solver": args.adjoint_method,
                   "kl_variance_captured": float(lam.sum() / (n * n))},
        "clocks": clk, "gpu_launches": launches,
        "failed_samples": int(((stv == 1) | (stv == 3)).sum()),
        "adjoint_linear_solve_limit_hit": int((stv == R.ADJ_MAXIT).sum()),
        "forward_mg_limit_hit": int((stv == R.MG_MAXIT).sum()),
        "picard_iters_per_sample": stats.picard_iters / S,
        "adjoint_preconditioner_applications_per_sample": stats.mg_cycles / S,
        "mean_qoi": float(np.nanmean(q.cpu().numpy())),
        "mean_abs_grad": float(np.nanmean(np.abs(dq.cpu().numpy()))),
    }
    if args.check:
        tight = dict(PHYS)
        tight.update(picard_tol=1e-13, mg_tol=1e-14, picard_maxit=200, mg_maxit=400)
        pt = R.Problem(nx=n, nz=n, nsteps=steps, dt=dt, **tight)
        sel = [0, 1]
        qa, dqa, _, sta, _, _ = R.solve_batch_adjoint(pt, Bd, xi[sel].contiguous(), al[sel].contiguous())
        errs = []
        for j in (0, 7):
            xp, xm = xi[sel].clone(), xi[sel].clone()
            xp[:, j] += 1e-6
            xm[:, j] -= 1e-6
            qp = R.solve_batch(pt, R.kl_fields(Bd, xp), al[sel].contiguous())[0]
            qm = R.solve_batch(pt, R.kl_fields(Bd, xm), al[sel].contiguous())[0]
            fd = ((qp - qm) / 2e-6).cpu().numpy()
            a = dqa[:, j].cpu().numpy()
            errs += list(np.abs(a - fd) / np.maximum(np.abs(fd), 1e-300))
        out["fd_check"] = {"samples": sel, "coefficients": [0, 7], "max_rel_err": float(max(errs)),
                           "tolerances": "Picard 1e-13, MG 1e-14, step 1e-6"}
    print(json.dumps(out))


def run_mc512(args):
    """512^2 grid, 160 steps of dt = 0.1/160 (h = dt scaling of the level
    hierarchy), the 32^2 workload's field model: FP32 V-cycles in FP64 defect
    correction vs the FP64 batched path on the same samples; QoI error of the
    mixed path relative to FP64."""
    import numpy as np
    import torch
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    n, S, steps = 512, args.samples or 1024, args.time_steps or 160
    dt = 0.1 / 160
    lk, al = R.sample_fields(n, n, S, R.FieldModel(seed=0))
    res = {}
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(0)
    clocks.start()
    from paper_1903_08741_gb300 import autotune
    tuning = {}
    for name, prec in (("mixed", R.MIXED), ("fp64", R.FP64)):
        pb = R.Problem(nx=n, nz=n, nsteps=steps, dt=dt, precision=prec, **PHYS)
        tuning[name] = autotune.tune(pb, S)
        R.solve_batch(pb, lk[:4].contiguous(), al[:4].contiguous())       # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q, _, st, stats, rc = R.solve_batch(pb, lk, al)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        res[name] = (q.cpu().numpy(), st.cpu().numpy(), e0.elapsed_time(e1), stats)
    clk = clocks.stop()
    qm, sm_, tm, stm = res["mixed"]
    qd, sd, td, std_ = res["fp64"]
    ok = (sm_ == 0) & (sd == 0)
    rel = np.abs(qm[ok] - qd[ok]) / np.abs(qd[ok])
    out = {
        "metric": "Picard-MG solves/s", "value": S / (tm / 1e3), "unit": "solves/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": tm, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-in-f64", "data": "synthetic",
        "config": {"workload": f"mc512: {n}x{n} grid, {S} samples, {steps} steps dt={dt:.6g}",
                   "launch": {k: {"block_threads": v[0], "mixed_inner": v[1]} for k, v in tuning.items()}},
        "clocks": clk,
        "fp64": {"value": S / (td / 1e3), "ms": td, "vcycles_per_sample": std_.mg_cycles / S},
        "mixed_vcycles_per_sample": stm.mg_cycles / S,
        "speedup_mixed_vs_fp64": td / tm,
        "qoi_rel_err_mixed_vs_fp64": {"max": float(rel.max()), "median": float(np.median(rel)), "n": int(ok.sum())},
        "failed": {"mixed": int(((sm_ == 1) | (sm_ == 3)).sum()), "fp64": int(((sd == 1) | (sd == 3)).sum())},
    }
    print(json.dumps(out))


def measure_fp64_rates(R, device):
    """The library's FP64 microbenchmark, with the SM clocks sampled meanwhile."""
    clocks = ClockSampler(device)
    clocks.start()
    r = R.measure_fp64(device)
    r2 = R.measure_fp64(device)          # two passes: the sampler sees ~2 s of load
    clk = clocks.stop()
    best = max((r, r2), key=lambda x: x["dfma_flops"])
    best["clocks"] = clk
    return best


def fp64_peak_tflops(fp64, clk):
    """FP64 roofline denominator: the measured FMA rate, scaled to the median SM
    clock of the timed region when the two clock readings differ; the nominal
    unit-count figure when no measurement exists."""
    if not fp64:
        return FP64_TFLOPS_NOMINAL, "FP64 nominal (152 SMs x 2 FMA/clk x 2.07 GHz)"
    peak = fp64["dfma_flops"] / 1e12
    f_meas = (fp64.get("clocks") or {}).get("sm_mhz")
    f_run = (clk or {}).get("sm_mhz")
    if f_meas and f_run and abs(f_meas - f_run) > 1:
        return peak * f_run / f_meas, (f"FP64 FMA microbenchmark (measured, {f_meas:.0f} MHz) "
                                       f"scaled to the timed region's {f_run:.0f} MHz")
    return peak, f"FP64 FMA microbenchmark (measured{f', %.0f MHz' % f_meas if f_meas else ''})"


def bench_extras(R, args, pb, lk, al, q64, s64, clk):
    """The rest of the headline metric on one GPU: (a) the mixed-precision
    batched solve of the same workload on the e2e step's fields, with its QoI
    error against the FP64 solve of those fields; (b) the five-level MLMC
    (coupling 2) to RMSE 1e-3 in FP64 and in mixed precision, with grid-only
    bias pairs and the total RMSE; (c) the per-level costs with one sample per
    launch and the ratio of that FP64 batch-1 cost to the mixed batched cost."""
    import numpy as np
    import torch
    from paper_1903_08741_gb300 import autotune
    out = {}
    dev = lk.device
    stream = torch.cuda.current_stream(dev)
    # (a) mixed precision, mc128
    pm = R.Problem(**{**pb.__dict__, "precision": R.MIXED})
    bt, mi = autotune.tune(pm, lk.shape[0])
    R.solve_batch(pm, lk[:8].contiguous(), al[:8].contiguous())
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    qm, _, sm_, stm, _ = R.solve_batch(pm, lk, al)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    mclk = clocks.stop()
    tm = e0.elapsed_time(e1)
    S = lk.shape[0]
    mixed = {"value": S / (tm / 1e3), "unit": "solves/s", "ms_per_step": tm, "clocks": mclk,
             "launch": {"block_threads": bt, "mixed_inner": mi},
             "failed_samples": stm.failed, "converged_solves_per_s": (S - stm.failed) / (tm / 1e3),
             "what": "one batch (4096 samples, 128^2, 20 steps) on the e2e step's fields, FP32 V-cycles in "
                     "FP64 defect correction"}
    if q64 is not None:
        qm, sm_ = qm.cpu().numpy(), sm_.cpu().numpy()
        ok = (sm_ == 0) & (s64 == 0)
        rel = np.abs(qm[ok] - q64[ok]) / np.abs(q64[ok])
        mixed["qoi_rel_err_vs_fp64"] = {"max": float(rel.max()), "median": float(np.median(rel)),
                                        "n": int(ok.sum()), "same_status": float((sm_ == s64).mean())}
    out["mixed_mc128"] = mixed
    # (b) MLMC, FP64 and mixed, coupling 2
    res = {}
    for name, prec in (("fp64", R.FP64), ("mixed", R.MIXED)):
        cfg = mlmc_config(R, prec, 2, bias_pairs=152 if prec == R.FP64 else 0)
        mlmc_warmup(R, cfg)
        clocks = ClockSampler(dev.index or 0)
        clocks.start()
        r = R.mlmc_estimate(cfg)
        rep = mlmc_report(r, cfg)
        rep["clocks"] = clocks.stop()
        res[name] = (r, cfg, rep)
    out["mlmc5"] = {"workload": "mlmc5: 16^2..256^2, N_l = 20000/5000/1200/300/80, 5*2^l steps to T=0.1, "
                                "alpha_l = alpha (l+1)/5, exp. cov. 0.3, seed 0, " + COUPLING_TEXT[2],
                    "fp64": res["fp64"][2], "mixed": res["mixed"][2]}
    # (c) batch-1 costs (FP64) and the ratio to the mixed batched cost
    r1 = mlmc_batch1(R, res["fp64"][1])
    w1 = w_eps(res["fp64"][0]["var"], r1["cost"])
    out["mlmc5"]["fp64_batch1"] = {"cost": r1["cost"], "n": r1["n"], "w_eps_s": w1,
                                   "note": "one sample per launch, N_l = 200/50/12/3/2; W(eps) from the "
                                           "batched FP64 V_l"}
    out["mlmc5"]["ratio_fp64_batch1_over_mixed_batched"] = w1 / res["mixed"][0]["w_eps"]
    out["mlmc5"]["ratio_fp64_batched_over_mixed_batched"] = res["fp64"][0]["w_eps"] / res["mixed"][0]["w_eps"]
    return out


def run_tunecheck(args):
    """The autotuner against the full batch: for the 128^2 workload (FP64 and
    mixed) and every level of the five-level MLMC hierarchy, time each launch
    shape on the whole batch (2 time steps, fresh fields) and report how far
    the tuner's choice is from the fastest."""
    import torch
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import autotune
    from paper_1903_08741_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    steps = args.time_steps or 2
    cases = []
    for prec in (R.FP64, R.MIXED):
        cases.append((R.Problem(nx=128, nz=128, nsteps=20, dt=0.005, precision=prec, **PHYS), 4096, "mc128"))
        for l, nl in enumerate(MLMC_LEVELS["nsamples"]):
            m, st_l = MLMC_LEVELS["n0"] << l, MLMC_LEVELS["steps0"] << l
            cases.append((R.Problem(nx=m, nz=m, nsteps=st_l, dt=MLMC_LEVELS["t_final"] / st_l, precision=prec,
                                    **PHYS), mlmc_launch_batch(MLMC_LEVELS, nl, l), f"mlmc5 level {l}"))
    out = []
    for pb, S, name in cases:
        src = autotune.source(pb, S)
        r = autotune.check(pb, S, steps=steps)
        r.update({"case": name, "tuner_source": src})
        out.append(r)
    print(json.dumps({"metric": "autotuner shortfall vs best shape on the full batch", "steps": steps,
                      "max_shortfall": max(r["tuner_shortfall"] for r in out), "cases": out}))


def run_ours(args):
    import numpy as np
    import torch
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build as B

    ws, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if pg is not None:
        pg.barrier()
    dev = torch.device(f"cuda:{local}")
    n, S, steps, dt = WORKLOADS[args.workload]
    S = args.samples or S
    steps = args.time_steps or steps
    prec = R.MIXED if args.precision == "mixed" else R.FP64
    pb = R.Problem(nx=n, nz=n, nsteps=steps, dt=dt, precision=prec, cycle=args.cycle, **PHYS)
    from paper_1903_08741_gb300 import autotune
    if args.launch:
        block_threads, mixed_inner = (int(x) for x in args.launch.split("/"))
        R.set_tuning(block_threads, mixed_inner, local)
        launch_from = "--launch"
    else:
        launch_from = "autotuner (" + autotune.source(pb, S, local) + ")"
        block_threads, mixed_inner = autotune.tune(pb, S, device=local)
    model = R.FieldModel(seed=0, **FIELDS[args.field])
    lk = torch.empty((S, n, n), dtype=torch.float64, device=dev)
    al = torch.empty_like(lk)
    acc = torch.zeros(8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sample_base = rank * 1_000_000

    step_acc = torch.zeros(8, dtype=torch.float64, device=dev)

    def step(k):
        R.sample_fields(n, n, S, model, level=0, first_sample=sample_base + k * S, device=local,
                        out=(lk, al))
        q, _, st, stats, rc = R.solve_batch(pb, lk, al, device=local)
        step_acc.zero_()
        R.mlmc_accumulate(step_acc, q, st)
        merge_step_sums(pg, step_acc, acc)
        return stats

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)
    default_run = (args.workload == "mc128" and not args.samples and not args.time_steps
                   and args.field == "exp" and args.cycle == 1 and prec == R.FP64)
    extras = ws == 1 and default_run and not args.no_extras
    fp64 = measure_fp64_rates(R, local) if (prec == R.FP64 and ws == 1) else None
    if pg is not None:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    R.profile(True, device=local)
    l0 = R.launch_count()
    acc.zero_()
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tot = R.Stats()
    for k in range(args.steps):
        st = step(args.warmup + k)
        for f in ("picard_iters", "mg_cycles", "cell_vcycles", "failed"):
            setattr(tot, f, getattr(tot, f) + getattr(st, f))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    launches = R.launch_count() - l0
    kms, klaunch, kbytes, kflops = R.profile_read(device=local)
    R.profile(False, device=local)
    clk = clocks.stop()
    ms = max_over_ranks(pg, ms, dev)
    total = S * args.steps * ws
    value = total / (ms / 1e3)
    a = acc.cpu().numpy()

    # the same step as one captured CUDA graph (device-side sample offset, async
    # solve, accumulation), replayed once on fresh samples
    graph = None
    if not args.no_graph:
        first = torch.tensor([sample_base + 8_000_000], dtype=torch.int64, device=dev)
        qg = torch.empty(S, dtype=torch.float64, device=dev)
        sg = torch.empty(S, dtype=torch.int32, device=dev)
        side = torch.cuda.Stream(dev)
        with torch.cuda.stream(side):
            R.sample_fields_at(n, n, S, first, (lk, al), model)
            R.solve_batch_async(pb, lk[:8], al[:8], qg[:8], sg[:8])
            torch.cuda.synchronize(dev)
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=side):
                R.sample_fields_at(n, n, S, first, (lk, al), model)
                R.solve_batch_async(pb, lk, al, qg, sg)
                R.mlmc_accumulate(acc, qg, sg)
                first.add_(S)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(side)
            gr.replay()
            g1.record(side)
            torch.cuda.synchronize(dev)
        gms = max_over_ranks(pg, g0.elapsed_time(g1), dev)
        graph = {"value": S * ws / (gms / 1e3), "unit": "solves/s", "ms_per_step": gms,
                 "what": "fields + fused solve + accumulation captured as one CUDA graph, one replay"}

    # end to end through the host-buffer entry point: H2D of the fields, solve,
    # D2H of QoI and status, every step inside the timed region
    e2e = None
    qh = sh = None
    if not args.no_e2e:
        R.sample_fields(n, n, S, model, level=0, first_sample=sample_base + 9_000_000, device=local,
                        out=(lk, al))
        hl = torch.empty((S, n, n), dtype=torch.float64, pin_memory=True)
        ha = torch.empty_like(hl, pin_memory=True)
        hl.copy_(lk)
        ha.copy_(al)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            qh, _, sh, _, _ = R.solve_batch_host(pb, hl.numpy(), ha.numpy(), device=local)
        t_e2e = max_over_ranks(pg, time.perf_counter() - t0, dev)
        e2e = {"value": S * ws * args.e2e_steps / t_e2e, "unit": "solves/s",
               "h2d_bytes_per_step": 2 * S * n * n * 8, "d2h_bytes_per_step": S * 8 + S * 4}

    if rank != 0:
        return
    hbm_peak, peak_kind = load_peaks()
    k_gbs = kbytes / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    k_tflops = kflops / (kms / 1e3) / 1e12 if kms > 0 else 0.0
    frac_hbm = k_gbs / hbm_peak
    fp64_peak, fp64_kind = fp64_peak_tflops(fp64, clk)
    frac_alu = k_tflops / fp64_peak if prec == R.FP64 else 0.0
    per_launch_bytes = kbytes / max(klaunch, 1)
    kname = f"k_fused<{'double' if prec == R.FP64 else 'float'},{block_threads}> (persistent fused solve)"
    traffic = captured_traffic("fp64" if prec == R.FP64 else "mixed", block_threads, per_launch_bytes)
    if prec == R.FP64 and frac_alu > frac_hbm:
        roof = {"bound": "alu", "achieved": k_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": frac_alu, "traffic": traffic, "kernel": kname, "peak_kind": fp64_kind,
                "hbm": {"achieved": k_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": frac_hbm,
                        "peak_kind": peak_kind}}
    else:
        roof = {"bound": "hbm", "achieved": k_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": frac_hbm,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": kname}
    roof.update({"launches": klaunch, "alg_bytes_per_launch": per_launch_bytes,
                 "avg_launch_us": 1e3 * kms / max(klaunch, 1), "kernel_ms_total": kms})
    out = {
        "metric": "Picard-MG solves/s", "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == R.FP64 else "f32-in-f64", "data": "synthetic",
        "config": {"workload": f"mc{n}: {n}x{n} grid, {S} samples/GPU, {steps} steps dt={dt}, "
                               f"{'FP64' if prec == R.FP64 else 'FP32 V-cycles in FP64 defect correction'}"
                               + workload_suffix(args),
                   "global_batch": S * ws, "grid": [n, n], "time_steps": steps,
                   "launch": {"block_threads": block_threads, "mixed_inner": mixed_inner, "from": launch_from},
                   "l2": "inputs larger than L2 (2 x %.0f MB fields per step, fresh samples each step)"
                         % (S * n * n * 8 / 1e6)},
        "clocks": clk, "gpu_launches": launches, "roofline": roof,
        "cell_updates_per_s": total * n * n * steps / (ms / 1e3),
        "cell_vcycles_per_s": tot.cell_vcycles * ws / (ms / 1e3),
        "picard_iters_per_sample": tot.picard_iters / (S * args.steps),
        "vcycles_per_sample": tot.mg_cycles / (S * args.steps),
        "failed_samples": tot.failed,
        "failed_fraction": tot.failed / total,
        "converged_solves_per_s": (total - tot.failed) / (ms / 1e3),
        "mc_estimate": {"mean_qoi": a[0] / max(a[2], 1), "n": int(a[2]), "failed": int(a[3]),
                        "note": "mean over converged samples (failed samples, Sec. 4.3, are excluded)"},
    }
    if fp64 is not None:
        out["fp64_rates"] = fp64
    if e2e:
        out["e2e"] = e2e
    if graph:
        out["graph"] = graph
    if extras:
        out.update(bench_extras(R, args, pb, lk, al, qh, sh, clk))
    if not args.no_cpu and ws == 1:
        cores = os.cpu_count() or 1
        ns = args.cpu_samples or cores
        v, c, secs = cpu_baseline(n, ns, steps, dt, field=args.field, cycle=args.cycle)
        out["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": c, "kind": "oracle",
                               "sample": f"{ns} samples of the {n}x{n}, {steps}-step workload "
                                         f"(fields + solves), {secs:.1f} s"}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["mlmc5", "mlmc5vg", "adjoint256", "mc512", "vgmap",
                                                               "tunecheck"],
                    default="mc128")
    ap.add_argument("--check", action="store_true", help="adjoint workload: finite-difference check")
    ap.add_argument("--adjoint-method", choices=["bicgstab", "gmres", "dc"], default="bicgstab",
                    help="adjoint workload: solver of the J^T systems")
    ap.add_argument("--adaptive-eps", type=float, default=0.0, help="mlmc5: also run Algorithm PC_MLMC to this RMSE")
    ap.add_argument("--coupling", type=int, default=0, help="MLMC field coupling (0 exact, 1 level grid)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--field", choices=sorted(FIELDS), default="exp",
                    help="covariance of the fields: exponential 0.3 (configured) or Matern Phi_1 / Phi_2")
    ap.add_argument("--batch1", action="store_true",
                    help="mlmc5: per-level costs with one sample per launch (reduced N_l)")
    ap.add_argument("--fixed-levels", type=int, default=1,
                    help="mlmc5vg: finest levels solved with the original (alpha, n) (Sec. 5.2)")
    ap.add_argument("--cycle", type=int, default=0, choices=[0, 1, 2, 3],
                    help="multigrid cycle index: 1 V-cycle, 2 W-cycle (0: the workload's own, V for the "
                         "configured workloads, W for vgmap)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--launch", default="", help="mc and vgmap workloads: launch shape block_threads/mixed_inner "
                                                 "(e.g. 512/4) instead of the autotuner's")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the mixed-precision, MLMC and batch-1 measurements")
    ap.add_argument("--bias-pairs", type=int, default=0, help="mlmc5: grid-only bias pairs (Eq. discErr)")
    ap.add_argument("--cpu-samples", type=int, default=0)
    ap.add_argument("--ref-samples", type=int, default=0)
    # profiling knobs (smaller cases for ncu captures; not bench workloads)
    ap.add_argument("--samples", type=int, default=0, help="override samples per GPU")
    ap.add_argument("--time-steps", type=int, default=0, help="override implicit-Euler steps")
    args = ap.parse_args()
    args.cycle = args.cycle or (2 if args.workload in ("vgmap", "mlmc5vg") else 1)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mlmc5":
        run_mlmc(args)
    elif args.workload == "adjoint256":
        run_adjoint(args)
    elif args.workload == "mc512":
        run_mc512(args)
    elif args.workload == "vgmap":
        run_vgmap(args)
    elif args.workload == "mlmc5vg":
        run_mlmc_vg(args)
    elif args.workload == "tunecheck":
        run_tunecheck(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
