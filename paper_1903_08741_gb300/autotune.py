"""Autotuner of the fused solver's launch shape.

Candidates: 32-thread CTAs (grids up to 32^2: a sample per warp, 32 resident
per SM, no CTA-wide barrier), 128- and 256-thread CTAs (eight or four resident
per SM: small grids, whose levels give a large CTA too little work between
barriers),
512-thread CTAs (two per
SM) or 1024-thread CTAs (one per SM: the fewest resident scratch slots, so more
of the hierarchy stays in L2, and the most threads per sample); for the mixed path
also the number of FP32 V-cycles per FP64 defect (1, 2, 3, 4, 6).  Each
candidate solves a probe batch of the same grid and precision (fresh seeded
fields, two time steps) timed with CUDA events.  The probe is the production
batch itself, up to 64 samples per SM: the persistent kernel balances samples
of unequal cost through its queue, so a probe with only a few samples per CTA
is set by its slowest samples and misranks the shapes.  The fastest candidate
is cached in a JSON file keyed by device, grid, precision and batch size
(rounded up to a power of two) and applied to the context with
rich_set_tuning.  Choices measured on GB300 ship with the package
(tune_defaults.json) and are used when the user cache has no entry.  The
choice never changes an FP64 result (block shape) or the FP64 tolerance
(inner cycles).
"""
from __future__ import annotations

import json
import os
import time


SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_defaults.json")


def cache_path():
    base = os.environ.get("RICH_TUNE_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(root, "librichards", "tune.json")


def _bucket(n):
    b = 1
    while b < n:
        b *= 2
    return b


def _key(problem, nsamples, device_name):
    prec = "mixed" if problem.precision else "fp64"
    cyc = "" if problem.cycle <= 1 else f"|W{problem.cycle}"    # V-cycle keys stay as they were
    clo = "" if problem.closure == 0 else "|VG"
    return f"{device_name}|{problem.nx}x{problem.nz}|{prec}|S{_bucket(nsamples)}{cyc}{clo}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def shapes(problem):
    """Candidate CTA sizes: one-warp CTAs (32 per SM, a whole sample on one
    warp) only for grids of at most 32^2 cells, where a larger CTA spends its
    time at barriers between a few cells of work; 128 ... 1024 for all."""
    small = problem.nx * problem.nz <= 32 * 32
    return ((32,) if small else ()) + (128, 256, 512, 1024)


def source(problem, nsamples, device=0):
    """Where tune() would take this key's choice from: "cache", "shipped" or
    "measure"."""
    import torch
    key = _key(problem, nsamples, torch.cuda.get_device_name(torch.device(f"cuda:{device}")))
    if key in _load(cache_path()):
        return "cache"
    return "shipped" if key in _load(SHIPPED) else "measure"


def tune(problem, nsamples, device=0, force=False, probe_steps=2, verbose=False, shipped=True):
    """Return (block_threads, mixed_inner) for this grid/precision/batch and
    apply it to the device's context; measures and caches when neither the
    user cache nor (with shipped=True) the package's defaults hold the key."""
    import torch
    import paper_1903_08741_gb300 as R
    dev = torch.device(f"cuda:{device}")
    name = torch.cuda.get_device_name(dev)
    path = cache_path()
    data = _load(path)
    key = _key(problem, nsamples, name)
    if not force:
        for src in (data, _load(SHIPPED) if shipped else {}):
            if key in src:
                bt, mi = src[key]["block_threads"], src[key]["mixed_inner"]
                R.set_tuning(bt, mi, device)
                return bt, mi
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    S = max(1, min(nsamples, 64 * sms))
    if problem.closure == R.VAN_GENUCHTEN:
        # van Genuchten kernels probe on soil fields of a mid-range soil
        flds = R.sample_soil(problem.nx, problem.nz, S, R.soil_field_model(2.0, R.FieldModel(seed=987654321)),
                             R.SoilModel(n_bl=1.6), device=device, thetas=False)[:3]
        solve = lambda k: R.solve_soil(probe, *[f[:k].contiguous() for f in flds])
    else:
        lk, al = R.sample_fields(problem.nx, problem.nz, S, R.FieldModel(seed=987654321), device=device)
        solve = lambda k: R.solve_batch(probe, lk[:k].contiguous(), al[:k].contiguous())
    probe = R.Problem(**{**problem.__dict__, "nsteps": max(1, min(problem.nsteps, probe_steps))})
    inners = [1, 2, 3, 4, 6] if problem.precision else [0]
    timings = {}
    stream = torch.cuda.current_stream(dev)
    for bt in shapes(problem):
        for mi in inners:
            R.set_tuning(bt, mi, device)
            solve(min(S, 8))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solve(S)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            timings[f"{bt}/{mi}"] = e0.elapsed_time(e1)
            if verbose:
                print(f"tune {key}: block {bt} inner {mi}: {timings[f'{bt}/{mi}']:.1f} ms")
    best = min(timings, key=timings.get)
    bt, mi = (int(x) for x in best.split("/"))
    data = _load(path)
    data[key] = {"block_threads": bt, "mixed_inner": mi, "probe_ms": timings, "probe_samples": S,
                 "probe_steps": probe.nsteps, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    _save(path, data)
    R.set_tuning(bt, mi, device)
    return bt, mi


def check(problem, nsamples, device=0, steps=None, verbose=False):
    """Time every candidate launch shape on the FULL batch (fresh seeded
    fields, `steps` time steps, default the problem's own) and compare the
    fastest with the shape tune() chooses.  Returns a dict with the
    per-candidate milliseconds, the best shape, the tuner's shape and the
    tuner's shortfall (its time / the best time - 1)."""
    import torch
    import paper_1903_08741_gb300 as R
    dev = torch.device(f"cuda:{device}")
    chosen = tune(problem, nsamples, device=device)
    pb = R.Problem(**{**problem.__dict__, "nsteps": steps or problem.nsteps})
    if problem.closure == R.VAN_GENUCHTEN:
        flds = R.sample_soil(problem.nx, problem.nz, nsamples, R.soil_field_model(2.0, R.FieldModel(seed=123457)),
                             R.SoilModel(n_bl=1.6), device=device, thetas=False)[:3]
        solve = lambda k: R.solve_soil(pb, *[f[:k].contiguous() for f in flds])
    else:
        lk, al = R.sample_fields(problem.nx, problem.nz, nsamples, R.FieldModel(seed=123457), device=device)
        solve = lambda k: R.solve_batch(pb, lk[:k].contiguous(), al[:k].contiguous())
    inners = [1, 2, 3, 4, 6] if problem.precision else [0]
    stream = torch.cuda.current_stream(dev)
    ms = {}
    try:
        for bt in shapes(problem):
            for mi in inners:
                R.set_tuning(bt, mi, device)
                solve(min(nsamples, 8))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                solve(nsamples)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms[f"{bt}/{mi}"] = e0.elapsed_time(e1)
                if verbose:
                    print(f"check {problem.nx}x{problem.nz} S{nsamples}: {bt}/{mi} {ms[f'{bt}/{mi}']:.1f} ms")
    finally:
        R.set_tuning(*chosen, device)
    best = min(ms, key=ms.get)
    key = f"{chosen[0]}/{chosen[1]}"
    return {"grid": [problem.nx, problem.nz], "precision": "mixed" if problem.precision else "fp64",
            "samples": nsamples, "steps": pb.nsteps, "ms": ms, "best": best, "tuner": key,
            "tuner_shortfall": ms[key] / ms[best] - 1.0}
