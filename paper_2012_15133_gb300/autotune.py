"""Autotuner of the launch schedules (FFT tile shapes) of the CUDA solver.

For a grid (d, N) and a precision, every schedule compiled into the library
(``spfc_num_schedules``) is timed through the C interface on a seeded
synthetic state: steady-state steps (CUDA-graph replay) and steps with the L2
flushed before each one. The fastest schedule by the sum of both times is
stored in a JSON table keyed by GPU name, d, N and precision;
``Solver(..., schedule="auto")`` reads it (schedule 0 when there is no entry).

Every candidate must also reproduce schedule 0's step to rounding (the
schedules only change tile shapes), which the tuner checks before timing.

    python -m paper_2012_15133_gb300.autotune --n 512 256 --precision fp32 fp64
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "autotune_cache.json")
_PREC = {"fp64": 0, "fp32": 1, 0: 0, 1: 1}


def cache_path() -> str:
    return os.environ.get("SPFC_TUNE_CACHE", DEFAULT_CACHE)


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _key(d, n, precision) -> str:
    return f"{_gpu_name()}|d{int(d)}|n{int(n)}|{'fp64' if _PREC[precision] == 0 else 'fp32'}"


def lookup(d, n, precision) -> int:
    """Tuned schedule for this GPU, grid and precision (0 if untuned)."""
    try:
        with open(cache_path()) as f:
            table = json.load(f)
        return int(table.get(_key(d, n, precision), {}).get("schedule", 0))
    except (OSError, ValueError):
        return 0


def _batch_key(n, precision) -> str:
    return f"{_gpu_name()}|batch|n{int(n)}|{'fp64' if _PREC[precision] == 0 else 'fp32'}"


def lookup_batch(n, precision) -> int:
    """Tuned batch schedule of grid size n for this GPU (-1, the default, if untuned)."""
    try:
        with open(cache_path()) as f:
            table = json.load(f)
        return int(table.get(_batch_key(n, precision), {}).get("schedule", -1))
    except (OSError, ValueError):
        return -1


def batch_schedules(n):
    """The schedules a batch class of grid size n can be built with."""
    from .spfc import load_library
    lib = load_library()
    return [s for s in range(6) if lib.spfc_batch_schedule_valid(int(n), s)]


def _batch_runs(n, count):
    """Ensemble runs of one grid size (the ensemble recipe at size n)."""
    from seeded_inputs import ensemble_run
    return [ensemble_run(i, sizes=(n,)) for i in range(count)]


def time_batch(n, precision, schedule, runs=16, steps=64):
    """us per batched step of `runs` runs at n^2 (graph replay; the class's
    working set, 5 half spectra per run, exceeds the L2 from 512^2 x 16)."""
    import torch
    from .spfc import Batch
    rs = _batch_runs(n, runs)
    b = Batch(rs, 0.02, precision, schedule={n: schedule})
    for i, r in enumerate(rs):
        b.init(i, r["phi0"], "bdf1")
    b.step(16)
    b.sync()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    b.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / steps


def check_batch(n, precision, schedule, runs=4, nsteps=3):
    """Relative L2 difference of a batch schedule's fields from the default's."""
    from .spfc import Batch
    rs = _batch_runs(n, runs)
    out = []
    for sch in (-1, schedule):
        b = Batch(rs, 0.02, precision, schedule={n: sch})
        for i, r in enumerate(rs):
            b.init(i, r["phi0"], "bdf1")
        b.step(nsteps)
        out.append(np.stack([b.get_field(i) for i in range(runs)]))
    return float(np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0]))


def tune_batch(n, precision, write=True, verbose=True):
    """Time every batch schedule of grid size n (after the parity check) and
    store the fastest under the key (GPU, batch, n, precision)."""
    tol = 1e-12 if _PREC[precision] == 0 else 1e-5
    results = {}
    for sch in batch_schedules(n):
        err = check_batch(n, precision, sch)
        if not err < tol:
            raise RuntimeError(f"batch schedule {sch} disagrees with the default (rel-L2 {err:.2e})")
        us = time_batch(n, precision, sch)
        results[sch] = {"step_us": us, "rel_l2_vs_default": err}
        if verbose:
            print(f"batch n={n} {precision} schedule {sch}: {us:.1f} us per batched step, rel-L2 {err:.1e}")
    best = min(results, key=lambda k: results[k]["step_us"])
    if write:
        path = cache_path()
        try:
            with open(path) as fh:
                table = json.load(fh)
        except (OSError, ValueError):
            table = {}
        table[_batch_key(n, precision)] = {"schedule": best, "timings": results}
        with open(path, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
    return best, results


def _field(n):
    """A fixed synthetic initial state (mean 0.2, noise 0.02): timing input only."""
    rng = np.random.default_rng(12345)
    return 0.2 + 0.02 * rng.uniform(-1.0, 1.0, size=(n, n))


def time_schedule(n, precision, schedule, steps=400, flushed_steps=100, L=None):
    """(resident us/step, L2-flushed us/step) of one schedule on a 2D n^2 run."""
    import torch
    from .spfc import Solver
    L = 0.5 * n if L is None else L
    s = Solver(2, n, L, 0.25, 1.0, 0.05, precision, schedule=schedule)
    s.init(_field(n), "bdf1")
    st = torch.cuda.current_stream()
    s.step(32)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    s.step(steps)
    b.record(st)
    torch.cuda.synchronize()
    resident = a.elapsed_time(b) * 1e3 / steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(flushed_steps)]
    for i in range(flushed_steps):
        flush.fill_(float(i))
        evs[i][0].record(st)
        s.step(1)
        evs[i][1].record(st)
    torch.cuda.synchronize()
    flushed = sum(x.elapsed_time(y) for x, y in evs) * 1e3 / flushed_steps
    s.sync()
    return resident, flushed


def check_schedule(n, precision, schedule, nsteps=3):
    """Relative L2 difference between a schedule's field and schedule 0's after nsteps."""
    from .spfc import Solver
    out = []
    for sch in (0, schedule):
        s = Solver(2, n, 0.5 * n, 0.25, 1.0, 0.05, precision, schedule=sch)
        s.init(_field(n), "bdf1")
        s.step(nsteps)
        out.append(s.get_field(0))
    return float(np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0]))


def tune(n, precision, write=True, verbose=True):
    from .spfc import num_schedules
    tol = 1e-12 if _PREC[precision] == 0 else 1e-5
    results = {}
    for sch in range(num_schedules(2, n)):
        err = check_schedule(n, precision, sch)
        if not err < tol:
            raise RuntimeError(f"schedule {sch} disagrees with schedule 0 (rel-L2 {err:.2e})")
        r, f = time_schedule(n, precision, sch)
        results[sch] = {"resident_us": r, "flushed_us": f, "rel_l2_vs_0": err}
        if verbose:
            print(f"n={n} {precision} schedule {sch}: resident {r:.2f} us, flushed {f:.2f} us, rel-L2 vs 0 {err:.1e}")
    best = min(results, key=lambda k: results[k]["resident_us"] + results[k]["flushed_us"])
    if write:
        path = cache_path()
        try:
            with open(path) as fh:
                table = json.load(fh)
        except (OSError, ValueError):
            table = {}
        table[_key(2, n, precision)] = {"schedule": best, "timings": results}
        with open(path, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
    return best, results


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[512, 256, 128])
    ap.add_argument("--precision", nargs="+", default=["fp32", "fp64"])
    ap.add_argument("--batch", action="store_true", help="tune the batched ensemble's classes instead")
    args = ap.parse_args()
    from .build import build
    build()
    for prec in args.precision:
        for n in args.n:
            if args.batch:
                best, _ = tune_batch(n, prec)
                print(f"best batch schedule for n={n} {prec}: {best}")
            else:
                best, _ = tune(n, prec)
                print(f"best schedule for n={n} {prec}: {best}")


if __name__ == "__main__":
    main()
