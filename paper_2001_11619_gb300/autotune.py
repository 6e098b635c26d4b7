"""Autotuner for the launch shapes of one workload.

The tuning parameters (``Solver.TUNING_KEYS``; the C call skel_set_tuning)
decide which kernel runs a box and how the sweeps cut right-hand sides
into CTAs.  They do not change the method.  The best values depend on the
tree the workload produces and on the form (FP64 or mixed).  Examples:
- a level of few, large boxes wants the 16-CTA cluster kernels;
- a crowded level wants one CTA per box.

:func:`tune` measures the quantity the bench reports, one factorization
plus one solve, with CUDA events on the solver's stream.  It searches one
parameter at a time over a short candidate list and keeps a change only
when it is faster by more than the measured noise.  It rejects a candidate
whose solution moves away from the default one by more than the solver's
tolerance: launch shapes may change rounding, not results.
:func:`save` and :func:`load` keep the result in a JSON file, keyed by a
workload signature.
"""
from __future__ import annotations

import json
import os

CANDIDATES = {
    "cluster_min_n": (96, 128, 160, 224, 320),
    "cluster_level_boxes": (0, 20, 40, 76, 152),
    "cluster_mid_min_n": (64, 80, 96, 112, 128, 1 << 30),
    "cluster_mid_level_boxes": (76, 152, 304, 608),
    "sweep_rhs_chunk": (4, 8, 16),
    "wide_min_n": (256, 384, 512, 768, 1024, 1 << 30),
    "wide_qr_min_n": (512, 768, 1024, 1536, 2048, 1 << 30),
}


def signature(solver, workload_name):
    """Key of a tuning result: the workload and the solver's form."""
    prm = solver.params
    return (f"{workload_name}|N={solver.N}|p={solver.p}|"
            f"leaf={prm.leaf_size}|prec={prm.precision}|tol={prm.id_tol:g}")


def _measure(solver, f, repeats):
    """Median over repeats of factor + solve, in ms (CUDA events on the
    current stream), and the last solution."""
    import torch
    times, x = [], None
    for _ in range(repeats):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        solver.factor()
        x = solver.solve(f)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2], x


def search(measure, start, candidates=CANDIDATES, noise=0.02):
    """Coordinate search: for each key in turn, try its candidates with the
    other keys held at the current best; keep the fastest if it beats the
    current time by more than ``noise`` (relative).  ``measure(config)``
    returns (ms, ok).  Returns (best config, best ms, log of trials)."""
    best = dict(start)
    best_ms, ok = measure(best)
    if not ok:
        raise RuntimeError("the starting configuration fails its check")
    log = [(dict(best), best_ms, True)]
    for key, values in candidates.items():
        cur = best.get(key)
        for v in values:
            if v == cur:
                continue
            cfg = dict(best, **{key: v})
            ms, ok = measure(cfg)
            log.append((cfg, ms, ok))
            if ok and ms < best_ms * (1.0 - noise):
                best, best_ms = cfg, ms
    return best, best_ms, log


def tune(solver, f, candidates=CANDIDATES, repeats=3, noise=0.02,
         rtol=1e-9):
    """Tune ``solver`` (any form) on right-hand side f; leaves the solver
    factored with the best configuration.  Returns {"config", "ms",
    "default_ms", "trials"}."""
    import torch
    start = solver.get_tuning()
    _measure(solver, f, 1)  # warm-up: buffers, graphs, module load
    ref_ms, ref = _measure(solver, f, repeats)
    ref_norm = float(torch.linalg.norm(torch.as_tensor(ref)))

    def measure(cfg):
        solver.set_tuning(**cfg)
        if cfg == start:
            return ref_ms, True
        ms, x = _measure(solver, f, repeats)
        diff = float(torch.linalg.norm(torch.as_tensor(x) -
                                       torch.as_tensor(ref)))
        return ms, diff <= rtol * ref_norm

    best, best_ms, log = search(measure, start, candidates, noise)
    solver.set_tuning(**best)
    solver.factor()
    return {"config": best, "ms": best_ms, "default_ms": ref_ms,
            "trials": [{"config": c, "ms": m, "ok": ok} for c, m, ok in log]}


def save(path, key, result):
    data = {}
    if os.path.exists(path):
        with open(path) as fh:
            data = json.load(fh)
    data[key] = {"config": result["config"], "ms": result["ms"],
                 "default_ms": result["default_ms"]}
    with open(path, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)


def load(path, key):
    """The stored configuration for key, or None."""
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        entry = json.load(fh).get(key)
    return None if entry is None else entry["config"]
