#!/usr/bin/env python
"""Benchmark of the GB300 skeletonization solver.

One step = the whole hot path on one synthetic geometry: build the quadtree
(geometry already resident in HBM), factor the bordered system level by
level, form the boundary data, solve, and evaluate the velocity at the
interior targets.  The workload is the 32768-node, 16-hole star geometry
(65584 unknowns).  The metric is unknowns per second of that step in the
mixed-precision form (FP32 factors with FP64 rank decisions, GMRES on the
FP64 operator); the same step in the all-FP64 form is timed beside it, and
the moved-hole update time of both forms is reported.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

With N > 1 (torchrun) every rank solves its own replica (no communication
on the data path); value is the sum over ranks divided by the slowest rank.
``--impl reference`` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("factor unknowns/s, update ms/moved hole: mixed vs FP64 GPU "
          "@1e-10 rel err")
UNIT = "unknowns/s"
WORKLOAD = "star16"
WORKLOAD_DESC = ("star r=1+0.15cos7t with 16 seeded ellipses "
                 "(semi-axes U[0.03,0.08]), 24576+16x512 = 32768 nodes, "
                 "65584 unknowns")
STEP_DESC = ("build_tree + factor + point-force boundary data + solve "
             "(1 rhs) + velocity at 1024 interior targets")
# the two forms: (precision, ID tolerance, GMRES tolerance)
# (10x below the 1e-10 target: the double-float residual decides it)
FORMS = {"mixed": ("MIXED", 1e-6, 1e-11), "fp64": ("FP64", None, None)}
# The mixed form's ID tolerance sets only how good a preconditioner the
# factorization is (GMRES reaches gmres_tol either way): per workload, the
# value that minimised factor + solve time in a sweep (star16: 1 GMRES
# iteration at 4e-7, 2 at 1e-6; quad64 and star256: 2 iterations at 3e-7,
# 3 at 1e-6, each costing an O(N^2) operator apply).
MIXED_ID_TOL = {"star16": 4e-7, "quad64": 3e-7, "star256": 3e-7}


def _id_tol(wl, form):
    if form == "mixed":
        return MIXED_ID_TOL.get(wl.name, FORMS["mixed"][1])
    return wl.id_tol


_T0 = time.perf_counter()


def _log(msg):
    """Progress with elapsed wall time, on stderr (the JSON line stays the
    only stdout output)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}",
          file=sys.stderr, flush=True)


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _rank():
    return _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), \
        _env_int("LOCAL_RANK", 0)


def _peaks(skel):
    """HBM copy bandwidth and bf16 GEMM rate from MEASURED_PEAKS.json (the
    pool's measurement; the fallback figures otherwise), and the FP64 and
    FP32 FMA rates measured here by the library's probe kernel."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk, kind = json.load(fh), "measured"
    except OSError:
        pk, kind = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                    "sm_max_mhz": 2070.0}, "fallback"
    alu = skel.measure_alu_peaks()
    return {"hbm_gbs": pk["hbm_gbs"], "hbm_source": f"{kind} copy bandwidth",
            "fp64_tflops": alu["fp64_tflops"],
            "fp32_tflops": alu["fp32_tflops"],
            "alu_source": ("measured in this run: FMA chains on every SM "
                           "(skel_measure_alu_peaks)")}


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        fd, self.path = tempfile.mkstemp(prefix=f"skel_clocks_{gpu_index}_",
                                         suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the GPU arm

def _dev_inputs(wl, device):
    import torch
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device=device)
    g = type("DevGeom", (), {})()
    for f in ("x", "y", "dx", "dy", "ddx", "ddy", "dt", "centers"):
        setattr(g, f, t(getattr(wl, f)))
    g.comp = t(wl.comp, torch.int32)
    return g, t(wl.src_xy), t(wl.src_f), t(wl.targets[:, 0].copy()), \
        t(wl.targets[:, 1].copy())


def _pinned_inputs(wl):
    import torch
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt).pin_memory()
    g = type("HostGeom", (), {})()
    for f in ("x", "y", "dx", "dy", "ddx", "ddy", "dt", "centers"):
        setattr(g, f, t(getattr(wl, f)))
    g.comp = t(wl.comp, torch.int32)
    return g, t(wl.src_xy), t(wl.src_f), t(wl.targets[:, 0].copy()), \
        t(wl.targets[:, 1].copy())


def _solver(skel, geom, wl, timing, form):
    prec, id_tol, gtol = FORMS[form]
    kw = {}
    if gtol is not None:
        kw = dict(gmres_tol=gtol, gmres_maxit=60)
    s = skel.Solver(geom, leaf_size=wl.leaf_size, n_proxy=wl.n_proxy,
                    proxy_ratio=wl.proxy_ratio,
                    id_tol=_id_tol(wl, form),
                    precision=getattr(skel, prec), **kw)
    if timing:
        s.set_timing(True)
    return s


def _step(skel, wl, inputs, form, timing=False, like=None):
    geom, sxy, sf, tx, ty = inputs
    s = _solver(skel, geom, wl, timing, form)
    s.factor()
    f = s.point_force_rhs(sxy, sf, holes_zero=wl.rhs_holes_zero, like=like)
    sol = s.solve(f)
    u = s.eval_velocity(sol, tx, ty)
    return s, f, sol, u


def _merge_kernels(acc, ks):
    for name, k in ks.items():
        a = acc.setdefault(name, {"launches": 0, "ms": 0.0, "flops": 0.0,
                                  "bytes": 0.0})
        for key in a:
            a[key] += k[key]


# the unit that bounds each kernel group, per form: "fp64" / "fp32" ALU
# pipes (measured FMA peaks), "hbm" (measured copy bandwidth).  The Gram
# product has no entry: it skips the zero rows of its operand, so the
# dense product's count would overstate its work.
_BOUND = {
    "fp64": {"matvec": "fp64", "cpqr": "fp64", "eliminate": "fp64",
             "top_lu": "fp64", "assemble_id": "fp64", "assemble_diag": "fp64",
             "eval_velocity": "fp64", "matvec_df": "fp32",
             "shape_gradient": "fp64", "solve_up": "hbm",
             "solve_down": "hbm"},
    "mixed": {"matvec": "fp64", "cpqr": "fp32", "eliminate": "fp64",
              "top_lu": "fp64", "assemble_id": "fp32",
              "assemble_diag": "fp64",
              "eval_velocity": "fp64", "matvec_df": "fp32",
              "shape_gradient": "fp64", "solve_up": "hbm",
              "solve_down": "hbm"},
}
# operations the pair-sum kernels issue per ordered source-target pair,
# against the 30 algorithmic flops counted per pair: FP64 instructions of
# the symmetric FP64 operator, FP32 operations of the double-float one
_ISSUED_PER_PAIR = {"matvec": ("fp64", 11.5), "matvec_df": ("fp32", 97.0)}
# DRAM bytes per launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the kernel behind a category, valid while its
# source file hashes to the captured one: {category: (source, sha256[:16],
# bytes per launch, kernel name)}
_TRAFFIC = {
    # k_dl_sym, one launch on the full 32768-node, 16-hole case
    "matvec": ("k_geom.cu", "fe0662a30d67eefc", 2200832 + 6933248,
               "k_dl_sym"),
    # k_dlf_sym on the full 32768-node, 16-hole case (mean of 3 launches)
    "matvec_df": ("k_dlf.cu", "a6f5e10af4823001",
                  (8745216 + 6520064 + 6284544) / 3.0, "k_dlf_sym"),
}


# counters of an ncu capture of the kernel behind a category (quarter-size
# case of the same workload), valid while its source hashes as captured
_COUNTERS = {
    # k_dlf_sym on the 8192-node (quarter-size) case
    "matvec_df": ("k_dlf.cu", "a6f5e10af4823001",
                  {"issue_active": 0.784, "fma_pipe_active": 0.685},
                  "k_dlf_sym, 8192-node case"),
}


def _src_sha(name):
    import hashlib
    path = os.path.join(ROOT, "paper_2001_11619_gb300", "csrc", name)
    try:
        with open(path, "rb") as fh:
            return hashlib.sha256(fh.read()).hexdigest()[:16]
    except OSError:
        return ""


def _rooflines(kernels, peaks, form):
    """Per kernel group: algorithmic work (counted from the realised box
    sizes, see the kernel table of the design notes) over its device time
    (CUDA events around its launches, on the launching stream), against
    the measured peak of the unit that bounds it."""
    out = {}
    for name, k in kernels.items():
        if k["ms"] <= 0:
            continue
        bound = _BOUND[form].get(name)
        if bound is None or (k["flops"] <= 0 and k["bytes"] <= 0):
            continue
        sec = k["ms"] * 1e-3
        nl = max(k["launches"], 1)
        if bound == "hbm":
            if k["bytes"] <= 0:
                continue
            ach, peak, unit = k["bytes"] / sec / 1e9, peaks["hbm_gbs"], "GB/s"
            work = {"algorithmic_bytes_per_launch": k["bytes"] / nl}
        else:
            if k["flops"] <= 0:
                continue
            peak = peaks[f"{bound}_tflops"]
            ach, unit = k["flops"] / sec / 1e12, "TFLOP/s"
            work = {"algorithmic_flops_per_launch": k["flops"] / nl}
        e = {"bound": "hbm" if bound == "hbm" else "alu", "unit": unit,
             "pipe": bound, "achieved": ach, "peak": peak,
             "frac": ach / peak, "ms": k["ms"], "launches": k["launches"],
             "ms_per_launch": k["ms"] / nl, **work, "traffic": None}
        if name in _ISSUED_PER_PAIR:
            pipe, per_pair = _ISSUED_PER_PAIR[name]
            lane_ops = k["flops"] / 30.0 * per_pair
            # FMA throughput counts 2 flops per lane operation
            e["issue_frac"] = lane_ops / sec / (peaks[f"{pipe}_tflops"] *
                                                1e12 / 2)
            e["issue_note"] = (f"{per_pair} {pipe.upper()} operations "
                               "issued per ordered pair over the pipe's "
                               "measured rate")
        t = _TRAFFIC.get(name)
        if t and _src_sha(t[0]) == t[1]:
            e["traffic"] = t[2]
            e["traffic_kernel"] = t[3]
        c = _COUNTERS.get(name)
        if c and _src_sha(c[0]) == c[1]:
            e["ncu_counters"] = dict(c[2], capture=c[3])
        out[name] = e
    return out


def _oracle_step(factor):
    """One oracle step on the workload's curves at 1/factor of the node
    counts: quadrature, boundary data, skeletonization, solve and the
    velocity at 64 targets (the cpu_baseline leg; runs in a child process
    whose BLAS thread count the parent sets)."""
    import oracle
    import workloads as W
    w = W.WORKLOADS[WORKLOAD]()
    if factor > 1:
        w = W.scaled(w, factor, n_targets=64)
    t0 = time.perf_counter()
    g = oracle.quadrature(w)
    f = oracle.boundary_data(g, w.src_xy, w.src_f, w.rhs_holes_zero)
    fac = oracle.factor(w)
    sol = oracle.solve(fac, f)
    oracle.interior_velocity(g, sol, w.targets[:64, 0], w.targets[:64, 1])
    return {"seconds": time.perf_counter() - t0, "N": w.N,
            "unknowns": w.n_unknowns}


def _oracle_child(factor, threads):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
              "BLIS_NUM_THREADS"):
        env[v] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__),
                        "--oracle-sample", str(factor)], env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {r.stderr[-400:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_baseline(budget_s=12.0):
    """The oracle (unchanged) on bounded samples of the workload (the same
    curves at reduced node counts), each in a child process with its BLAS
    thread count fixed: one thread, and every host core.  The sample of
    each is the largest of 1/2 ... 1/16 of the node counts whose estimated
    time (from a 1/16 probe, scaled linearly in N) fits budget_s."""
    cores = os.cpu_count() or 1
    out = {}
    for threads in (cores, 1):
        probe = _oracle_child(16, threads)
        factor = 16
        for fct in (8, 4, 2):
            if probe["seconds"] * 16 / fct <= budget_s:
                factor = fct
        run = probe if factor == 16 else _oracle_child(factor, threads)
        out[threads] = {
            "value": run["unknowns"] / run["seconds"], "unit": UNIT,
            "cores": threads, "seconds": run["seconds"],
            "sample": (f"{WORKLOAD} curves at 1/{factor} of the node counts "
                       f"({run['N']} nodes, {run['unknowns']} unknowns): "
                       "oracle factor + solve + velocity at 64 targets, "
                       f"numpy/BLAS with {threads} thread(s)")}
    res = dict(out[cores])
    res["kind"] = "oracle"
    res["one_thread"] = out[1]
    return res


def _timed_form(skel, wl, dev, form, args, flush, stream):
    """Warm-up, then exactly args.steps timed steps of one form (CUDA events
    on the launching stream, L2 flushed before each step outside the
    events).  Returns the per-step times, merged kernel stats, the launch
    count and the last step's solver and results."""
    import torch
    for _ in range(args.warmup):
        s, *_ = _step(skel, wl, dev, form, timing=True, like=dev[0].x)
        s.close()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernels = {}
    l0 = skel.kernel_launches()
    last = None
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        last = _step(skel, wl, dev, form, timing=True, like=dev[0].x)
        ev[i][1].record(stream)
        _merge_kernels(kernels, last[0].stats()["kernels"])
        if i < args.steps - 1:
            last[0].close()
    torch.cuda.synchronize()
    launches = skel.kernel_launches() - l0
    return [a.elapsed_time(b) for a, b in ev], kernels, launches, last


# Closed-form fields for the accuracy checks of the timed results (the
# exact solutions the synthetic data are made from; nothing of the solver).

def _stokeslet_velocity(tx, ty, src_xy, src_f):
    """u(x) = sum_s (1/4 pi)(-ln|r| I + r r^T/|r|^2) f_s, r = x - s:
    the velocity of point forces (Stokeslets).  Returns (nt, 2)."""
    import numpy as np
    rx = np.subtract.outer(np.asarray(tx), src_xy[:, 0])
    ry = np.subtract.outer(np.asarray(ty), src_xy[:, 1])
    r2 = rx * rx + ry * ry
    lg = -0.5 * np.log(r2)
    fx, fy = src_f[:, 0], src_f[:, 1]
    rf = (rx * fx + ry * fy) / r2
    ux = (lg * fx + rx * rf).sum(axis=1) / (4 * np.pi)
    uy = (lg * fy + ry * rf).sum(axis=1) / (4 * np.pi)
    return np.stack([ux, uy], axis=1)


def _accuracy(wl, s, f, sol, u):
    """Relative residual with the library's FP64 operator and the velocity
    error against the exact point-force field, per right-hand side (the
    largest)."""
    import numpy as np
    import torch
    r = s.matvec(sol)
    rel_res = float(torch.linalg.norm(r - f) / torch.linalg.norm(f))
    uu = u.cpu().numpy()
    err = 0.0
    for c in range(uu.shape[2]):
        ue = _stokeslet_velocity(wl.targets[:, 0], wl.targets[:, 1],
                                 wl.src_xy[c], wl.src_f[c])
        err = max(err, float(np.abs(uu[:, :, c] - ue).max() /
                             np.abs(ue).max()))
    return {"rel_residual_fp64_operator": rel_res,
            "velocity_max_rel_err_vs_exact": err}


def _events_ms(stream, fn):
    """fn() bracketed by CUDA events on the launching stream (synchronised
    on both sides); returns (ms, fn's result)."""
    import torch
    a, b = torch.cuda.Event(True), torch.cuda.Event(True)
    torch.cuda.synchronize()
    a.record(stream)
    out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), out


def _update_leg(skel, W, wl, device, stream, form, n_moves, nrhs,
                solve_every, id_tol=None, seed=77, n_targets=256):
    """Moved-hole updates as in the paper's repositioning runs (Sec. 2.8,
    Sec. 4.3 Table 1): factor once, then n_moves times translate a random
    hole by 0.05 x its radius, update the factorization, and (every
    solve_every-th step and the last) solve nrhs point-force right-hand
    sides of the moved geometry.  Each update and each solve is timed
    alone with CUDA events.  At the end, the last solution's accuracy and a
    fresh factorization of the final geometry, which must give the same
    solution bit for bit."""
    import numpy as np
    import torch
    geom = _dev_inputs(wl, device)[0]
    prec, tol, gtol = FORMS[form]
    kw = dict(leaf_size=wl.leaf_size, n_proxy=wl.n_proxy,
              proxy_ratio=wl.proxy_ratio, precision=getattr(skel, prec),
              id_tol=id_tol or _id_tol(wl, form))
    if gtol is not None:
        kw.update(gmres_tol=gtol, gmres_maxit=80)
    s = skel.Solver(geom, **kw)
    t_fac, _ = _events_ms(stream, s.factor)
    _log(f"  {wl.name} {form}: factor {t_fac:.0f} ms")
    sxy, sf = wl.src_xy[:nrhs], wl.src_f[:nrhs]
    cur = wl
    upd, sol_ms, dirty, iters = [], [], [], []
    moves = W.random_moves(wl, n_moves, seed=seed)
    _log(f"  {len(moves)} moves drawn")
    x = f = None
    for step, (h, d) in enumerate(moves):
        cur = W.move_hole(cur, h, d)
        g = _dev_inputs(cur, device)[0]
        sl = cur.node_slice(h)
        ids = torch.arange(sl.start, sl.stop, device=device)
        ms, _ = _events_ms(stream, lambda: s.update_moved_nodes(ids, g))
        upd.append(ms)
        st = s.stats()
        dirty.append(st["last_dirty"] / max(st["last_boxes"], 1))
        if step % solve_every == solve_every - 1 or step == len(moves) - 1:
            f = s.point_force_rhs(sxy, sf, like=g.x)
            ms, x = _events_ms(stream, lambda: s.solve(f))
            sol_ms.append(ms)
            iters.append(s.stats().get("gmres_iters", 0))
    # accuracy of the last solution: the residual of its first columns
    # (the O(N^2) FP64 operator takes 21 s per column at a million nodes,
    # so above 200000 nodes the double-float one, 2e-13 from it, is used)
    # and every column's velocity against the exact field
    tx = torch.tensor(cur.targets[:n_targets, 0].copy(), device=device)
    ty = torch.tensor(cur.targets[:n_targets, 1].copy(), device=device)
    u = s.eval_velocity(x, tx, ty).cpu().numpy()
    ncheck = min(nrhs, 2)
    big = wl.N > 200000
    xc = x[:, :ncheck]
    r = (s.matvec_df(xc) if big else s.matvec(xc)) - f[:, :ncheck]
    res = float((torch.linalg.norm(r, dim=0) /
                 torch.linalg.norm(f[:, :ncheck], dim=0)).max())
    verr = 0.0
    for c in range(nrhs):
        ue = _stokeslet_velocity(cur.targets[:n_targets, 0],
                                 cur.targets[:n_targets, 1], sxy[c], sf[c])
        verr = max(verr, float(np.abs(u[:, :, c] - ue).max() /
                               np.abs(ue).max()))
    s.close()
    _log(f"  updates done ({statistics.mean(upd):.0f} ms mean), "
         f"solves {statistics.mean(sol_ms):.0f} ms")
    fresh = skel.Solver(_dev_inputs(cur, device)[0], **kw)
    t_fresh, _ = _events_ms(stream, fresh.factor)
    same = bool(torch.equal(fresh.solve(f), x))
    fresh.close()
    return {"moves": len(upd), "nodes_per_hole": int(wl.counts[1]),
            "ms_per_moved_hole_mean": statistics.mean(upd),
            "ms_per_moved_hole_std": statistics.pstdev(upd),
            "ms_first_update": upd[0], "ms_last_update": upd[-1],
            "boxes_recomputed_frac_mean": statistics.mean(dirty),
            "factor_ms": t_fac, "fresh_factor_ms_final_geometry": t_fresh,
            "update_over_factor": statistics.mean(upd) / t_fac,
            "nrhs": nrhs, "solves_timed": len(sol_ms),
            "solve_ms_mean": statistics.mean(sol_ms),
            "gmres_iters_max": max(iters),
            "rel_residual": res,
            "residual_operator": (f"{'double-float' if big else 'fp64'}, "
                                  f"first {ncheck} column(s)"),
            "velocity_max_rel_err_vs_exact": verr,
            "update_equals_fresh_bitwise": same,
            "id_tol": kw["id_tol"], "gmres_tol": gtol}


def _scale_leg(skel, W, device, stream, args):
    """The 1M-node, 256-hole workload: both forms factor, solve (32
    right-hand sides in the FP64 form; the mixed form's GMRES solves one
    column at a time, so one column is timed) and update moved holes."""
    wl = W.star256()
    out = {"workload": ("star256: star 1+0.1cos9t with 256 seeded ellipses "
                        "(semi-axes U[0.015,0.04]), 786432+256x1024 = "
                        "1048576 nodes, 2097920 unknowns"),
           "unknowns": wl.n_unknowns}
    for form, nrhs in (("fp64", 32), ("mixed", 1)):
        _log(f"scale_c5 {form}")
        r = _update_leg(skel, W, wl, device, stream, form, args.c5_updates,
                        nrhs, max(args.c5_updates, 1), n_targets=64)
        r["unknowns_per_s_factor_plus_solve"] = wl.n_unknowns / (
            (r["factor_ms"] + r["solve_ms_mean"]) * 1e-3)
        out[form] = r
    out["mixed_over_fp64_factor_plus_solve"] = (
        out["mixed"]["unknowns_per_s_factor_plus_solve"] /
        out["fp64"]["unknowns_per_s_factor_plus_solve"])
    out["note"] = ("factor_plus_solve counts one solve of the form's nrhs "
                   "(FP64: 32 columns, mixed: 1 column)")
    return out


def _update_c3_leg(skel, W, device, stream, args):
    """The 131072-node, 64 clustered-hole workload: 100 moved holes in both
    forms, 8 right-hand sides per solve (Table 1's protocol)."""
    wl = W.quad64()
    out = {"workload": ("quad64: unit circle with 64 seeded ellipses in the "
                        "quadrant x,y>0 (semi-axes U[0.02,0.04]), "
                        "98304+64x512 = 131072 nodes, leaves of 128, "
                        "262336 unknowns"), "unknowns": wl.n_unknowns}
    for form, every in (("fp64", 1), ("mixed", 10)):
        _log(f"update_c3 {form}")
        r = _update_leg(skel, W, wl, device, stream, form, args.c3_moves, 8,
                        every)
        r["unknowns_per_s_factor_plus_solve"] = wl.n_unknowns / (
            (r["factor_ms"] + r["solve_ms_mean"]) * 1e-3)
        out[form] = r
    out["mixed_over_fp64_update"] = (out["fp64"]["ms_per_moved_hole_mean"] /
                                     out["mixed"]["ms_per_moved_hole_mean"])
    out["mixed_over_fp64_factor_plus_solve"] = (
        out["mixed"]["unknowns_per_s_factor_plus_solve"] /
        out["fp64"]["unknowns_per_s_factor_plus_solve"])
    return out


def _shape_gradient_timing(skel, W, device, stream, steps):
    """The differentiation path on the 16384-node, 8 Fourier-hole geometry
    (no-slip holes, 1024 interior targets): J = sum |u|^2 and dJ/d(samples,
    centres) by the adjoint method, against one objective evaluation (the
    paper's shape optimisation differences J four times per parameter)."""
    import torch
    wl = W.fourier8()
    geom = _dev_inputs(wl, device)
    tx, ty = geom[3], geom[4]

    def run(grad, mixed=False):
        kw = (dict(precision=skel.MIXED, id_tol=1e-6, gmres_tol=1e-12,
                   gmres_maxit=60) if mixed else dict(id_tol=wl.id_tol))
        s = skel.Solver(geom[0], leaf_size=wl.leaf_size, n_proxy=wl.n_proxy,
                        proxy_ratio=wl.proxy_ratio, **kw)
        s.set_timing(True)
        s.factor()
        f = s.point_force_rhs(wl.src_xy, wl.src_f, holes_zero=True,
                              like=geom[0].x)
        if grad:
            out = s.velocity_energy_gradient(f, tx, ty)
        else:
            sol = s.solve(f)
            u = s.eval_velocity(sol, tx, ty)
            out = float((u * u).sum())
        k = s.stats()["kernels"]
        s.close()
        return out, k

    for _ in range(2):
        run(True)
        run(False)
    t_grad, t_J, kern = [], [], {}
    for _ in range(steps):
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize()
        a.record(stream)
        (J, _, g), k = run(True)
        b.record(stream)
        torch.cuda.synchronize()
        t_grad.append(a.elapsed_time(b))
        _merge_kernels(kern, k)
        a.record(stream)
        run(False)
        b.record(stream)
        torch.cuda.synchronize()
        t_J.append(a.elapsed_time(b))
    gk = kern.get("shape_gradient", {"ms": 0.0, "launches": 0})
    n_params = 10 * wl.p
    mg, mj = statistics.mean(t_grad), statistics.mean(t_J)
    # the same gradient in the mixed form (FP32 IDs preconditioning GMRES,
    # forward and adjoint), and its distance to the FP64 one
    import numpy as np
    run(True, True)
    t_mix = []
    for _ in range(steps):
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize()
        a.record(stream)
        (Jm, _, gm), _k = run(True, True)
        b.record(stream)
        torch.cuda.synchronize()
        t_mix.append(a.elapsed_time(b))
    flat = lambda d: np.concatenate([np.asarray(
        d[k].cpu() if hasattr(d[k], "cpu") else d[k]).ravel()
        for k in sorted(d)])
    g64, gmx = flat(g), flat(gm)
    mixed = {"ms_value_and_gradient": statistics.mean(t_mix),
             "gradient_rel_diff_vs_fp64":
                 float(np.linalg.norm(gmx - g64) / np.linalg.norm(g64)),
             "J_rel_diff_vs_fp64": abs(Jm - J) / abs(J)}
    return {"workload": ("fourier8: star 1+0.2cos5t with 8 holes of 8 "
                         "Fourier radius modes + centre (80 parameters), "
                         "12288+8x512 = 16384 nodes, no-slip holes, 1024 "
                         "targets"),
            "ms_value_and_gradient": mg, "ms_value_only": mj,
            "ms_shape_derivative_kernels": gk["ms"] / steps,
            "fd4_equivalent_ms": 4 * n_params * mj,
            "adjoint_over_fd4_speedup": 4 * n_params * mj / mg,
            "J": J, "mixed": mixed}


def _log_potential(tx, ty, src, q):
    """u = sum_k q_k log|x - s_k|: harmonic away from the sources."""
    import numpy as np
    return sum(qk * np.log(np.hypot(tx - sx, ty - sy))
               for (sx, sy), qk in zip(src, q))


def _log_flux(x, y, nx, ny, src, q):
    """n . grad u on the nodes for u of _log_potential."""
    out = 0.0
    for (sx, sy), qk in zip(src, q):
        rx, ry = x - sx, y - sy
        out = out + qk * (rx * nx + ry * ny) / (rx * rx + ry * ry)
    return out


def _laplace_timing(skel, W, device, stream, steps):
    """The Laplace Neumann variant (Sec. 4.4.1) at the paper's 16384 nodes:
    factor + solve with the paper's flux data, in unknowns/s, and the error
    of a closed-form harmonic field recovered from its flux."""
    import numpy as np
    import torch
    wl = W.heat2()
    geom = _dev_inputs(wl, device)[0]
    f = torch.tensor(W.heat_flux(wl), device=device)

    def step():
        s = skel.Solver(geom, leaf_size=wl.leaf_size, id_tol=1e-12,
                        kernel=skel.LAPLACE)
        s.factor()
        mu = s.solve(f)
        return s, mu

    for _ in range(2):
        step()[0].close()
    times = []
    for _ in range(steps):
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize()
        a.record(stream)
        s, mu = step()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        st = s.stats()
        s.close()
    # unit normals out of the domain from the curve samples
    sp = np.hypot(wl.dx, wl.dy)
    nx, ny = wl.dy / sp, -wl.dx / sp
    src = np.array([[2.1, 0.4], [-1.7, -1.6], list(wl.centers[0]),
                    list(wl.centers[1])])
    q = np.array([0.8, -1.1, 0.6, -0.4])
    fh = torch.tensor(0.7 * nx - 0.3 * ny + _log_flux(wl.x, wl.y, nx, ny,
                                                      src, q),
                      device=device)
    s, _ = step()
    mu = s.solve(fh)
    tx, ty = wl.targets[:, 0], wl.targets[:, 1]
    u = s.eval_potential(mu, tx, ty)[:, 0].cpu().numpy()
    s.close()
    ue = 0.7 * tx - 0.3 * ty + _log_potential(tx, ty, src, q)
    err = float(np.abs((u - u[0]) - (ue - ue[0])).max() /
                np.abs(ue - ue[0]).max())
    ms = statistics.mean(times)
    return {"workload": ("heat2: star 1+0.2cos5t with two starfish holes "
                         "16% its size, 10924+2x2730 = 16384 nodes, flux "
                         "0 / +1 / -1 (Sec. 4.4.1)"),
            "unknowns": wl.N, "ms_factor_and_solve": ms,
            "unknowns_per_s": wl.N / (ms * 1e-3),
            "factor_ms": st["t_factor_ms"], "root_skeleton":
                st["root_skeleton"],
            "harmonic_field_error": err}


def run_gpu(args):
    import torch
    import workloads as W
    import paper_2001_11619_gb300 as skel

    rank, world, local = _rank()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    device = torch.device("cuda", local)
    _log("start")
    wl = W.WORKLOADS[WORKLOAD]()
    if args.scale > 1:   # smaller case of the same curves (profiling only)
        wl = W.scaled(wl, args.scale)
    dev = _dev_inputs(wl, device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32,
                        device=device)
    stream = torch.cuda.current_stream()
    forms = ["mixed", "fp64"] if args.form == "both" else [args.form]
    head = forms[0]

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    res = {}
    t0 = time.perf_counter()
    for form in forms:
        res[form] = _timed_form(skel, wl, dev, form, args, flush, stream)
        if form == head:
            wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()

    per_form = {}
    for form in forms:
        step_ms, kernels, launches, (s, f, sol, u) = res[form]
        mean_ms = sum(step_ms) / len(step_ms)
        if dist:
            t = torch.tensor([mean_ms], device=device, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            mean_ms = float(t.item())
        st = s.stats()
        acc = _accuracy(wl, s, f, sol, u)
        s.close()
        per_form[form] = {
            "value": world * wl.n_unknowns / (mean_ms * 1e-3),
            "ms_per_step": mean_ms, "step_ms": step_ms,
            "kernels": kernels, "launches": launches, "accuracy": acc,
            "factor": {"ms": st["t_factor_ms"], "levels": st["levels"],
                       "root_skeleton": st["root_skeleton"],
                       "per_level": st["per_level"]},
            "solve": {"ms": st["t_solve_ms"],
                      "gmres_iters": st.get("gmres_iters", 0),
                      "gmres_relres": st.get("gmres_relres", 0.0)},
            "id_tol": _id_tol(wl, form),
            "gmres_tol": FORMS[form][2]}

    # e2e: the headline step through host (pinned) buffers
    host = _pinned_inputs(wl)
    e2e_ms = []
    for i in range(0 if args.no_e2e else max(2, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s2, f2, sol2, u2 = _step(skel, wl, host, head, timing=False,
                                 like=None)
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
        s2.close()
    ldf = wl.n_unknowns
    h2d = (7 * wl.N * 8 + 4 * wl.N + 16 * wl.p + 2 * wl.src_xy.size * 8
           + 2 * ldf * 8 + 2 * wl.targets.shape[0] * 8)
    d2h = 2 * ldf * 8 + 2 * wl.targets.shape[0] * 8
    e2e_mean = sum(e2e_ms) / len(e2e_ms) if e2e_ms else float("nan")

    # The legs after the headline step are reported in the line; one that
    # raises is reported as {"error": ...} in its place, so the measured
    # headline is not lost with it.
    def leg(name, fn):
        try:
            return fn()
        except Exception as e:  # noqa: BLE001 (recorded in the output)
            _log(f"{name} failed: {type(e).__name__}: {e}")
            return {"error": f"{type(e).__name__}: {e}"}

    # moved-hole updates on the headline geometry (quick look, both forms)
    if args.updates > 0:
        for form in forms:
            per_form[form]["update"] = leg(
                f"update {form}",
                lambda form=form: _update_leg(skel, W, wl, device, stream,
                                              form, args.updates, 1, 1))

    _log("headline forms and updates done")
    legs = {}
    if args.c3_moves > 0:
        legs["update_c3"] = leg("update_c3", lambda: _update_c3_leg(
            skel, W, device, stream, args))
        _log("update_c3 leg done")
    if args.c5_updates > 0:
        legs["scale_c5"] = leg("scale_c5", lambda: _scale_leg(
            skel, W, device, stream, args))
        _log("scale_c5 leg done")

    grad = {}
    if not args.no_grad:
        grad = leg("shape_gradient", lambda: _shape_gradient_timing(
            skel, W, device, stream, max(2, min(args.steps, 3))))

    lap = {}
    if not args.no_grad:
        lap = leg("laplace", lambda: _laplace_timing(
            skel, W, device, stream, max(2, min(args.steps, 3))))
    _log("gradient and Laplace timings done")

    peaks = _peaks(skel)
    out = None
    if rank == 0:
        H = per_form[head]
        kernels = H["kernels"]
        tot = sum(k["ms"] for k in kernels.values())
        roofs = _rooflines(kernels, peaks, head)
        # the dominant kernel group of the headline step
        top = max(roofs, key=lambda n: roofs[n]["ms"])
        roof = dict(roofs[top])
        roof["kernel"] = top
        roof["peak_source"] = (peaks["hbm_source"] if roof["bound"] == "hbm"
                               else peaks["alu_source"])
        kern = {n: {"launches_per_step": k["launches"] / args.steps,
                    "ms_per_step": k["ms"] / args.steps,
                    "share": k["ms"] / tot if tot else None}
                for n, k in sorted(kernels.items(),
                                   key=lambda kv: -kv[1]["ms"])}
        forms_out = {}
        for form in forms:
            F = per_form[form]
            forms_out[form] = {k: F[k] for k in
                               ("value", "ms_per_step", "step_ms",
                                "accuracy", "factor", "solve", "id_tol",
                                "gmres_tol", "launches")}
            forms_out[form]["update"] = F.get("update", {})
            forms_out[form]["kernel_ms_per_step"] = {
                n: k["ms"] / args.steps for n, k in sorted(
                    F["kernels"].items(), key=lambda kv: -kv[1]["ms"])}
            forms_out[form]["rooflines"] = _rooflines(F["kernels"], peaks,
                                                      form)
        out = {
            "metric": METRIC, "value": H["value"], "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": H["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if head == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}",
                       "N": wl.N, "p": wl.p, "unknowns": wl.n_unknowns,
                       "form": head, "id_tol": H["id_tol"],
                       "gmres_tol": H["gmres_tol"],
                       "leaf_size": wl.leaf_size, "n_proxy": wl.n_proxy,
                       "proxy_ratio": wl.proxy_ratio, "step": STEP_DESC,
                       "l2": "flushed between timed steps (256 MiB write "
                             "outside the timed events)",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk,
            "e2e": {"value": world * wl.n_unknowns / (e2e_mean * 1e-3),
                    "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_mean,
                    "how": f"same {head} step through the Python binding "
                           "with pinned host arrays (library copies "
                           "inside)"},
            "gpu_launches": H["launches"],
            "roofline": roof,
            "rooflines": roofs,
            "peaks": peaks,
            "kernels": kern,
            "accuracy": H["accuracy"],
            "update": H.get("update", {}),
            **legs,
            "shape_gradient": grad,
            "laplace": lap,
            "forms": forms_out,
            "wall_s_timed_region": wall,
        }
        if "fp64" in per_form and head != "fp64":
            out["mixed_over_fp64"] = H["value"] / per_form["fp64"]["value"]
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = leg("cpu_baseline", _cpu_baseline)
            _log("cpu baseline done")
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


# ---------------------------------------------------------------------------
# the reference arm: the CPU oracle

def run_reference(args):
    import workloads as W
    rank, world, local = _rank()
    if rank != 0:
        return None
    import oracle
    wl = W.WORKLOADS[WORKLOAD]()
    # each step a sample of the workload sized so that the whole run ends
    # within a few minutes: the largest of 1/2 ... 1/16 of the node counts
    # whose estimated step time (from a 1/16 probe, linear in N) fits
    budget = 150.0 / max(args.steps + args.warmup, 1)
    probe = _oracle_step(16)
    factor = 16
    for fct in (8, 4, 2):
        if probe["seconds"] * 16 / fct <= budget:
            factor = fct
    sample = W.scaled(wl, factor, n_targets=64)
    sample_desc = (f"{WORKLOAD} curves at 1/{factor} of the node counts "
                   f"({sample.N} nodes, {sample.n_unknowns} unknowns): "
                   "oracle factor + solve + velocity at 64 targets, "
                   "numpy/BLAS on all host cores")

    def step():
        g = oracle.quadrature(sample)
        f = oracle.boundary_data(g, sample.src_xy, sample.src_f,
                                 sample.rhs_holes_zero)
        fac = oracle.factor(sample)
        sol = oracle.solve(fac, f)
        oracle.interior_velocity(g, sol, sample.targets[:, 0],
                                 sample.targets[:, 1])

    for _ in range(args.warmup):
        step()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t0)
    mean = sum(ts) / len(ts)
    value = sample.n_unknowns / mean
    out = {"impl": "reference", "metric": METRIC, "value": value,
           "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": mean * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}",
                      "form": "cpu oracle", "step": STEP_DESC},
           "cpu_baseline": {"value": value, "unit": UNIT,
                            "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample_desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def _factor_case(workload, form):
    """One factorization of a named workload in one form, alone (build,
    factor), with its per-kernel times: the case the launch-list profiles
    of the large-box kernels capture."""
    import torch
    import workloads as W
    import paper_2001_11619_gb300 as skel
    wl = W.WORKLOADS[workload]()
    device = torch.device("cuda")
    geom = _dev_inputs(wl, device)[0]
    prec, tol, gtol = FORMS[form]
    kw = dict(leaf_size=wl.leaf_size, precision=getattr(skel, prec),
              id_tol=_id_tol(wl, form))
    s = skel.Solver(geom, **kw)
    s.set_timing(True)
    ms, _ = _events_ms(torch.cuda.current_stream(), s.factor)
    st = s.stats()
    s.close()
    print(json.dumps({"workload": workload, "form": form, "factor_ms": ms,
                      "kernels": {k: v["ms"] for k, v in
                                  st["kernels"].items()}}), flush=True)


def _tc_gemm_case(M, N, K, steps, warmup):
    """The 3xTF32 tensor-core GEMM C -= A B alone on column-major FP64
    operands (skel_gemm_tf32x3), timed with CUDA events."""
    import torch
    import paper_2001_11619_gb300 as skel
    dev = torch.device("cuda")
    A = torch.randn(K, M, dtype=torch.float64, device=dev).t()
    B = torch.randn(N, K, dtype=torch.float64, device=dev).t()
    C = torch.randn(N, M, dtype=torch.float64, device=dev).t()
    for _ in range(warmup):
        skel.gemm_tf32x3(A, B, C)
    ms = []
    for _ in range(steps):
        t, _ = _events_ms(torch.cuda.current_stream(),
                          lambda: skel.gemm_tf32x3(A, B, C))
        ms.append(t)
    m = statistics.mean(ms)
    print(json.dumps({"kernel": "k_tc_gemm", "M": M, "N": N, "K": K,
                      "ms": m, "useful_tflops": 2.0 * M * N * K / m / 1e9,
                      "tf32_mma_tflops": 6.0 * M * N * K / m / 1e9}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--updates", type=int, default=8,
                    help="moved holes on the headline geometry")
    ap.add_argument("--c3-moves", type=int, default=100,
                    help="moved holes on the 131072-node workload (0: skip)")
    ap.add_argument("--c5-updates", type=int, default=10,
                    help="moved holes on the 1M-node workload (0: skip)")
    ap.add_argument("--oracle-sample", type=int, default=0,
                    help=argparse.SUPPRESS)
    ap.add_argument("--tc-gemm", default="",
                    help="M,N,K: time the 3xTF32 tensor-core GEMM alone")
    ap.add_argument("--factor-only", default="",
                    help="WORKLOAD:FORM (e.g. quad64:fp64): one build and "
                         "factorization alone, timed (profiling case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-grad", action="store_true",
                    help="skip the shape-gradient and Laplace timings")
    ap.add_argument("--form", choices=["both", "mixed", "fp64"],
                    default="both",
                    help="forms to time; the first is the headline")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide the node counts (small profiling cases)")
    args = ap.parse_args()
    if args.oracle_sample:   # child process of the cpu_baseline leg
        print(json.dumps(_oracle_step(args.oracle_sample)), flush=True)
        return
    if args.factor_only:
        _factor_case(*args.factor_only.split(":"))
        return
    if args.tc_gemm:
        _tc_gemm_case(*[int(v) for v in args.tc_gemm.split(",")],
                      steps=args.steps, warmup=args.warmup)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
