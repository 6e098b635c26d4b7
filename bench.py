#!/usr/bin/env python
"""Benchmark of the GB300 skeletonization solver.

One step = the whole hot path on one synthetic geometry: build the quadtree
(geometry already resident in HBM), factor the bordered system level by
level, form the boundary data, solve, and evaluate the velocity at the
interior targets.  The workload is the 32768-node, 16-hole star geometry
(65584 unknowns).  The metric is unknowns per second of that step; the
moved-hole update time is reported beside it.

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
FP64_FMA_PER_CLK_PER_SM = 2     # GB300 FP64 units (measured 1.19 TF/s)
SMS = 152


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _rank():
    return _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), \
        _env_int("LOCAL_RANK", 0)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                "sm_max_mhz": 2070.0}, "fallback"


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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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


def _solver(skel, geom, wl, timing):
    s = skel.Solver(geom, leaf_size=wl.leaf_size, n_proxy=wl.n_proxy,
                    proxy_ratio=wl.proxy_ratio, id_tol=wl.id_tol)
    if timing:
        s.set_timing(True)
    return s


def _step(skel, wl, inputs, timing=False, like=None):
    geom, sxy, sf, tx, ty = inputs
    s = _solver(skel, geom, wl, timing)
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


def _roofline(kernels, peaks, peak_kind, clocks):
    factor_kernels = {k: v for k, v in kernels.items() if v["ms"] > 0}
    name = max(factor_kernels, key=lambda k: factor_kernels[k]["ms"])
    k = factor_kernels[name]
    per_launch_ms = k["ms"] / max(k["launches"], 1)
    if name.startswith("solve_") or name == "bordered_sweeps":
        achieved = k["bytes"] / (k["ms"] * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
        return {"kernel": name, "bound": "hbm", "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_source": f"{peak_kind} HBM copy",
                "ms_per_launch": per_launch_ms,
                "algorithmic_bytes_per_launch":
                    k["bytes"] / max(k["launches"], 1)}
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    peak = SMS * FP64_FMA_PER_CLK_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = k["flops"] / (k["ms"] * 1e-3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None,
            "peak_source": ("FP64 ALU: 152 SMs x 2 DFMA/clk x 2 flop x "
                            f"{sm_max:.0f} MHz (derived from unit counts "
                            "and the max SM clock)"),
            "ms_per_launch": per_launch_ms,
            "algorithmic_flops_per_launch":
                k["flops"] / max(k["launches"], 1)}


def _cpu_baseline(wl_full, budget_s=25.0):
    """The oracle (unchanged) on a bounded sample of the workload: the same
    curves at reduced node counts, factor + solve + velocity, timed on the
    host cores."""
    import numpy as np
    import oracle
    import workloads as W

    def run(w):
        t0 = time.perf_counter()
        g = oracle.quadrature(w)
        f = oracle.boundary_data(g, w.src_xy, w.src_f, w.rhs_holes_zero)
        fac = oracle.factor(w)
        sol = oracle.solve(fac, f)
        oracle.interior_velocity(g, sol, w.targets[:64, 0],
                                 w.targets[:64, 1])
        return time.perf_counter() - t0

    probe = W.scaled(wl_full, 16, n_targets=64)
    tp = run(probe)
    factor = 16
    for fct in (8, 4, 2, 1):
        if tp * 16 / fct <= budget_s:
            factor = fct
    sample = W.scaled(wl_full, factor, n_targets=64) if factor != 16 else probe
    dt = run(sample) if factor != 16 else tp
    return {"value": sample.n_unknowns / dt, "unit": UNIT, "factor": factor,
            "cores": os.cpu_count(), "kind": "oracle",
            "seconds": dt,
            "sample": (f"{wl_full.name} curves at 1/{factor} of the node "
                       f"counts ({sample.N} nodes, {sample.n_unknowns} "
                       "unknowns): oracle factor + solve + velocity at 64 "
                       "targets, numpy/BLAS on all host cores")}


def run_gpu(args):
    import numpy as np
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
    wl = W.WORKLOADS[WORKLOAD]()
    if args.scale > 1:   # smaller case of the same curves (profiling only)
        wl = W.scaled(wl, args.scale)
    dev = _dev_inputs(wl, device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32,
                        device=device)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        _step(skel, wl, dev, timing=True, like=dev[0].x)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernels = {}
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    l0 = skel.kernel_launches()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        s, f, sol, u = _step(skel, wl, dev, timing=True, like=dev[0].x)
        ev[i][1].record(stream)
        _merge_kernels(kernels, s.stats()["kernels"])
        if i < args.steps - 1:
            s.close()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = skel.kernel_launches() - l0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    mean_ms = sum(step_ms) / len(step_ms)
    if dist:
        t = torch.tensor([mean_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        mean_ms = float(t.item())
    value = world * wl.n_unknowns / (mean_ms * 1e-3)

    # accuracy of the last step against the operator and the exact field
    r = s.matvec(sol)
    rel_res = float(torch.linalg.norm(r - f) / torch.linalg.norm(f))
    ue = np.zeros((wl.targets.shape[0], 2))
    import oracle  # exact point-force field only (closed form)
    ue = oracle.point_force_velocity(wl.targets[:, 0], wl.targets[:, 1],
                                     wl.src_xy[0], wl.src_f[0])
    u_err = float(np.linalg.norm(u[:, :, 0].cpu().numpy() - ue) /
                  np.linalg.norm(ue))
    st = s.stats()
    s.close()

    # e2e: the same step through host (pinned) buffers
    host = _pinned_inputs(wl)
    e2e_ms = []
    for i in range(0 if args.no_e2e else max(2, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s2, f2, sol2, u2 = _step(skel, wl, host, timing=False, like=None)
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
        s2.close()
    ldf = wl.n_unknowns
    h2d = (7 * wl.N * 8 + 4 * wl.N + 16 * wl.p + 2 * wl.src_xy.size * 8
           + 2 * ldf * 8 + 2 * wl.targets.shape[0] * 8)
    d2h = 2 * ldf * 8 + 2 * wl.targets.shape[0] * 8
    e2e_mean = sum(e2e_ms) / len(e2e_ms) if e2e_ms else float("nan")

    # moved-hole updates (Sec. 2.8): ms per moved hole
    upd = {}
    if args.updates > 0:
        s3 = _solver(skel, dev[0], wl, False)
        s3.factor()
        cur = wl
        moves = W.random_moves(wl, args.updates, seed=77)
        times, dirty = [], []
        for h, d in moves:
            cur = W.move_hole(cur, h, d)
            g3 = _dev_inputs(cur, device)[0]
            sl = cur.node_slice(h)
            ids = torch.arange(sl.start, sl.stop, device=device)
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            torch.cuda.synchronize()
            a.record(stream)
            s3.update_moved_nodes(ids, g3)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
            st3 = s3.stats()
            dirty.append(st3["last_dirty"] / max(st3["last_boxes"], 1))
        upd = {"ms_per_moved_hole_mean": statistics.mean(times),
               "ms_per_moved_hole_std": statistics.pstdev(times),
               "moves": len(times),
               "nodes_per_hole": int(wl.counts[1]),
               "boxes_recomputed_frac_mean": statistics.mean(dirty),
               "factor_ms_same_geometry": s3.stats()["t_factor_ms"]}
        s3.close()

    peaks, peak_kind = _peaks()
    out = None
    if rank == 0:
        tot = sum(k["ms"] for k in kernels.values())
        roof = _roofline(kernels, peaks, peak_kind, clk)
        kern = {n: {"launches_per_step": k["launches"] / args.steps,
                    "ms_per_step": k["ms"] / args.steps,
                    "share": k["ms"] / tot if tot else None}
                for n, k in sorted(kernels.items(),
                                   key=lambda kv: -kv[1]["ms"])}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": mean_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}",
                       "N": wl.N, "p": wl.p, "unknowns": wl.n_unknowns,
                       "form": "fp64", "id_tol": wl.id_tol,
                       "leaf_size": wl.leaf_size, "n_proxy": wl.n_proxy,
                       "proxy_ratio": wl.proxy_ratio, "step": STEP_DESC,
                       "l2": "flushed between timed steps (256 MiB write "
                             "outside the timed events)",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk,
            "e2e": {"value": world * wl.n_unknowns / (e2e_mean * 1e-3),
                    "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_mean,
                    "how": "same step through the Python binding with "
                           "pinned host arrays (library copies inside)"},
            "gpu_launches": launches,
            "roofline": roof,
            "kernels": kern,
            "accuracy": {"rel_residual_fp64_operator": rel_res,
                         "velocity_rel_err_vs_exact": u_err},
            "update": upd,
            "factor": {"ms": st["t_factor_ms"], "levels": st["levels"],
                       "root_skeleton": st["root_skeleton"],
                       "per_level": st["per_level"]},
            "wall_s_timed_region": wall,
        }
        if world == 1 and not args.no_cpu_baseline:
            cb = _cpu_baseline(wl)
            cb.pop("factor")
            out["cpu_baseline"] = cb
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
    budget = 150.0 / max(args.steps + args.warmup, 1)
    base = _cpu_baseline(wl, budget_s=budget)
    sample = W.scaled(wl, base["factor"], n_targets=64)

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
                            "sample": base["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--updates", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide the node counts (small profiling cases)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
