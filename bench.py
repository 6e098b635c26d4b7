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
FORMS = {"mixed": ("MIXED", 1e-6, 1e-12), "fp64": ("FP64", None, None)}
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


def _solver(skel, geom, wl, timing, form):
    prec, id_tol, gtol = FORMS[form]
    kw = {}
    if gtol is not None:
        kw = dict(gmres_tol=gtol, gmres_maxit=60)
    s = skel.Solver(geom, leaf_size=wl.leaf_size, n_proxy=wl.n_proxy,
                    proxy_ratio=wl.proxy_ratio,
                    id_tol=id_tol if id_tol is not None else wl.id_tol,
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


# the unit that bounds each kernel group, per form
_PIPE = {
    "fp64": {"matvec": "fp64", "cpqr": "fp64", "eliminate": "fp64",
             "top_lu": "fp64", "assemble_id": "fp64",
             "assemble_diag": "fp64", "gram": "fp64", "eval_velocity": "fp64",
             "matvec_df": "fp32"},
    "mixed": {"matvec": "fp64", "cpqr": "fp32", "eliminate": "fp64",
              "top_lu": "fp64", "assemble_id": "fp32",
              "assemble_diag": "fp64", "gram": "fp64",
              "eval_velocity": "fp64", "matvec_df": "fp32"},
}
# lanes per SM per clock: FP64 DFMA (2, measured) and FP32 FFMA (128)
_LANES = {"fp64": FP64_FMA_PER_CLK_PER_SM, "fp32": 128}


# ncu capture of one full-size k_dl_sym launch (32768 nodes): DRAM read
# 2200832 + write 6933248 bytes, for this hash of k_geom.cu
_TRAFFIC_K_GEOM_SHA = "fe0662a30d67eefc"
_TRAFFIC_DL_SYM = 2200832 + 6933248


def _roofline(kernels, peaks, peak_kind, clocks, form):
    timed_k = {k: v for k, v in kernels.items() if v["ms"] > 0}
    name = max(timed_k, key=lambda k: timed_k[k]["ms"])
    k = timed_k[name]
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
    pipe = _PIPE[form].get(name, "fp64")
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    peak = SMS * _LANES[pipe] * 2 * sm_max * 1e6 / 1e12
    achieved = k["flops"] / (k["ms"] * 1e-3) / 1e12
    extra = {}
    if name == "matvec":
        # DRAM bytes of one k_dl_sym launch from a full-size ncu capture,
        # valid while the kernel source is the captured one
        import hashlib
        src = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                           "paper_2001_11619_gb300", "csrc", "k_geom.cu")
        try:
            with open(src, "rb") as fh:
                h = hashlib.sha256(fh.read()).hexdigest()[:16]
        except OSError:
            h = ""
        if h == _TRAFFIC_K_GEOM_SHA:
            extra["traffic_bytes_per_kernel_launch"] = _TRAFFIC_DL_SYM
            extra["traffic_source"] = (
                "profiles/k_dl_sym_star16_full_traffic.md (ncu dram__bytes_"
                "read.sum + dram__bytes_write.sum, one k_dl_sym launch)")
        # the symmetric pair sums issue 11.5 FP64 instructions per ordered
        # pair (flops are counted at 30 per pair)
        issued = 11.5 * k["flops"] / 30.0
        extra["fp64_issue_frac"] = issued / (k["ms"] * 1e-3) / (
            SMS * _LANES["fp64"] * sm_max * 1e6)
    return {**extra, "kernel": name, "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": extra.get("traffic_bytes_per_kernel_launch"),
            "pipe": pipe,
            "peak_source": (f"{pipe.upper()} ALU: 152 SMs x "
                            f"{_LANES[pipe]} FMA lanes/clk x 2 flop x "
                            f"{sm_max:.0f} MHz (derived from unit counts "
                            "and the max SM clock)"),
            "flops_note": ("algorithmic FP64-equivalent flops from the "
                           "realised box sizes (see the kernel table)"),
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


def _accuracy(wl, s, f, sol, u):
    import numpy as np
    import torch
    import oracle  # exact point-force field only (closed form)
    r = s.matvec(sol)
    rel_res = float(torch.linalg.norm(r - f) / torch.linalg.norm(f))
    ue = oracle.point_force_velocity(wl.targets[:, 0], wl.targets[:, 1],
                                     wl.src_xy[0], wl.src_f[0])
    u_err = float(np.linalg.norm(u[:, :, 0].cpu().numpy() - ue) /
                  np.linalg.norm(ue))
    return {"rel_residual_fp64_operator": rel_res,
            "velocity_rel_err_vs_exact": u_err}


def _updates(skel, W, wl, dev_geom, device, stream, form, n):
    """Moved-hole updates (Sec. 2.8): ms per moved hole."""
    import torch
    s3 = _solver(skel, dev_geom, wl, False, form)
    s3.factor()
    cur = wl
    times, dirty = [], []
    for h, d in W.random_moves(wl, n, seed=77):
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
    out = {"ms_per_moved_hole_mean": statistics.mean(times),
           "ms_per_moved_hole_std": statistics.pstdev(times),
           "moves": len(times), "nodes_per_hole": int(wl.counts[1]),
           "boxes_recomputed_frac_mean": statistics.mean(dirty),
           "factor_ms_same_geometry": s3.stats()["t_factor_ms"]}
    s3.close()
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


def _laplace_timing(skel, W, device, stream, steps):
    """The Laplace Neumann variant (Sec. 4.4.1) at the paper's 16384 nodes:
    factor + solve with the paper's flux data, in unknowns/s, and the error
    of a closed-form harmonic field recovered from its flux."""
    import numpy as np
    import torch
    import oracle.laplace as L  # closed-form field and its flux only
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
    g = L.quadrature(wl)
    src = np.array([[2.1, 0.4], [-1.7, -1.6], list(wl.centers[0]),
                    list(wl.centers[1])])
    q = np.array([0.8, -1.1, 0.6, -0.4])
    fh = torch.tensor(0.7 * g.nx - 0.3 * g.ny + L.source_flux(g, src, q),
                      device=device)
    s, _ = step()
    mu = s.solve(fh)
    tx, ty = wl.targets[:, 0], wl.targets[:, 1]
    u = s.eval_potential(mu, tx, ty)[:, 0].cpu().numpy()
    s.close()
    ue = 0.7 * tx - 0.3 * ty + L.source_potential(tx, ty, src, q)
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
            "id_tol": FORMS[form][1] or wl.id_tol,
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

    if args.updates > 0:
        for form in forms:
            per_form[form]["update"] = _updates(skel, W, wl, dev[0], device,
                                                stream, form, args.updates)

    grad = {}
    if not args.no_grad:
        grad = _shape_gradient_timing(skel, W, device, stream,
                                      max(2, min(args.steps, 3)))

    lap = {}
    if not args.no_grad:
        lap = _laplace_timing(skel, W, device, stream,
                              max(2, min(args.steps, 3)))

    peaks, peak_kind = _peaks()
    out = None
    if rank == 0:
        H = per_form[head]
        kernels = H["kernels"]
        tot = sum(k["ms"] for k in kernels.values())
        roof = _roofline(kernels, peaks, peak_kind, clk, head)
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
            "kernels": kern,
            "accuracy": H["accuracy"],
            "update": H.get("update", {}),
            "shape_gradient": grad,
            "laplace": lap,
            "forms": forms_out,
            "wall_s_timed_region": wall,
        }
        if "fp64" in per_form and head != "fp64":
            out["mixed_over_fp64"] = H["value"] / per_form["fp64"]["value"]
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
    ap.add_argument("--no-grad", action="store_true",
                    help="skip the shape-gradient and Laplace timings")
    ap.add_argument("--form", choices=["both", "mixed", "fp64"],
                    default="both",
                    help="forms to time; the first is the headline")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide the node counts (small profiling cases)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
