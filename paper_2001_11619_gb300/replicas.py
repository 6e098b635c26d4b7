"""Independent replicas, one process per GPU.

The paper does not split one factorization over processors.  It runs
independent updates side by side, one per processor, for example the
finite-difference probes and line-search trials of its shape optimisation
(Sec. 4.4, allocation schemes A-C).  This module does that over
``torch.distributed`` ranks.

- Each rank evaluates its share of a batch of independent tasks, assigned
  round-robin.
- The per-task results (a few floats each) are gathered once per batch.
- No step of a factorization, update or solve crosses ranks, so the data
  path has no collective.
- The gather doubles as the failure check.  A task that raises on any rank
  makes every rank raise :class:`ReplicaError` naming that rank, instead
  of leaving the other ranks waiting.

The module is plain host logic.  The GPU work happens inside the
``evaluate`` callables, for example :func:`moved_hole_objective`, which
runs an update, a solve and a velocity evaluation through
:class:`paper_2001_11619_gb300.Solver` on the rank's own GPU.
"""
from __future__ import annotations

import numpy as np


class ReplicaError(RuntimeError):
    """A task failed on some rank; raised on every rank of the batch."""


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def world():
    """(rank, number of ranks) of the default process group, (0, 1) when
    none is initialised."""
    d = _dist()
    return (d.get_rank(), d.get_world_size()) if d else (0, 1)


def shard(n_tasks, rank, size):
    """Indices of the tasks a rank evaluates: round-robin, so consecutive
    tasks (e.g. the two sides of one central difference) land on
    different ranks and every rank gets n_tasks / size of them, +-1."""
    if size < 1 or not 0 <= rank < size:
        raise ValueError("invalid rank / size")
    return list(range(rank, n_tasks, size))


def run_batch(tasks, evaluate, group=None):
    """Evaluate ``evaluate(task)`` for every task, spread over the ranks;
    returns the results in task order on every rank.

    Each rank evaluates its shard and stops at its first failing task.
    One ``all_gather_object`` then exchanges the results, or the error, of
    every rank.  If any rank failed, all ranks raise :class:`ReplicaError`."""
    d = _dist()
    rank, size = (d.get_rank(group), d.get_world_size(group)) if d else (0, 1)
    local, err = [], None
    for i in shard(len(tasks), rank, size):
        try:
            local.append((i, evaluate(tasks[i])))
        except Exception as e:  # reported to every rank below
            err = f"task {i}: {type(e).__name__}: {e}"
            break
    payload = {"rank": rank, "error": err, "results": local}
    if d is None:
        gathered = [payload]
    else:
        gathered = [None] * size
        d.all_gather_object(gathered, payload, group=group)
    failed = [g for g in gathered if g["error"] is not None]
    if failed:
        raise ReplicaError("; ".join(f"rank {g['rank']}: {g['error']}"
                                     for g in failed))
    out = [None] * len(tasks)
    for g in gathered:
        for i, v in g["results"]:
            out[i] = v
    return out


# central-difference stencils: (offset in units of h, weight)
_STENCIL = {2: ((1, 0.5), (-1, -0.5)),
            4: ((-2, 1.0 / 12), (-1, -8.0 / 12), (1, 8.0 / 12),
                (2, -1.0 / 12))}


def fd_gradient(J, theta, h, order=4, coords=None, group=None):
    """Central-difference gradient of the scalar objective J at theta.

    The paper's optimisation uses fourth-order differences (Sec. 4.3).
    order: 2 or 4.  coords: the coordinates to differentiate (all by
    default).  The len(stencil) x len(coords) evaluations of J are spread
    over the ranks.  The weighted sums run in a fixed order, so the result
    does not depend on the number of ranks."""
    theta = np.asarray(theta, dtype=np.float64)
    st = _STENCIL[order]
    coords = list(range(theta.size)) if coords is None else list(coords)
    tasks = [(k, off) for k in coords for off, _ in st]

    def ev(task):
        k, off = task
        t = theta.copy()
        t.flat[k] += off * h
        return float(J(t))

    vals = run_batch(tasks, ev, group)
    g = np.zeros(len(coords))
    for c in range(len(coords)):
        acc = 0.0
        for s, (_, wgt) in enumerate(st):
            acc += wgt * vals[c * len(st) + s]
        g[c] = acc / h
    return g


def line_search(J, theta, direction, alphas, group=None):
    """J at theta + alpha * direction for every trial step alpha, spread
    over the ranks.  Returns (the alpha with the smallest J, all J values in
    the order of alphas; ties go to the first)."""
    theta = np.asarray(theta, dtype=np.float64)
    direction = np.asarray(direction, dtype=np.float64)
    vals = run_batch(list(alphas),
                     lambda a: float(J(theta + a * direction)), group)
    best = int(np.argmin(vals))
    return list(alphas)[best], vals


def max_over_ranks(x, group=None):
    """Largest value of x over the ranks: a step of a replica batch takes
    as long as its slowest rank."""
    d = _dist()
    if d is None:
        return float(x)
    out = [None] * d.get_world_size(group)
    d.all_gather_object(out, float(x), group=group)
    return max(out)


def moved_hole_objective(solver, workload, targets, to_device, move_hole):
    """Evaluator for hole-move trials on this rank's GPU.

    Returns ``evaluate((hole, dx, dy))``: move hole ``hole`` of
    ``workload`` by (dx, dy) from its original position and refactor only
    the affected boxes (Sec. 2.8).  Then solve for the workload's
    point-force data and return J = sum |u|^2 at the interior targets.

    solver: a factored :class:`Solver` of ``workload``.  Successive trials
    update it from trial to trial; an update reproduces a fresh
    factorization bit for bit, so the order of the trials does not matter.
    targets: (tx, ty) device tensors.  to_device: maps a workload to the
    solver's geometry (device tensors).  move_hole(workload, hole, (dx, dy)):
    the moved workload (same node ids)."""
    import torch

    tx, ty = targets

    def evaluate(task):
        hole, dx, dy = task
        cur = move_hole(workload, hole, (dx, dy))
        sl = cur.node_slice(hole)
        ids = torch.arange(sl.start, sl.stop, device=tx.device)
        solver.update_moved_nodes(ids, to_device(cur))
        f = solver.point_force_rhs(cur.src_xy, cur.src_f, like=tx)
        u = solver.eval_velocity(solver.solve(f), tx, ty)
        return float((u.double() ** 2).sum().item())

    return evaluate
