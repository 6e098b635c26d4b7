"""Seeded synthetic workloads shaped like the paper's Stokes experiments.

The paper's own boundaries are cubic splines through knots it does not list
(Sec. 4, experiments of Sec. 4.2-4.4), so analytic curves stand in for them
with the paper's proportions: about 3/4 of the nodes on the outer boundary and
the rest split evenly across the holes (Sec. 4.2, Fig. demo1/demo2 captions).

Five named workloads (sizes are nodes N; the bordered system has 2N+3p
unknowns, Sec. 3.1-3.2):

* ``star1``   : star r=1+0.2cos5t, one circular hole r=0.2 at (0.3,0.1);
                1536+512 nodes, leaf 64.
* ``star16``  : star r=1+0.15cos7t, 16 random ellipses (semi-axes
                U[0.03,0.08]); 24576+16*512 nodes.
* ``quad64``  : unit circle, 64 ellipses clustered in the quadrant x,y>0
                (semi-axes U[0.02,0.04]); 98304+64*512 nodes, leaf 128.
* ``fourier8``: star r=1+0.2cos5t, 8 holes with 8 real Fourier radius
                coefficients each; 12288+8*512 nodes.
* ``star256`` : star r=1+0.1cos9t, 256 ellipses (U[0.015,0.04]);
                786432+256*1024 nodes.

Everything is drawn from ``numpy.random.default_rng(seed)``; no solver
arithmetic lives here (curves are sampled by ``workloads.curves``).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from .curves import Curve, circle, ellipse, fourier_hole, star

SEED_BASE = 1000


@dataclass
class Workload:
    name: str
    curves: list
    counts: list
    x: np.ndarray
    y: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    ddx: np.ndarray
    ddy: np.ndarray
    dt: np.ndarray          # parameter spacing per node
    comp: np.ndarray        # int32 component id (0 = outer, 1..p holes)
    centers: np.ndarray     # (p,2) parametric hole centres c_i
    src_xy: np.ndarray      # (nrhs, ns, 2) point-force locations for the RHS
    src_f: np.ndarray       # (nrhs, ns, 2) point-force strengths
    rhs_holes_zero: bool    # True: boundary data only on Gamma_0, 0 on holes
    targets: np.ndarray     # (nt,2) interior evaluation points
    leaf_size: int = 64
    n_proxy: int = 64
    proxy_ratio: float = 1.5
    id_tol: float = 1e-12
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.x.shape[0])

    @property
    def p(self) -> int:
        return int(self.centers.shape[0])

    @property
    def n_unknowns(self) -> int:
        return 2 * self.N + 3 * self.p

    def node_slice(self, c: int) -> slice:
        start = int(sum(self.counts[:c]))
        return slice(start, start + int(self.counts[c]))


def _flatten(name, curves, counts, **kw) -> Workload:
    parts = [cv.sample(n) for cv, n in zip(curves, counts)]
    cat = lambda a: np.ascontiguousarray(np.concatenate(a).astype(np.float64))
    comp = np.concatenate([np.full(n, i, dtype=np.int32)
                           for i, n in enumerate(counts)])
    dt = np.concatenate([np.full(n, s.dt) for s, n in zip(parts, counts)])
    centers = np.array([cv.center for cv in curves[1:]],
                       dtype=np.float64).reshape(-1, 2)
    return Workload(name=name, curves=list(curves), counts=list(counts),
                    x=cat([s.x for s in parts]), y=cat([s.y for s in parts]),
                    dx=cat([s.dx for s in parts]), dy=cat([s.dy for s in parts]),
                    ddx=cat([s.ddx for s in parts]),
                    ddy=cat([s.ddy for s in parts]),
                    dt=np.ascontiguousarray(dt), comp=comp, centers=centers,
                    **kw)


# ---------------------------------------------------------------------------
# geometry helpers (input generation only)

def _contains(curve: Curve, pts: np.ndarray) -> np.ndarray:
    cx, cy = curve.center
    px, py = pts[:, 0] - cx, pts[:, 1] - cy
    if curve.kind == "ellipse":
        a, b, phi = curve.params["a"], curve.params["b"], curve.params["phi"]
        c, s = np.cos(phi), np.sin(phi)
        u = (c * px + s * py) / a
        v = (-s * px + c * py) / b
        return u * u + v * v < 1.0
    th = np.arctan2(py, px)
    r = curve._polar(th)[0]
    return np.hypot(px, py) < r


def _min_dist(pts: np.ndarray, poly: np.ndarray) -> np.ndarray:
    """Distance from each point to the nearest polygon vertex (k-d tree)."""
    from scipy.spatial import cKDTree
    return cKDTree(poly).query(pts)[0]


def _perimeter(curve: Curve) -> float:
    poly = curve.polygon(2048)
    return float(np.sum(np.hypot(*(np.roll(poly, -1, 0) - poly).T)))


def _place_holes(rng, outer: Curve, n_holes: int, make, n_per_hole: int,
                 region, max_tries=200000):
    """Random sequential placement with the gap rule: gap >= max(0.02,
    10 x local node spacing) to Gamma_0 and to every other hole."""
    outer_poly = outer.polygon(8192)
    holes, polys, rads = [], [], []
    tries = 0
    while len(holes) < n_holes:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"could not place {n_holes} holes "
                               f"(placed {len(holes)})")
        cand = make(rng, region(rng))
        R = cand.bounding_radius()
        gap = max(0.02, 10.0 * _perimeter(cand) / n_per_hole)
        c = np.array(cand.center)
        poly = cand.polygon(256)
        if not np.all(_contains(outer, poly)):
            continue
        if _min_dist(poly, outer_poly).min() < gap:
            continue
        ok = True
        for h, hp, hr in zip(holes, polys, rads):
            d = np.hypot(*(c - np.array(h.center)))
            if d > R + hr + gap:
                continue
            if d < max(R, hr):
                ok = False
                break
            if _min_dist(poly, hp).min() < gap or np.any(_contains(h, poly)):
                ok = False
                break
        if ok:
            holes.append(cand)
            polys.append(poly)
            rads.append(R)
    return holes


def _rand_ellipse(lo, hi):
    def make(rng, center):
        a = rng.uniform(lo, hi)
        b = rng.uniform(lo, hi)
        phi = rng.uniform(0.0, np.pi)
        return ellipse(a, b, phi, center)
    return make


def interior_targets(curves, n, rng, min_dist=0.05):
    """Points of Omega at distance >= min_dist from every boundary curve."""
    outer, holes = curves[0], curves[1:]
    R = outer.bounding_radius()
    polys = np.concatenate([cv.polygon(4096) for cv in curves])
    out = []
    while sum(len(o) for o in out) < n:
        pts = rng.uniform(-R, R, size=(4 * n, 2)) + np.array(outer.center)
        keep = _contains(outer, pts)
        for h in holes:
            keep &= ~_contains(h, pts)
        pts = pts[keep]
        if pts.shape[0] == 0:
            continue
        pts = pts[_min_dist(pts, polys) >= min_dist]
        out.append(pts)
    return np.ascontiguousarray(np.concatenate(out)[:n])


def exterior_point_forces(rng, nrhs, n_src=3, radius=2.0):
    """Point forces on the circle |x| = radius at uniform random angles with
    N(0,1) strengths: their velocity restricted to Gamma is boundary data
    with a known interior solution."""
    th = rng.uniform(0.0, 2.0 * np.pi, size=(nrhs, n_src))
    xy = np.stack([radius * np.cos(th), radius * np.sin(th)], axis=-1)
    f = rng.standard_normal(size=(nrhs, n_src, 2))
    return xy, f


# ---------------------------------------------------------------------------
# the five workloads

def star1(seed=SEED_BASE + 0, n_outer=1536, n_hole=512, n_targets=256):
    rng = np.random.default_rng(seed)
    curves = [star(1.0, 0.2, 5), circle(0.2, (0.3, 0.1), ccw=False)]
    sxy, sf = exterior_point_forces(rng, 1)
    return _flatten("star1", curves, [n_outer, n_hole], src_xy=sxy, src_f=sf,
                    rhs_holes_zero=False,
                    targets=interior_targets(curves, n_targets, rng))


def star16(seed=SEED_BASE + 1, n_outer=24576, n_hole=512, n_holes=16,
           n_targets=1024, nrhs=1):
    rng = np.random.default_rng(seed)
    outer = star(1.0, 0.15, 7)
    region = lambda r: tuple(r.uniform(-0.8, 0.8, size=2))
    holes = _place_holes(rng, outer, n_holes, _rand_ellipse(0.03, 0.08),
                         n_hole, region)
    curves = [outer] + holes
    sxy, sf = exterior_point_forces(rng, nrhs)
    return _flatten("star16", curves, [n_outer] + [n_hole] * n_holes,
                    src_xy=sxy, src_f=sf, rhs_holes_zero=False,
                    targets=interior_targets(curves, n_targets, rng))


def quad64(seed=SEED_BASE + 2, n_outer=98304, n_hole=512, n_holes=64,
           n_targets=1024, nrhs=8):
    rng = np.random.default_rng(seed)
    outer = circle(1.0)
    region = lambda r: tuple(r.uniform(0.02, 0.95, size=2))
    holes = _place_holes(rng, outer, n_holes, _rand_ellipse(0.02, 0.04),
                         n_hole, region)
    curves = [outer] + holes
    sxy, sf = exterior_point_forces(rng, nrhs)
    return _flatten("quad64", curves, [n_outer] + [n_hole] * n_holes,
                    src_xy=sxy, src_f=sf, rhs_holes_zero=False,
                    targets=interior_targets(curves, n_targets, rng),
                    leaf_size=128)


def fourier8(seed=SEED_BASE + 3, n_outer=12288, n_hole=512, n_holes=8,
             n_targets=1024):
    rng = np.random.default_rng(seed)
    outer = star(1.0, 0.2, 5)

    def make(r, center):
        a0 = r.uniform(0.05, 0.1)
        modes = 0.1 * a0 * r.standard_normal(7)
        a = [a0, modes[0], modes[2], modes[4], modes[6]]
        b = [0.0, modes[1], modes[3], modes[5]]
        return fourier_hole(a, b, center)

    region = lambda r: tuple(r.uniform(-0.65, 0.65, size=2))
    holes = _place_holes(rng, outer, n_holes, make, n_hole, region)
    curves = [outer] + holes
    sxy, sf = exterior_point_forces(rng, 1)
    return _flatten("fourier8", curves, [n_outer] + [n_hole] * n_holes,
                    src_xy=sxy, src_f=sf, rhs_holes_zero=True,
                    targets=interior_targets(curves, n_targets, rng))


def star256(seed=SEED_BASE + 4, n_outer=786432, n_hole=1024, n_holes=256,
            n_targets=1024, nrhs=32):
    rng = np.random.default_rng(seed)
    outer = star(1.0, 0.1, 9)
    region = lambda r: tuple(r.uniform(-0.88, 0.88, size=2))
    holes = _place_holes(rng, outer, n_holes, _rand_ellipse(0.015, 0.04),
                         n_hole, region)
    curves = [outer] + holes
    sxy, sf = exterior_point_forces(rng, nrhs)
    return _flatten("star256", curves, [n_outer] + [n_hole] * n_holes,
                    src_xy=sxy, src_f=sf, rhs_holes_zero=False,
                    targets=interior_targets(curves, n_targets, rng))


def heat2(theta1=0.0, theta2=np.pi, N=16384, seed=SEED_BASE + 5,
          n_targets=256):
    """The Laplace Neumann experiment's geometry (Sec. 4.4.1): a starfish
    outer curve and two starfish holes 16 % of its size, their centres on
    a half-size copy of the outer curve at parameters theta1, theta2; 2/3
    of the N nodes on the outer curve, 1/6 on each hole.  The paper's
    outer curve is a spline through unlisted knots; r = 1 + 0.2 cos 5t
    stands in for it.  Flux data (Eq. neumanndata): 0 on the outer curve,
    +1 on hole 1, -1 on hole 2 (see heat_flux)."""
    rng = np.random.default_rng(seed)
    outer = star(1.0, 0.2, 5)

    def on_path(th):
        r = 0.5 * (1.0 + 0.2 * np.cos(5 * th))
        return (r * np.cos(th), r * np.sin(th))

    holes = [star(0.16, 0.032, 5, on_path(th), ccw=False)
             for th in (theta1, theta2)]
    n_hole = N // 6
    counts = [N - 2 * n_hole, n_hole, n_hole]
    curves = [outer] + holes
    sxy, sf = exterior_point_forces(rng, 1)
    return _flatten("heat2", curves, counts, src_xy=sxy, src_f=sf,
                    rhs_holes_zero=False,
                    targets=interior_targets(curves, n_targets, rng))


def heat_flux(w: Workload) -> np.ndarray:
    """The paper's flux data on the two-hole geometry: 0 on Gamma_0, +1 on
    Gamma_1, -1 on Gamma_2 (per node)."""
    c = np.asarray(w.comp)
    return np.where(c == 1, 1.0, np.where(c == 2, -1.0, 0.0))


WORKLOADS = {"star1": star1, "star16": star16, "quad64": quad64,
             "fourier8": fourier8, "star256": star256, "heat2": heat2}


def custom(curves, counts, name="custom", n_targets=64, seed=7, nrhs=1,
           **kw) -> Workload:
    """Any list of curves (outer first) with node counts per curve."""
    rng = np.random.default_rng(seed)
    sxy, sf = exterior_point_forces(rng, nrhs)
    tg = interior_targets(curves, n_targets, rng) if n_targets else \
        np.zeros((0, 2))
    kw.setdefault("rhs_holes_zero", False)
    return _flatten(name, curves, counts, src_xy=sxy, src_f=sf, targets=tg,
                    **kw)


def scaled(w: Workload, factor: int, name=None, n_targets=None) -> Workload:
    """The same curves with node counts divided by ``factor`` (for quick
    cases with the shape of a large workload)."""
    counts = [max(16, c // factor) for c in w.counts]
    out = _flatten(name or f"{w.name}/{factor}", w.curves, counts,
                   src_xy=w.src_xy, src_f=w.src_f,
                   rhs_holes_zero=w.rhs_holes_zero,
                   targets=w.targets if n_targets is None
                   else w.targets[:n_targets],
                   leaf_size=w.leaf_size, n_proxy=w.n_proxy,
                   proxy_ratio=w.proxy_ratio, id_tol=w.id_tol)
    return out


def move_hole(w: Workload, hole: int, delta) -> Workload:
    """Translate hole ``hole`` (1-based component id) rigidly by ``delta``.
    Node ids are unchanged; only that hole's positions and centre move."""
    curves = list(w.curves)
    curves[hole] = curves[hole].translated(float(delta[0]), float(delta[1]))
    sl = w.node_slice(hole)
    x = w.x.copy()
    y = w.y.copy()
    x[sl] += float(delta[0])
    y[sl] += float(delta[1])
    centers = w.centers.copy()
    centers[hole - 1] += np.asarray(delta, dtype=np.float64)
    return replace(w, curves=curves, x=x, y=y, centers=centers)


def remove_hole(w: Workload, hole: int):
    """Delete hole ``hole`` (1-based component id).  Its nodes go, the later
    holes are renumbered and their nodes shift down.  Returns (the new
    workload, old_id) with old_id[j] = id in ``w`` of node j of the new one."""
    keep = np.ones(w.N, dtype=bool)
    keep[w.node_slice(hole)] = False
    old_id = np.nonzero(keep)[0].astype(np.int64)
    comp = w.comp[keep]
    comp = np.where(comp > hole, comp - 1, comp).astype(np.int32)
    pick = lambda a: np.ascontiguousarray(a[keep])
    out = replace(w, curves=[c for i, c in enumerate(w.curves) if i != hole],
                  counts=[n for i, n in enumerate(w.counts) if i != hole],
                  x=pick(w.x), y=pick(w.y), dx=pick(w.dx), dy=pick(w.dy),
                  ddx=pick(w.ddx), ddy=pick(w.ddy), dt=pick(w.dt),
                  comp=np.ascontiguousarray(comp),
                  centers=np.ascontiguousarray(
                      np.delete(w.centers, hole - 1, axis=0)))
    return out, old_id


def add_hole(w: Workload, curve: Curve, n: int):
    """Append a hole sampled at n nodes; its nodes get the ids after the
    existing ones.  Returns (the new workload, old_id) with old_id[j] = -1
    for the new nodes."""
    s = curve.sample(n)
    cat = lambda a, b: np.ascontiguousarray(
        np.concatenate([a, np.asarray(b, dtype=np.float64)]))
    out = replace(w, curves=list(w.curves) + [curve],
                  counts=list(w.counts) + [n],
                  x=cat(w.x, s.x), y=cat(w.y, s.y), dx=cat(w.dx, s.dx),
                  dy=cat(w.dy, s.dy), ddx=cat(w.ddx, s.ddx),
                  ddy=cat(w.ddy, s.ddy), dt=cat(w.dt, np.full(n, s.dt)),
                  comp=np.ascontiguousarray(np.concatenate(
                      [w.comp, np.full(n, w.p + 1, dtype=np.int32)])),
                  centers=np.ascontiguousarray(np.vstack(
                      [w.centers.reshape(-1, 2),
                       np.asarray(curve.center, dtype=np.float64)[None]])))
    old_id = np.concatenate([np.arange(w.N, dtype=np.int64),
                             np.full(n, -1, dtype=np.int64)])
    return out, old_id


def random_moves(w: Workload, n_steps: int, seed: int, frac: float = 0.05):
    """Random hole translations by frac x the hole's bounding radius in a
    random direction; a move that would break the gap rule is redrawn."""
    rng = np.random.default_rng(seed)
    outer_poly = w.curves[0].polygon(8192)
    cur = w
    out = []
    for _ in range(n_steps):
        for _attempt in range(100):
            h = int(rng.integers(1, w.p + 1))
            ang = rng.uniform(0, 2 * np.pi)
            step = frac * cur.curves[h].bounding_radius()
            d = (step * np.cos(ang), step * np.sin(ang))
            moved = cur.curves[h].translated(*d)
            poly = moved.polygon(256)
            gap = 0.01
            if _min_dist(poly, outer_poly).min() < gap or \
                    not np.all(_contains(cur.curves[0], poly)):
                continue
            ok = True
            for j, cv in enumerate(cur.curves[1:], start=1):
                if j == h:
                    continue
                dd = np.hypot(*(np.array(cv.center) - np.array(moved.center)))
                if dd > cv.bounding_radius() + moved.bounding_radius() + gap:
                    continue
                if _min_dist(poly, cv.polygon(256)).min() < gap:
                    ok = False
                    break
            if ok:
                out.append((h, d))
                cur = move_hole(cur, h, d)
                break
    return out
