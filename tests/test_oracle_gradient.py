"""Pins for the oracle's shape derivatives (oracle.gradient): every analytic
derivative against central finite differences of the dense bordered
matrix, on small curves where the dense system is cheap.  CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import gradient as G

H = 1e-6


def _geometry(seed=0):
    curves = [W.star(1.0, 0.2, 5),
              W.fourier_hole([0.18, 0.02, -0.015, 0.01, 0.005],
                             [0.0, 0.01, 0.02, -0.01], (0.3, 0.1)),
              W.ellipse(0.12, 0.07, 0.4, (-0.45, -0.2))]
    w = W.custom(curves, [96, 40, 40], n_targets=12, seed=seed)
    return w, G.samples(w.x, w.y, w.dx, w.dy, w.ddx, w.ddy, w.dt, w.comp,
                        w.centers)


def _perturbed(sm, field, j, h):
    out = G.samples(sm.x, sm.y, sm.dx, sm.dy, sm.ddx, sm.ddy, sm.dt,
                    sm.comp, sm.centers)
    if field == "centers":
        c = out.centers.copy()
        c.flat[j] += h
        out.centers = c
    else:
        a = getattr(out, field).copy()
        a[j] += h
        setattr(out, field, a)
    return out


def _fd(fun, sm, field, j):
    return (fun(_perturbed(sm, field, j, H)) -
            fun(_perturbed(sm, field, j, -H))) / (2 * H)


@pytest.mark.parametrize("field", list(G.FIELDS) + ["centers"])
def test_bilinear_gradient_matches_finite_differences(field):
    w, sm = _geometry()
    rng = np.random.default_rng(3)
    n = w.n_unknowns
    z, s = rng.standard_normal(n), rng.standard_normal(n)
    g, gc = G.bilinear_grad(sm, z, s)
    fun = lambda q: G.bilinear(q, z, s)
    # nodes on the outer curve, on both holes, and the centres
    idx = [0, 7, 50, 95, 96, 113, 135, 136, 150, 175] if field != "centers" \
        else list(range(4))
    scale = np.abs(z).max() * np.abs(s).max() * 50
    for j in idx:
        fd = _fd(fun, sm, field, j)
        an = gc.flat[j] if field == "centers" else g[field][j]
        assert abs(fd - an) < 1e-6 * scale + 1e-6 * abs(fd), (field, j, fd, an)


def test_energy_gradient_matches_finite_differences():
    w, sm = _geometry(1)
    tx, ty = w.targets[:, 0], w.targets[:, 1]
    rng = np.random.default_rng(4)
    s = rng.standard_normal(w.n_unknowns)
    J, gs, ge, gc = G.energy_grad(sm, s, tx, ty)
    Jf = lambda q: float((G.velocity(q, s, tx, ty) ** 2).sum())
    assert abs(J - Jf(sm)) < 1e-12 * J
    for j in (3, 100, 140, 170):
        for field in ("x", "dy"):
            fd = _fd(Jf, sm, field, j)
            assert abs(fd - ge[field][j]) < 1e-6 * (1 + abs(fd))
    for j in range(4):
        fd = _fd(Jf, sm, "centers", j)
        assert abs(fd - gc.flat[j]) < 1e-6 * (1 + abs(fd))
    # with respect to s: J is quadratic, central differences are exact
    for k in (0, 11, 2 * w.N + 1, w.n_unknowns - 1):
        e = np.zeros_like(s)
        e[k] = H
        u1 = G.velocity(sm, s + e, tx, ty)
        u0 = G.velocity(sm, s - e, tx, ty)
        fd = ((u1 ** 2).sum() - (u0 ** 2).sum()) / (2 * H)
        assert abs(fd - gs[k]) < 1e-6 * (1 + abs(fd))


def test_shape_gradient_through_fourier_parameters():
    """The adjoint gradient of J = sum |u|^2 (no-slip holes, point forces
    on the fixed outer curve) with respect to a hole's Fourier coefficients
    and centre, chained through the samples, against central differences
    of J computed with dense solves."""
    import oracle
    rng = np.random.default_rng(5)
    a = [0.16, 0.015, -0.01, 0.008, 0.004]
    b = [0.0, 0.01, 0.012, -0.006]
    cen = np.array([0.3, 0.1])
    outer = W.star(1.0, 0.2, 5)
    other = W.ellipse(0.12, 0.07, 0.4, (-0.45, -0.2))

    def build(a, b, cen):
        curves = [outer, W.fourier_hole(a, b, tuple(cen)), other]
        return W.custom(curves, [96, 48, 40], n_targets=16, seed=2,
                        rhs_holes_zero=True)

    def J_of(a, b, cen):
        w = build(a, b, cen)
        sm = G.samples(w.x, w.y, w.dx, w.dy, w.ddx, w.ddy, w.dt, w.comp,
                       w.centers)
        g = oracle.quadrature(w)
        f = oracle.boundary_data(g, w.src_xy, w.src_f, True)[:, 0]
        return w, sm, f

    w, sm, f = J_of(a, b, cen)
    tx, ty = w.targets[:, 0].copy(), w.targets[:, 1].copy()  # held fixed
    J, gsm, gc = G.shape_gradient(sm, f, tx, ty)
    # chain to the parameters: the hole's samples are linear in (a, b, c)
    sl = w.node_slice(1)

    def samples_of(a, b, cen):
        return w.curves[1].__class__("polar", tuple(cen), False,
                                     {"fourier": {"a": list(a),
                                                  "b": list(b)}}).sample(48)

    def dJ_dparam(kind, m):
        # d samples / d param by differencing the (linear) sampling map
        aa, bb, cc = list(a), list(b), cen.copy()
        if kind == "a":
            aa[m] += 1.0
        elif kind == "b":
            bb[m] += 1.0
        else:
            cc[m] += 1.0
        s1, s0 = samples_of(aa, bb, cc), samples_of(a, b, cen)
        tot = 0.0
        for fld in G.FIELDS:
            tot += (gsm[fld][sl] * (getattr(s1, fld) - getattr(s0, fld))).sum()
        if kind == "c":
            tot += gc[0, m]
        return tot

    def J_fd(kind, m):
        vals = []
        for sgn in (1, -1):
            aa, bb, cc = list(a), list(b), cen.copy()
            if kind == "a":
                aa[m] += sgn * H
            elif kind == "b":
                bb[m] += sgn * H
            else:
                cc[m] += sgn * H
            w2, sm2, f2 = J_of(aa, bb, cc)
            vals.append(G.shape_gradient(sm2, f2, tx, ty)[0])
        return (vals[0] - vals[1]) / (2 * H)

    for kind, m in (("a", 0), ("a", 2), ("b", 3), ("c", 0), ("c", 1)):
        fd = J_fd(kind, m)
        an = dJ_dparam(kind, m)
        assert abs(fd - an) < 1e-5 * abs(J) + 1e-6 * abs(fd), (kind, m, fd, an)
