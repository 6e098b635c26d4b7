"""The differentiation path on the GPU: the shape-derivative kernels
against the oracle's analytic derivatives, the adjoint gradient against the
oracle's dense-LU gradient at 2048 nodes, and the torch autograd path
through Fourier hole parameters against central finite differences on the
16384-node, 8-hole geometry."""
import numpy as np
import pytest

import workloads as W
from gpu_util import solver

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _samples(w):
    from oracle import gradient as G
    return G.samples(w.x, w.y, w.dx, w.dy, w.ddx, w.ddy, w.dt, w.comp,
                     w.centers)


def _small():
    curves = [W.star(1.0, 0.2, 5),
              W.fourier_hole([0.18, 0.02, -0.015, 0.01, 0.005],
                             [0.0, 0.01, 0.02, -0.01], (0.3, 0.1)),
              W.ellipse(0.12, 0.07, 0.4, (-0.45, -0.2))]
    return W.custom(curves, [384, 160, 160], n_targets=32, seed=1,
                    leaf_size=32)


@pytest.mark.parametrize("case", ["small", "star1"])
def test_grad_bilinear_matches_oracle(case):
    from oracle import gradient as G
    w = _small() if case == "small" else W.star1()
    rng = np.random.default_rng(7)
    z, s = rng.standard_normal(w.n_unknowns), rng.standard_normal(w.n_unknowns)
    go, gco = G.bilinear_grad(_samples(w), z, s)
    sv = solver(w)
    g = sv.grad_bilinear(z, s)
    for f in G.FIELDS:
        assert _rel(g[f], go[f]) < 1e-11, f
    assert _rel(g["centers"], gco) < 1e-11


def test_grad_velocity_matches_oracle():
    from oracle import gradient as G
    w = _small()
    rng = np.random.default_rng(8)
    s = rng.standard_normal(w.n_unknowns)
    tx, ty = w.targets[:, 0].copy(), w.targets[:, 1].copy()
    J, gso, geo, gco = G.energy_grad(_samples(w), s, tx, ty)
    ubar = 2.0 * G.velocity(_samples(w), s, tx, ty)
    sv = solver(w)
    gs, g = sv.grad_velocity(s, tx, ty, ubar)
    assert _rel(gs, gso) < 1e-12
    for f in ("x", "y", "dx", "dy"):
        assert _rel(g[f], geo[f]) < 1e-11, f
    assert np.abs(g["ddx"]).max() == 0.0
    assert _rel(g["centers"], gco) < 1e-11


def test_adjoint_gradient_matches_dense_oracle_2048():
    """J = sum |u|^2 on the 8 Fourier-hole geometry at 2048 nodes (no-slip
    holes): the GPU's skeletonized adjoint gradient against the oracle's
    dense-LU adjoint gradient."""
    import oracle
    from oracle import gradient as G
    w = W.scaled(W.fourier8(), 8, n_targets=128)
    g = oracle.quadrature(w)
    f = oracle.boundary_data(g, w.src_xy, w.src_f, True)[:, 0]
    tx, ty = w.targets[:, 0].copy(), w.targets[:, 1].copy()
    Jo, go, gco = G.shape_gradient(_samples(w), f, tx, ty)
    sv = solver(w)
    sv.factor()
    J, s, gr = sv.velocity_energy_gradient(f, tx, ty)
    assert abs(J - Jo) < 1e-10 * Jo
    # errors against the whole gradient's size (the centres' own part is
    # tiny with no-slip holes: it enters only through H)
    scale = np.sqrt(sum(np.linalg.norm(go[f]) ** 2 for f in G.FIELDS) +
                    np.linalg.norm(gco) ** 2)
    for fld in G.FIELDS:
        assert np.linalg.norm(gr[fld] - go[fld]) < 1e-9 * scale, fld
        assert _rel(gr[fld], go[fld]) < 1e-8, fld
    assert np.linalg.norm(gr["centers"] - gco) < 1e-9 * scale


def _fourier_geometry(torch, theta, w, holes):
    """Samples of the outer curve (fixed, from w) and of the Fourier holes
    (from theta: per hole a0..a4, b1..b3, cx, cy) as torch tensors."""
    outs = {f: [torch.tensor(getattr(w, f)[w.node_slice(0)])]
            for f in ("x", "y", "dx", "dy", "ddx", "ddy")}
    cen = []
    for h in range(holes):
        n = w.counts[h + 1]
        p = theta[10 * h:10 * h + 10]
        a, b, c = p[0:5], p[5:8], p[8:10]
        t = -2.0 * np.pi * torch.arange(n, dtype=torch.float64) / n  # p(-t)
        r = a[0] + sum(a[m] * torch.cos(m * t) for m in range(1, 5)) + \
            sum(b[m - 1] * torch.sin(m * t) for m in range(1, 4))
        r1 = sum(m * (-a[m] * torch.sin(m * t)) for m in range(1, 5)) + \
            sum(m * b[m - 1] * torch.cos(m * t) for m in range(1, 4))
        r2 = sum(-m * m * a[m] * torch.cos(m * t) for m in range(1, 5)) + \
            sum(-m * m * b[m - 1] * torch.sin(m * t) for m in range(1, 4))
        cs, sn = torch.cos(t), torch.sin(t)
        outs["x"].append(c[0] + r * cs)
        outs["y"].append(c[1] + r * sn)
        # clockwise: gamma(t) = p(-t), gamma' = -p'(-t), gamma'' = p''(-t)
        outs["dx"].append(-(r1 * cs - r * sn))
        outs["dy"].append(-(r1 * sn + r * cs))
        outs["ddx"].append(r2 * cs - 2.0 * r1 * sn - r * cs)
        outs["ddy"].append(r2 * sn + 2.0 * r1 * cs - r * sn)
        cen.append(c)
    geo = {k: torch.cat(v) for k, v in outs.items()}
    geo["centers"] = torch.stack(cen)
    return geo


def test_autograd_fourier_parameters_against_finite_differences():
    """The 16384-node geometry with 8 Fourier holes (80 shape parameters):
    the torch gradient of J through velocity_energy against central
    differences (h = 1e-6) of J itself, for several parameters."""
    import torch
    from paper_2001_11619_gb300.autograd import velocity_energy
    w = W.fourier8()
    holes = w.p
    th0 = []
    for h in range(holes):
        par = w.curves[h + 1].params["fourier"]
        th0 += list(par["a"]) + list(par["b"][1:4]) + list(w.centers[h])
    dev = torch.device("cuda")
    tx = torch.tensor(w.targets[:, 0].copy(), device=dev)
    ty = torch.tensor(w.targets[:, 1].copy(), device=dev)
    dt = torch.tensor(w.dt, device=dev)
    comp = torch.tensor(w.comp, dtype=torch.int32, device=dev)
    opts = dict(leaf_size=w.leaf_size, n_proxy=w.n_proxy,
                proxy_ratio=w.proxy_ratio, id_tol=1e-12)

    def J_of(theta, grad=False):
        geo = _fourier_geometry(torch, theta, w, holes)
        geo = {k: v.to(dev) for k, v in geo.items()}
        return velocity_energy(geo["x"], geo["y"], geo["dx"], geo["dy"],
                               geo["ddx"], geo["ddy"], geo["centers"], dt,
                               comp, w.src_xy, w.src_f, tx, ty, **opts)

    theta = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    geo0 = _fourier_geometry(torch, theta.detach(), w, holes)
    for f in ("x", "y", "dx", "dy", "ddx", "ddy"):
        assert np.allclose(geo0[f].numpy(), getattr(w, f), rtol=0,
                           atol=1e-13), f
    J = J_of(theta)
    J.backward()
    gth = theta.grad.numpy()
    assert np.all(np.isfinite(gth)) and np.abs(gth).max() > 0
    h = 1e-6
    for k in (0, 1, 5, 8, 19, 44, 79):
        tp = theta.detach().clone()
        tm = theta.detach().clone()
        tp[k] += h
        tm[k] -= h
        fd = (J_of(tp).item() - J_of(tm).item()) / (2 * h)
        assert abs(fd - gth[k]) < 1e-5 * np.abs(gth).max() + 1e-4 * abs(fd), \
            (k, fd, gth[k])


def test_autograd_all_80_fourier_parameters_against_dense_oracle():
    """The torch path on the 8 Fourier-hole geometry at 2048 nodes: dJ/dtheta
    for all 80 shape parameters (per hole a0..a4, b1..b3 and the centre)
    from velocity_energy's backward pass (skeletonized adjoint) against the
    oracle's dense-LU adjoint gradient of the samples, taken through the
    same parametrisation by torch's chain rule; and J itself."""
    import torch
    import oracle
    from oracle import gradient as G
    from paper_2001_11619_gb300.autograd import velocity_energy
    w = W.scaled(W.fourier8(), 8, n_targets=128)
    holes = w.p
    th0 = []
    for h in range(holes):
        par = w.curves[h + 1].params["fourier"]
        th0 += list(par["a"]) + list(par["b"][1:4]) + list(w.centers[h])
    assert len(th0) == 80
    # the oracle: dense adjoint gradient of the samples, then theta
    g = oracle.quadrature(w)
    f = oracle.boundary_data(g, w.src_xy, w.src_f, True)[:, 0]
    tx, ty = w.targets[:, 0].copy(), w.targets[:, 1].copy()
    Jo, go, gco = G.shape_gradient(_samples(w), f, tx, ty)
    th = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    geo = _fourier_geometry(torch, th, w, holes)
    outs = [geo[k] for k in G.FIELDS] + [geo["centers"]]
    gouts = [torch.tensor(np.asarray(go[k])) for k in G.FIELDS] + \
        [torch.tensor(np.asarray(gco).reshape(holes, 2))]
    g_oracle = torch.autograd.grad(outs, th, gouts)[0].numpy()
    # the GPU through autograd
    dev = torch.device("cuda")
    thg = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    geo = {k: v.to(dev) for k, v in
           _fourier_geometry(torch, thg, w, holes).items()}
    J = velocity_energy(geo["x"], geo["y"], geo["dx"], geo["dy"],
                        geo["ddx"], geo["ddy"], geo["centers"],
                        torch.tensor(w.dt, device=dev),
                        torch.tensor(w.comp, dtype=torch.int32, device=dev),
                        w.src_xy, w.src_f, torch.tensor(tx, device=dev),
                        torch.tensor(ty, device=dev),
                        leaf_size=w.leaf_size, n_proxy=w.n_proxy,
                        proxy_ratio=w.proxy_ratio, id_tol=1e-12)
    assert abs(J.item() - Jo) < 1e-10 * Jo
    J.backward()
    g_gpu = thg.grad.numpy()
    assert np.abs(g_oracle).max() > 0
    err = np.abs(g_gpu - g_oracle).max() / np.abs(g_oracle).max()
    assert err < 1e-8, err


def test_velocity_energy_value_and_gradient_calls():
    """skel_velocity_energy gives the same J and solution as a solve plus
    an evaluation, and skel_velocity_energy_gradient the same gradient as
    the four calls it combines (2048-node Fourier-hole case)."""
    import oracle
    w = W.scaled(W.fourier8(), 8, n_targets=64)
    g = oracle.quadrature(w)
    f = oracle.boundary_data(g, w.src_xy, w.src_f, True)[:, 0]
    tx, ty = w.targets[:, 0].copy(), w.targets[:, 1].copy()
    sv = solver(w)
    sv.factor()
    J, s = sv.velocity_energy(f, tx, ty)
    s2 = sv.solve(f)
    assert np.array_equal(np.asarray(s), np.asarray(s2))
    u = sv.eval_velocity(s2, tx, ty)[:, :, 0]
    assert abs(J - float((u * u).sum())) < 1e-13 * J
    gr = sv.velocity_energy_gradient_at(s, tx, ty)
    gs, gE = sv.grad_velocity(s, tx, ty, 2.0 * u)
    z = sv.solve_adjoint(gs)
    gA = sv.grad_bilinear(z, s)
    for k in gE:
        ref = np.asarray(gE[k]) - np.asarray(gA[k])
        assert np.abs(np.asarray(gr[k]) - ref).max() <= \
            1e-13 * max(np.abs(ref).max(), 1e-300), k
