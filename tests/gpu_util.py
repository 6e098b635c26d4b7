"""Helpers shared by the GPU tests: move a workload to cuda:0 and run the
library through its Python binding."""
import numpy as np


def to_device(wl, device="cuda:0"):
    import torch
    tw = type("DevWorkload", (), {})()
    for f in ("x", "y", "dx", "dy", "ddx", "ddy", "dt", "centers"):
        setattr(tw, f, torch.tensor(np.asarray(getattr(wl, f)),
                                    dtype=torch.float64, device=device))
    tw.comp = torch.tensor(np.asarray(wl.comp), dtype=torch.int32,
                           device=device)
    return tw


def solver(wl, **kw):
    import paper_2001_11619_gb300 as skel
    kw.setdefault("leaf_size", wl.leaf_size)
    kw.setdefault("n_proxy", wl.n_proxy)
    kw.setdefault("proxy_ratio", wl.proxy_ratio)
    kw.setdefault("id_tol", wl.id_tol)
    return skel.Solver(to_device(wl), **kw)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _col2(a):
    a = np.asarray(a.cpu() if hasattr(a, "cpu") else a, dtype=np.float64)
    return a.reshape(a.shape[0], -1)


def lam_scale(wl):
    """Largest 1-norm of a row of Psi^T (Sec. 3.1): the rows integrate mu_x,
    mu_y and x^perp . mu over one hole, so |lambda| <= this x max|mu| for
    lambda = Psi^T mu, and errors in mu reach lambda with the same factor."""
    w = np.hypot(np.asarray(wl.dx), np.asarray(wl.dy)) * np.asarray(wl.dt)
    r = np.maximum(1.0, np.hypot(np.asarray(wl.x), np.asarray(wl.y)))
    comp = np.asarray(wl.comp)
    return max([float((w * r)[comp == i].sum()) for i in range(1, wl.p + 1)]
               or [0.0])


def block_errors(got, ref, wl):
    """Element-wise errors of a bordered-system solution [mu; lambda] (or
    its adjoint) against the oracle's, per column, each block against its
    own scale: max|mu - mu_ref| / max|mu_ref|, and
    max|lambda - lambda_ref| / max(max|lambda_ref|, L max|mu_ref|) with L
    from ``lam_scale`` (lambda of point forces outside Gamma_0 is zero in
    exact arithmetic, so its own maximum alone is no scale).  Returns the
    worst of each over the columns."""
    g, r = _col2(got), _col2(ref)
    n2 = r.shape[0] - 3 * wl.p
    emu, elam = 0.0, 0.0
    L = lam_scale(wl)
    for c in range(r.shape[1]):
        smu = np.abs(r[:n2, c]).max()
        emu = max(emu, float(np.abs(g[:n2, c] - r[:n2, c]).max() / smu))
        if wl.p:
            sl = max(np.abs(r[n2:, c]).max(), L * smu)
            elam = max(elam, float(np.abs(g[n2:, c] - r[n2:, c]).max() / sl))
    return emu, elam


def assert_solution_close(got, ref, wl, tol, what="solution"):
    """``block_errors`` of both blocks within tol."""
    emu, elam = block_errors(got, ref, wl)
    assert emu < tol and elam < tol, (
        f"{what}: max error mu {emu:.2e}, lambda {elam:.2e} (tol {tol:.0e})")


def assert_velocity_close(u, ue, tol, what="velocity"):
    """Element-wise: every velocity component within tol x the largest
    reference component, per right-hand side."""
    a = np.asarray(u.cpu() if hasattr(u, "cpu") else u, dtype=np.float64)
    b = np.asarray(ue, dtype=np.float64)
    a = a.reshape(a.shape[0], 2, -1)
    b = b.reshape(b.shape[0], 2, -1)
    err = max(float(np.abs(a[:, :, c] - b[:, :, c]).max() /
                    np.abs(b[:, :, c]).max()) for c in range(b.shape[2]))
    assert err < tol, f"{what}: max error {err:.2e} (tol {tol:.0e})"
