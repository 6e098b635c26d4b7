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
