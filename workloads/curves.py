"""Analytic closed curves sampled uniformly in their parameter.

This module only produces curve samples: positions gamma(t_j), first and
second parameter derivatives gamma'(t_j), gamma''(t_j) and the parameter
spacing dt.  It contains none of the solver's arithmetic (no normals, weights,
curvature terms or kernels); both the CUDA library and the CPU oracle derive
those themselves from these samples.

Orientation convention: the outer curve Gamma_0 is traversed
counter-clockwise, every hole clockwise (the domain lies to the left of the
direction of travel on every component).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CurveSamples:
    x: np.ndarray
    y: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    ddx: np.ndarray
    ddy: np.ndarray
    dt: float


@dataclass
class Curve:
    """A closed curve. ``kind`` is 'polar' (r(theta) about a centre) or
    'ellipse'.  ``ccw`` selects the direction of travel."""
    kind: str
    center: tuple
    ccw: bool
    params: dict = field(default_factory=dict)

    def translated(self, dx: float, dy: float) -> "Curve":
        return Curve(self.kind, (self.center[0] + dx, self.center[1] + dy),
                     self.ccw, dict(self.params))

    # -- radius function for polar curves: r, r', r'' at theta ------------
    def _polar(self, th):
        p = self.params
        if "fourier" in p:
            # r = a0 + sum_m (a_m cos m th + b_m sin m th)
            a = p["fourier"]["a"]
            b = p["fourier"]["b"]
            r = np.full_like(th, a[0])
            r1 = np.zeros_like(th)
            r2 = np.zeros_like(th)
            for m in range(1, len(a)):
                c, s = np.cos(m * th), np.sin(m * th)
                bm = b[m] if m < len(b) else 0.0
                r += a[m] * c + bm * s
                r1 += m * (-a[m] * s + bm * c)
                r2 += -m * m * (a[m] * c + bm * s)
            return r, r1, r2
        R0, amp, k = p["R0"], p["amp"], p["k"]
        r = R0 * (1.0 + amp * np.cos(k * th))
        r1 = -R0 * amp * k * np.sin(k * th)
        r2 = -R0 * amp * k * k * np.cos(k * th)
        return r, r1, r2

    def eval(self, s):
        """Position, first and second derivative at parameter values s
        (counter-clockwise parameterisation)."""
        cx, cy = self.center
        if self.kind == "polar":
            r, r1, r2 = self._polar(s)
            c, sn = np.cos(s), np.sin(s)
            x = cx + r * c
            y = cy + r * sn
            dx = r1 * c - r * sn
            dy = r1 * sn + r * c
            ddx = r2 * c - 2.0 * r1 * sn - r * c
            ddy = r2 * sn + 2.0 * r1 * c - r * sn
            return x, y, dx, dy, ddx, ddy
        if self.kind == "ellipse":
            a, b, phi = self.params["a"], self.params["b"], self.params["phi"]
            cp, sp = np.cos(phi), np.sin(phi)
            ex, ey = a * np.cos(s), b * np.sin(s)
            ex1, ey1 = -a * np.sin(s), b * np.cos(s)
            ex2, ey2 = -ex, -ey
            rot = lambda u, v: (cp * u - sp * v, sp * u + cp * v)
            x, y = rot(ex, ey)
            dx, dy = rot(ex1, ey1)
            ddx, ddy = rot(ex2, ey2)
            return cx + x, cy + y, dx, dy, ddx, ddy
        raise ValueError(self.kind)

    def sample(self, n: int) -> CurveSamples:
        t = 2.0 * np.pi * np.arange(n) / n
        if self.ccw:
            x, y, dx, dy, ddx, ddy = self.eval(t)
        else:
            # gamma(t) = p(-t): gamma' = -p'(-t), gamma'' = p''(-t)
            x, y, dx, dy, ddx, ddy = self.eval(-t)
            dx, dy = -dx, -dy
        return CurveSamples(x, y, dx, dy, ddx, ddy, 2.0 * np.pi / n)

    def polygon(self, n: int = 256):
        t = 2.0 * np.pi * np.arange(n) / n
        x, y, *_ = self.eval(t)
        return np.stack([x, y], axis=1)

    def bounding_radius(self) -> float:
        if self.kind == "ellipse":
            return max(self.params["a"], self.params["b"])
        th = np.linspace(0, 2 * np.pi, 1024, endpoint=False)
        return float(np.max(self._polar(th)[0]))


def star(R0=1.0, amp=0.2, k=5, center=(0.0, 0.0), ccw=True) -> Curve:
    return Curve("polar", tuple(center), ccw, {"R0": R0, "amp": amp, "k": k})


def circle(radius, center=(0.0, 0.0), ccw=True) -> Curve:
    return Curve("polar", tuple(center), ccw, {"R0": radius, "amp": 0.0, "k": 0})


def ellipse(a, b, phi, center, ccw=False) -> Curve:
    return Curve("ellipse", tuple(center), ccw, {"a": a, "b": b, "phi": phi})


def fourier_hole(a, b, center, ccw=False) -> Curve:
    return Curve("polar", tuple(center), ccw,
                 {"fourier": {"a": list(a), "b": list(b)}})
