"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the
CPU oracle.  Curve samples only: no solver arithmetic lives in this package."""
from .curves import Curve, CurveSamples, circle, ellipse, fourier_hole, star  # noqa: F401
from .configs import (WORKLOADS, Workload, custom, interior_targets,  # noqa: F401
                      move_hole, random_moves, remove_hole, add_hole, scaled, star1, star16, quad64,
                      fourier8, star256, heat2, heat_flux)
