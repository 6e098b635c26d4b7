"""CPU oracle for the skeletonization solver.  TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 restatement of what the paper computes, written from the
paper's text: the Nystrom discretisation of the bordered Stokes system
(Sec. 3.1), a dense LU solve of it, and a straightforward serial recursive
skeletonization with the proxy method, the bordered top-level solve and fast
updating (Sec. 2.2-2.8, 3.2).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run anything in this package.  The CUDA library
never calls it, and it never calls the CUDA library; the two share only the
seeded curve generators in ``workloads``.

Every function is pinned by a CPU test against something other than itself
(closed forms, invariants, library reductions, brute force); see
``tests/test_oracle_*.py``.
"""
from .stokes import (Geom, quadrature, dl_blocks, a11_entries,  # noqa: F401
                     k_entries, h_columns, psi_columns, dense_system,
                     dense_solve, dense_matvec_rows, point_force_velocity,
                     boundary_data, interior_velocity)
from .skeleton import (build_tree, factor, solve, solve_adjoint,  # noqa: F401
                       update, cpqr_id)
from . import laplace  # noqa: F401  (the Laplace Neumann variant)
