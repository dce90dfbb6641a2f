"""Plain FP64 CPU oracle of PiTSBiCG (Riahi, arXiv 2203.10148).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import, call or execute
anything under ``oracle/``.  The product path (the C-ABI library and its
Python binding) never touches it and shares no code with it; both sides only
consume the same seeded input arrays.

Pins (tests/test_oracle_pins.py) tie every function to something other than
itself: scalar closed forms of implicit Euler and RK4, sine/Fourier
eigenmodes of the discrete operators, the explicitly assembled block matrices
of eqs. (4) and (7), the serial fine trajectory as the exact solution,
parareal exactness after k iterations, BiCGStab finite termination, and a
hand-derived set of Algorithm 1 iterates (tests/golden/).

Parity unpinned: the paper prints no iteration counts or residual values
(its Fig. 1 images are missing), so iteration *counts* of the paper's runs
cannot be pinned.
"""
from .operators import (OracleProblem, block_dot, block_norms, chebyshev_ie_propagator,
                        dense_rk4_propagator_matrix,
                        implicit_euler_propagator, matrix_propagator, norm2, norm_N_inf,
                        rk4_propagator, rk4_step_matrix, spatial_operator)
from .solvers import SolveInfo, parareal, pitsbicg

__all__ = ["OracleProblem", "block_dot", "block_norms", "chebyshev_ie_propagator",
           "dense_rk4_propagator_matrix",
           "implicit_euler_propagator", "matrix_propagator", "norm2", "norm_N_inf",
           "rk4_propagator", "rk4_step_matrix", "spatial_operator", "SolveInfo",
           "parareal", "pitsbicg"]
