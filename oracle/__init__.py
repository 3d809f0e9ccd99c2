"""FP64 CPU oracle for near-circulant splitting (Ryu, Ko, Won, arXiv 1810.13100).

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline / reference leg may import, call or link anything in
this package.  The CUDA library never does; the two share no code.

Plain, slow, obviously correct: every quantity in float64, the algorithms in
the paper's order and notation, numpy / numpy.fft as library primitives, and
the Joseph projector pair in plain C (joseph_fp64.c) because pure Python loops
are too slow at the paper's sizes.

Parts (each function cites the passage it follows):
  operators  - geometry, Joseph K and its transpose, finite differences D, D^T
  circulant  - eigenvalues of M (eqs. (f-diff), (circ_R), (circ_D)), FFT solve,
               probe estimator (eq. (H-fan))
  prox       - proximal maps of the conjugates (Sec. 2, Sec. 4)
  solvers    - NCS, PDHG, textbook dense ADMM, objective, seminorm D, power
               iterations for (A3)
  cone       - 3-D cone beam on a circular orbit: geometry, Joseph K / K^T (in the C
               file), 3-D D, circulant M and NCS, dense ADMM (Sec. 4)
"""
from . import circulant, cone, operators, prox, solvers  # noqa: F401
from .operators import Geometry, K, KT, D, DT  # noqa: F401
from .solvers import Problem, State  # noqa: F401
