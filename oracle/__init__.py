"""Plain FP64 CPU oracle for the KFBI boundary-integral operator application.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, calls or
links anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may use it.  It shares no code,
tables or helpers with the CUDA path.

What it computes (arXiv 2404.14864, "A GPU-accelerated Cartesian grid method
for the heat, wave and Schroedinger equations on irregular domains"):

* ``geometry``  -- Procedure 1 of Sec. 3.3: boundary nodes, the Cartesian
  grid, regular/irregular node classification, intersections of the
  interface with grid lines.
* ``interface`` -- Procedure 2 of Sec. 3.3: jumps (Eq. 3.35 and the 3x3
  system of Sec. 3.2.5), the correction terms C+/C- (Sec. 3.2.4), the box
  solve of the five-point system (Eq. 3.31) by DST-I and an eigenvalue
  division (Sec. 3.4.2), and boundary extraction by the 6x6 Taylor system
  (Eq. 3.36).  ``apply_operator`` chains them: it evaluates the interior
  limit u+ at the boundary nodes of the solution of the interface problem
  (Eq. 3.30) with Phi = phi, Psi = psi, F = f-tilde; ``apply_neumann``
  evaluates the interior normal derivative with Phi = 0, Psi = psi (the
  Neumann BIE operator of Eq. 3.19).
* ``richardson`` -- the Richardson iteration of Eq. 3.21
* ``gmres``     -- restarted GMRES with modified Gram-Schmidt and Givens
  rotations for the Dirichlet BIE (Eq. 3.17) (Sec. 5 names GMRES as the
  Krylov alternative to the Richardson iteration of Eq. 3.21).
* ``steppers``  -- Procedure 3 / Sec. 3.1: Crank-Nicolson heat
  (Eqs. 3.1-3.4), the theta = 1/4 wave scheme (Eqs. 3.5-3.7) and Strang
  splitting for Schroedinger (Eqs. 3.8-3.12).

Everything is float64 (complex128 where kappa is complex).  Library
primitives used as steps: numpy matrix products (the DST as dense sums),
numpy.linalg.solve (the 2x2, 3x3 and 6x6 direct solves the paper asks for).

Readings of passages the paper leaves silent or garbled are listed in the
module docstrings where they are used; every function is pinned by a
``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""

from .geometry import Domain, PolarCurve, EllipseCurve, make_domain, curve_from_desc
from .interface import (
    box_solve,
    dst_matrix,
    eigenvalues,
    lagrange6_weights,
    density_derivatives,
    jumps_at,
    jump_matrix3,
    correction_rhs,
    extraction,
    extraction_stencil,
    apply_neumann,
    apply_operator,
    interface_solve,
)
from .gmres import gmres, richardson
from .steppers import HeatStepper, WaveStepper, SchrodingerStepper

__all__ = [
    "Domain", "PolarCurve", "EllipseCurve", "make_domain", "curve_from_desc",
    "box_solve", "dst_matrix", "eigenvalues", "lagrange6_weights",
    "density_derivatives", "jumps_at", "jump_matrix3", "correction_rhs",
    "extraction", "extraction_stencil", "apply_operator", "apply_neumann", "interface_solve",
    "gmres", "richardson", "HeatStepper", "WaveStepper", "SchrodingerStepper",
]
