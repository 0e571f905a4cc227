"""CPU FP64 oracle for the FR-PCPF hot path (arXiv 2006.10967).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product (the CUDA
library under ``paper_2006_10967_gb300``) never calls it, and it shares no code
with that library: it builds its own points, operators, geometry and face
pairing from the paper's definitions.

It follows the paper in the paper's order:
  Section 2   conservative phase field with local multiplier (Eq.
              altconservativephasefieldeq), normal from psi, psi advection,
              psi reset and preconditioning equation (Eq. lsequation)
  Section 3.1 FR Steps 1-6 (Eqs. extrapolateSoln, continuousGrad,
              extrapolateGrad, normalTransFlux, commonFlux, inviscidFlux,
              viscousFlux, continuousDivFlux) and the 4-stage RK march
  Section 3.2 preconditioning system (Eqs. peudoSystem1, pseudotimesystem),
              resolution indicator (Eq. resolutionIndicator), element
              viscosity (Eq. nu_s) and the L2 stop rule
  Section 3.3 copy ghost states
  Section 4   error measures E_L1, E_r, E_m and the initial condition
              (Eqs. initialCond, discEq)

Precision: float64 throughout (torch CPU tensors, so that autograd gives the
oracle's discrete adjoint).  Every function is pinned by a test in
tests/test_oracle_*.py against closed forms, library routines, invariants or
brute force; none is marked "parity unpinned".
"""
from .polys import (gauss_legendre, legendre, legendre_deriv, lagrange_matrix,
                    radau_left, radau_left_deriv)
from .element import RefElement, ref_element
from .mesh import Geometry, build_geometry
from .solver import Params, Solver, velocity, circle_ic

__all__ = ["gauss_legendre", "legendre", "legendre_deriv", "lagrange_matrix",
           "radau_left", "radau_left_deriv", "RefElement", "ref_element",
           "Geometry", "build_geometry", "Params", "Solver", "velocity", "circle_ic"]
