"""Plain, slow FP64 CPU oracle for the generalized-harmonic (GH) shell evolution.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library, its
CUDA kernels or the Python binding) may import, call or link this package.
It is used by ``tests/``, by ``__graft_entry__.smoke()`` (to check one small
GPU invocation) and by ``bench.py``'s ``cpu_baseline`` / ``--impl reference``
legs, which time it as a CPU baseline.

The paper (Lewis & Pfeiffer, "GPU-Accelerated Simulations of Isolated Black
Holes", arXiv:1804.09101) fixes the structure of the computation: collocation
values on Chebyshev x spherical-harmonic shells (Sec. 3.4, Eqs.
SpecToPhys/PhysToSpec and DifferentiatorI1S2), the module list Deriv /
Jacobian / Filter / GHEqns / ApplyBCs (Sec. 3.1), Kerr-Schild data for one
spinning hole (Sec. 3.1, Eq. dimensionlessspin) and the three boundary types
(Sec. 5).  It does not print the GH equations, the Kerr-Schild metric, the
filter functions or the boundary formulas; those are the standard first-order
GH system of Lindblom, Scheel, Kidder, Owen & Rinne (2006), restated here
from the mathematics.  Every function names the passage it follows.

Modules
  grid        collocation points and quadrature weights
  spectral    naive Chebyshev / spherical-harmonic analysis, synthesis,
              derivatives and filters (never a folded matrix)
  kerr_schild analytic Kerr-Schild metric and its derivatives (sympy)
  gh          3+1 split, GH right-hand side, constraints, characteristic
              fields and boundary conditions
  evolve      RK4, constraint energy, finite-difference gradients
  dp5         Dormand-Prince 5(4) adaptive step (the paper's stepper, Sec. 2.1)
  frame       rotating dual frame: SpatialCoordJac and the grid velocity (Sec. 3.1)
  tensor_filter  tensor (spin-weighted) spherical-harmonic truncation on S2 (Secs. 3.1, 3.4)
  perturb     seeded-coefficient perturbations added to the exact data
  opcount     operation-counting build: gh's pointwise algebra run on
              symbolic scalars, for the algorithmic flop count per point

Nothing here is blocked, fused or reordered beyond what the definitions
state: transforms are analysis sums followed by synthesis sums; tensor
algebra is written with einsum index strings that mirror the equations.
"""
