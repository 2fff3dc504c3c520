"""Plain FP64 CPU oracle for the implicit neutrino--matter collision solve.

TEST INFRASTRUCTURE ONLY.  This package is a slow, direct restatement of the
paper's nested fixed-point algorithm (Algorithm 1 with its convergence checks,
Algorithms 2 and 3) and of every equation it calls, written with numpy in
float64.  It exists so that the CUDA path can be checked against something
whose correctness can be read off the paper.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
(the C-ABI library and its Python binding) never imports, calls or links
anything in here, and this package imports nothing from the product package.

Modules
-------
constants    physical constants and units used by the oracle
grid         geometric energy grid, Legendre--Gauss rule, integration weights
eos          closed-form synthetic equation of state and its inversion
equilibrium  Fermi--Dirac projection and the bound-enforcing limiter
opacities    table interpolation and the NES / pair kernel construction
solver       rates, the maps Q and q, Anderson acceleration, Algorithm 1,
             and an independent damped-Newton root solve for tiny nodes
velocity     the O(v/c) solve: Minerbo closure, conserved old moments, the
             velocity terms of Q and q, the momentum update
c2p          conserved-to-primitive moment recovery (Anderson-accelerated
             fixed point of Sec. 3.4)
adjoint      the gradient of a converged solve by the implicit-function theorem
"""

from . import constants, grid, eos, equilibrium, opacities, solver, velocity, c2p  # noqa: F401
