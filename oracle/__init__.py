"""FP64 CPU oracle for the tetrahedral FEM hot path -- TEST INFRASTRUCTURE.

This package is a plain, slow, obviously-correct restatement of what the
CUDA library computes.  It exists only to check that library: nothing in the
product path may import it.  The only callers are ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``.  It shares no code with the CUDA path; both consume the
seeded inputs of the ``meshgen`` package.

What it follows.  The paper (Ebb, arXiv:1506.07577) names the simulations but
prints none of their formulas: Section 7.2 runs Vega's St. Venant-Kirchhoff
(StVK) model on a tet mesh with implicit backward Euler and a Jacobi-
preconditioned conjugate gradient solve; Section 7.3 runs a neo-Hookean model
with implicit integration and CG; Section 5.2 ("Example: FEM tetmesh") gives
the domain (``tets.v[4]`` keys into vertices; per-tet values reduced with
``+=`` into vertex fields, Section 4.1 and Section 6.2 "Reductions").  The
element formulas are therefore the standard textbook ones (linear tet, constant
strain; first Piola-Kirchhoff stress P; H = -V P Dm^-T), written out in
``fem.py``; the step is linearised backward Euler with Jacobi PCG, in
``implicit.py``.  Every reading of a silence is listed in the design notes.

Pins.  The paper prints no worked example, so each function is pinned in
``tests/test_oracle_*.py`` by mathematics, not by itself: zero force at rest
and under rigid motions, balance of net force and torque, force = -dE/dx by
central differences of the energy, analytic uniform-stretch patch tests, K
symmetry and finite-difference consistency, a dense direct solve for PCG, and
free fall for the integrator.  ``springs.py`` is the spring-mass example of
Section 4.1 on the mesh's edges, pinned by physics (rest state, Newton's third
law, momentum, a two-mass harmonic oscillator).
"""
from . import fem, implicit, springs  # noqa: F401
