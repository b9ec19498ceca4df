"""FP64 CPU oracle of the variational multiscale Newton-Schur method (test infrastructure).

This package is a plain, slow, obviously-correct restatement of the paper's equations, used only
to check the CUDA path: the tests, the smoke check and the benchmark's CPU-baseline leg import it.
It shares no code with the CUDA library, and the library never imports it.

Every function cites the passage of the paper it follows (equation labels and section names of
Turner, Nakshatrala & Hjelmstad, "A variational multiscale Newton-Schur approach for the
incompressible Navier-Stokes equations"). The paper defers the element tangent matrices to a
companion paper; they are derived here by exact differentiation of the residuals of Section 4.1
and pinned by central finite differences in the tests.

Parity status: pinned (closed forms on affine cubes, patch tests, integration-by-parts identity,
finite-difference consistency, Schur exactness against the uncondensed system, Newton
quadratic convergence). The paper prints no numerical element or solve result, so no value here
is pinned against a printed number from the paper itself; Table 1's DOF bookkeeping is.
"""
from .vms import (  # noqa: F401
    Params, gauss_rule, q1_basis, bubble, element_kernel, pack_element, condense,
    assemble, apply_dirichlet, residual_vector, newton_solve, uncondensed_system,
    fine_recovery, element_residual_only, elementary_integrals, assemble_vector,
    element_dofs, gather, pack_residual, NegativeJacobian, CORNERS,
    tet_rule, p1_basis, tet_bubble, element_basis, TET_CORNERS,
)
