"""FP64 CPU oracle for the Lagrangian high-order finite-element hydrodynamics hot path.

TEST INFRASTRUCTURE ONLY. Only the test suite, the package smoke check and the
CPU-baseline leg of the benchmark may import or run anything in this package;
the product path (the CUDA library and its Python binding) never calls it.

The oracle is written from the paper's equations as plain, slow, obviously
checkable numpy/scipy code with full (global sparse) assembly of the mass and
force matrices. It shares no code with the CUDA path; the only module both
sides use is the seeded input generator `paper_2112_07075_b300.inputs`, which
holds none of the method's arithmetic.

Sources followed (arXiv 2112.07075):
  * Section 2.1, Eqs. (1)-(5): the single-material Lagrangian Euler equations
    (eta = 1, alpha = 0) with a total stress = physical + artificial viscosity.
  * Section 3.3, Eqs. (14)-(18): the semi-discrete system
    M_v dv/dt = -F.1, rho|J| = rho0|J0|, M_E de/dt = F^T v, dx/dt = v.
  * Section 3.1: the operator decomposition A = P^T G^T B^T D B G P; the oracle
    forms the dense element matrices and assembles them (the "traditional full
    assembly" row of Table 1).
  * Section 3.2: the element mass matrix (M_E)_ij = sum_k alpha_k phi_i phi_j |J|.
  * Section 6: the four major computations of the Lagrange step (mass CG
    inversion, quadrature-point data, artificial viscosity, force operator).

Where the paper is silent (force-matrix entries, equation of state, artificial
viscosity, time integrator, time-step estimate, bases, quadrature, boundary
conditions) the oracle follows one stated reading per gap, written out in
each module's docstrings.

Parity status per function is stated in each module header. Functions whose
result no closed form, invariant or special case pins are marked
"parity unpinned".
"""
