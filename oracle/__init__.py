"""CPU oracle for the generalized Stokes saddle-point solver (TEST INFRASTRUCTURE).

This package is a plain, slow, FP64 restatement of what the solver computes,
written from the paper (Creff & Guermond, "Preconditioning of the generalized
Stokes problem arising from the approximation of the time-dependent
Navier-Stokes equations", arXiv 2407.01783). It exists only to check the CUDA
path. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product package never does, and this package
never imports the product package. The two share no code; the only common
dependency is the seeded input generator in ``workload``.

Because the method is an iterative solver for a linear system, the oracle's
answer is the *exact discrete solution* of that system (sparse direct solve),
plus the plain definitions of every matrix and preconditioner operator:

* ``reference_element``: P2/P1 basis on a tetrahedron and exact integrals
  (Sec. 2.2, definitions of M_V, M_Q, E_V; Sec. 3.2, L_V and D; Sec. 4.1,
  L_Q and the lumped mass Lambda_V).
* ``mesh``: Kuhn (Freudenthal) tetrahedral mesh topology and DOF numbering.
* ``assemble``: global sparse matrices A = M_V/dt + mu E_V, B, M_Q, L_Q, ...
  (Eq. for A_ij, B_kj; Eq. def_of_A; Eqs. for A_lambda,1..3; Eq. for L_Q).
* ``solve``: sparse direct solve of [A -B^T; B 0][U;P] = [F;g] with the
  pressure mean fixed (Eq. Saddle_point_A_BT_B), true residuals, L2 errors.
* ``operators``: dense (tiny-mesh) Schur complement S, S_lambda and the
  Cahouet-Chabard preconditioners C_lambda, C^Lambda_lambda, C^Delta_lambda
  (Eqs. def_Schur_LA_problem, Schur_complement_preconditioners).
* ``quadrature``: conical-product Gauss rule on a tetrahedron, used only to
  pin the closed-form integrals and to measure L2 errors.

Parity status: every function here is pinned by tests under ``tests/`` against
closed forms, quadrature, invariants or brute force; see the test docstrings.
"""
