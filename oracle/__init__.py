"""Oracle: a plain, slow, FP64 CPU implementation of the entropy-stable modal
DSEM of Montoya & Zingg (arXiv 2312.07874), written step by step from the
paper's definitions for use as TEST INFRASTRUCTURE ONLY.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  The CUDA library shares no code with it.

Modules
  jacobi     Section 2.5   Jacobi polynomials, Gauss-Jacobi rules, Lagrange polynomials
  reference  Section 3     tensor-product SBP operators on the reference triangle/tetrahedron
  pkd        Section 4.3   Proriol-Koornwinder-Dubiner basis and Vandermonde matrix
  geometry   Section 4.1-2 polynomial mapping, exact/curl-form metrics, Nanson normals,
                           interpolated Jacobian, facet matching (Assumption 2)
  euler      Section 7.1-2 Euler flux, entropy variables, log mean, Ranocha flux, Davis speed
  residual   Section 4.4-6, 5, 6   dense, sparse and hybridized residual routes; projection;
                           weight-adjusted inverse; diagnostics
  skew       Section 4.4   conservative and skew-symmetric nodal forms (Eq. (rhs_cons),
                           Eq. (rhs_skew)) for Euler and scalar linear advection
  timestep   classical RK4 (not in the paper)
  jacobian   complex-step Jacobian-vector products (not in the paper)

Parity status: every function here is pinned by a test in tests/test_oracle_*.py
against closed forms, library routines, theorems of Section 6, or brute force.
"""
