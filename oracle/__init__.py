"""CPU oracle for the multigrid-preconditioned SIMP elasticity solve -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of what the method computes, written from the paper and the
textbook definitions it relies on.  It exists to check the CUDA path; it is never a fallback:
only the test suite, ``__graft_entry__.smoke()`` and the bench's ``cpu_baseline`` /
``--impl reference`` legs may import it.  It shares no code with the CUDA library; the only
common module is :mod:`workloads`, which generates seeded inputs and holds none of the
method's arithmetic.

Modules
  fem      element stiffness (Gauss quadrature), SIMP interpolation, CSR assembly, boundary
           conditions, sparse direct solve, compliance
  gmg      geometric bilinear/trilinear prolongation, Galerkin coarse operators, level counts
  amg      smoothed aggregation: block strength of connection, distance-2 MIS aggregation,
           tentative prolongator by Gram-Schmidt QR, Jacobi-smoothed prolongator
  mg       V-cycle (Algorithm 1) with point-block Jacobi or Chebyshev smoothing and a dense
           Cholesky coarse solve; hierarchy builders for GMG / AMG / hybrid
  design   linear density filter rho = S alpha and the compliance sensitivities (Eq. 3)
  stability  stress stiffness matrix (Eq. 4-5) and the generalized Davidson eigensolver
           (Algorithm 2)
  krylov   textbook preconditioned CG and flexible CG
  solve    one call that mirrors the library's solve options
  hashing  splitmix64, the counter-based generator both sides implement from its published
           definition (aggregation priorities, power-iteration start vectors)

Parity status per function is stated in each module header; every function is pinned by
the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` against closed forms, invariants,
brute force or the paper's printed numbers.
"""
