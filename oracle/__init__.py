"""Plain FP64 CPU oracle for the nonlinear FAS multigrid method of Lee, Hamon, Castelletto, Vassilevski, White,
"Nonlinear multigrid based on local spectral coarsening for heterogeneous diffusion problems".

TEST INFRASTRUCTURE ONLY. Nothing in the product library imports, links or runs this package; only the tests,
the package entry point's smoke check and the CPU-baseline leg of the benchmark use it. It shares no code with the
CUDA path: it is written directly from the paper's equations with numpy/scipy, slowly and obviously.

Modules:
  tpfa       - fine-level TPFA flux, mixed and reduced residuals, Jacobian (Sec. 2.1, eqs. TPFA_flux, FV_matrix)
  newton     - brute-force damped Newton with a sparse direct solve: the definitional solution p*
  aggregation- deterministic greedy graph aggregation (stands in for METIS, Sec. 3.1 / App. A.1)
  hierarchy  - spectral pressure bases, coarse flux space, Q, D, static local M, Pi~ weights (App. A, B)
  coarse     - level operators A^l(x) (eq. structure, Prop. 1), the Picard step (eq. picardian_system) and the
               coarse Newton Jacobian (Sec. 3.3.2, Props. 2-3, eq. jacobian_matrix)
  fas        - Algorithm 1 (backtracking), the level-0 smoothers (Picard, Picard-then-Newton, nonlinear Jacobi),
               the coarse smoothers (Picard, Newton), Algorithm 2 (FAS V-cycle) and the nonlinear cascadic start
               (Sec. 4.2)
  krylov     - fixed-length Jacobi-PCG, BiCGStab and the hybridized coarse solve of Sec. 3.4 (step-parity references)
  precond    - the linear multigrid V-cycle that preconditions the level-0 Krylov solves (Sec. 3.4's AMG stand-in)
The single-level Picard and Newton iterations of Sec. 2.2 have no module of their own: newton.solve is that
iteration (Picard steps, then Newton steps, each solved exactly) run to its limit p*, the value the library's
single-level baselines are compared with.

Every function whose result is not pinned by a test to something other than itself says "parity unpinned".
"""
