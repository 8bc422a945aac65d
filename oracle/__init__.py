"""Plain FP64 CPU oracle for the DG multigrid-Schwarz elliptic solver (arXiv 2111.06767).

TEST INFRASTRUCTURE ONLY. Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg
of `bench.py` may import this package. The product (the CUDA library and its Python binding)
never calls it and shares no code with it; the only common module is `workloads`, which
generates seeded inputs and holds none of the method's arithmetic.

Each function restates the paper's definition or algorithm step in plain numpy, in the
paper's order and notation, so it can be checked against the paper by eye:

  lgl.py      LGL collocation points, weights, Lagrange differentiation/interpolation
              (Sec. II, Eqs. field_expansion and lagrprod)
  dg.py       strong DG operator with the generalized internal-penalty flux and
              Dirichlet boundary fluxes (Sec. II, Eqs. dg_op_auxvars, dg_op_primal,
              massmat, stiffmat, liftop, numflux, penalty, bc); dense assembly
  mg.py       h-multigrid hierarchy, prolongation (Eq. prol), restriction R = P^T and
              the V-cycle (Sec. III.C, Eqs. mg_problem, mg_res)
  schwarz.py  element-centred overlapping subdomains, subdomain operator R_S A R_S^T,
              weighting (Eqs. schwarz_subd_problem, schwarz_weighting,
              schwarz_weight_prod, schwarz_weight_function), Schwarz smoothing (Sec. III.D)
  krylov.py   flexible GMRES (Sec. III.B, Saad Alg. 9.6)
  newton.py   Newton-Raphson with a sufficient-decrease line search (Sec. III.A, Eq. linearized)
  puncture.py puncture-method source terms (Sec. V names puncture problems; the
              alpha/beta definitions are the textbook Brandt-Bruegmann ones)

Parity status: the DG operator, transfers, Schwarz weights, FGMRES and Newton are pinned by
the `-m "not gpu"` tests (closed forms, invariants, dense direct solves, manufactured
solutions). The puncture fields (alpha, beta), for which the paper prints no values, are pinned
by the Bowen-York invariants (traceless, divergence-free curvature whose surface integrals give
the punctures' linear and angular momenta) and the closed form of 1/alpha.
"""
