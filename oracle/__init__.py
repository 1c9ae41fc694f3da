"""Plain, slow, FP64 CPU oracle for the NSFR-EC residual hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never links, imports or calls it, and it shares no code with the
library: the operators, geometry, fluxes and residual are all recomputed here
in numpy, written from the paper (Cicchino & Nadarajah, "Weight-adjusted
nonlinearly stable flux reconstruction ...", arXiv 2312.07725) and the
standard definitions it cites.

Every routine is written generically over the scalar type: called with
float64 arrays it is the FP64 reference, called with complex128 arrays (all
branch decisions taken on real parts) it yields exact directional derivatives
by the complex-step method, which is the oracle's reference gradient.

Layout conventions inside the oracle:
  * nodal fields are (..., n, n, n) with the last three axes (zeta, eta, xi),
    so flattening gives xi fastest, as in the library's [N_e][var][n^3];
  * conserved state U has shape (5, N_e, n, n, n);
  * metric C has shape (3 [reference direction d], 3 [physical component],
    N_e, n, n, n): C[d, c] = (J a^d)_c, the d-th row of C^T.

Modules:
  quadrature   Gauss-Legendre / Gauss-Lobatto nodes and weights
  operators1d  Lagrange interpolation/differentiation, SBP, ESFR K and Pi~
  geometry     conservative-curl metric terms, Jacobians, face normals
  physics      entropy variables, EC fluxes (Chandrashekar; with Ranocha's pressure terms), dissipations
  residual     NSFR residual, line-wise (sum-factorised) and dense forms
  mass         weight-adjusted inverse of the FR mass matrix
  timestep     classic RK4, CFL time step
  diagnostics  entropy rate, conserved totals, kinetic energy
  problem      a small driver bundling the above for a structured mesh

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, library routines, identities proved in the paper, or a dense
brute-force assembly; the time step, wave speed, RK4 weights, kinetic energy
and entropy total by tests/test_oracle_time_diagnostics.py (closed-form wave
speeds, the RK4 stability polynomial and observed order 4, the Taylor-Green
kinetic energy pi^3, the entropy of a constant state).  Parity unpinned: the
numerical value of c_+ (not printed; the oracle takes c as an input) and the
paper's exact Roe variant (not printed; classical Roe is pinned by its
linearisation property only).
"""
