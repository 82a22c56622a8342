"""CPU FP64 oracle for the space-time Petrov-Galerkin heat solve (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The GPU library never
imports it, and it shares no code with the CUDA path: no kernels, headers, helper
tables or constant generators.  It is plain and slow on purpose.  Every function
names the passage of the paper (Henning, Palitta, Simoncini, Urban, "Matrix
oriented reduction of space-time Petrov-Galerkin variational problems",
arXiv:1912.10082) that it restates.

Modules
-------
fem       spatial P1 / Q1 mass, stiffness and convection matrices (Section 3, "X_h"), and P1 on
          simplex meshes (general meshes, Section 5 Example 1's kind)
timefe    time matrices D_t, C_t of hat trial / indicator test functions (Section 3)
kron      Kronecker assembly B = D_t (x) M + C_t (x) A, its vec identity and exact
          direct solves (Section 3 eqs. par1/par2; Section 4 eq. Kroneckersum)
rhs       manufactured loads with exact integrals; trapezoidal loads (Section 3)
cn        Crank-Nicolson time stepping (Section 3 remark, Section 5)
residual  relative residual norms of dense and low-rank iterates (Section 4)
rksm      rational Krylov Galerkin projection (RKSM) reference (Section 4)
lrfgmres  low-rank flexible GMRES preconditioned by RKSM, the comparison solver
          of Section 5, Example 1 (Table 1)
wave      the wave equation's space-time system with cubic B-splines, its direct
          solve and GMRES+LYAP (Section 3 "The Wave Equation", Section 4
          eq. 3terms, Section 5 Example 2)

Pins (tests marked ``not gpu``): closed-form 1D generalised eigenpairs, Gauss
quadrature of every matrix entry from the basis functions, an exact rational
solve of a tiny system, Crank-Nicolson equivalence, the manufactured closed form,
second-order convergence, and the Galerkin invariants of the RKSM reference;
for LR-FGMRES+RKSM the Eckart-Young truncation error, GMRES's minimal residual
over the explicit Krylov space, one step with an exact preconditioner and the
direct solution; for the simplex P1 matrices the domain measure, constants, linear
exactness and the difference-stencil closed form; for the wave equation the textbook
cubic B-spline stencils, SPD, the preconditioner inverse and second-order convergence
to Example 2's solution.
Parity unpinned: the RKSM iteration counts and shift sequence (the paper only
says the shifts are chosen adaptively); the converged solution is pinned.
"""

from . import fem, timefe, kron, rhs, cn, residual, rksm, lrfgmres  # noqa: F401
