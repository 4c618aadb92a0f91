"""CPU oracle for the RT_k x DGQ_k Stokes multigrid method (Cui & Kanschat,
"Multigrid methods for the Stokes problem on GPU systems", arXiv 2410.09497).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the tests, the smoke check and the CPU-baseline leg of the
benchmark use it.  It is deliberately slow and plain: the global Stokes matrix
is assembled by literal quadrature of the bilinear form (Sec. 2.1, eq.
`bilinear` and eq. `weak_form`), stored in CSR, and every patch problem of the
smoother is solved by dense LU (the "Direct solver" of Sec. 3.3).  All
arithmetic is float64.  It shares no code, table or constant generator with
the CUDA library.

Modules
  basis         Gauss / Gauss-Lobatto rules and 1D Lagrange bases.
  discretization  DoF numbering, local matrices by quadrature, CSR assembly.
  manufactured  seeded manufactured solution, right-hand side, L2 errors.
  transfer      prolongation by interpolation (canonical embedding, Sec. 3).
  multigrid     coloured vertex-patch smoother (Algorithm 2), V-cycle,
                coarse solve, flexible GMRES, Schur-complement local solver.
  planar        the same method on the unit square (Kronecker-form operator,
                2 x 2-cell patches in four colours) for the 2D counts of Table 1.

What pins each part (tests/test_oracle_pins.py and tests/test_oracle_planar.py,
each through a route the function itself does not use):
  basis            closed-form nodes, weights and polynomial exactness; Lagrange
                   reproduction of monomials and their derivatives.
  Discretization   assemble: an independent Kronecker form of 1D matrices,
                   symmetry, B^T 1 = 0, coercivity, closed-form energies (interior
                   and boundary penalty), (x, div u), DoF counts of Table 2 and
                   Sec. 4.2.  apply_rows: assemble.  evaluate / divergence: the
                   embedding test and pointwise div u_h = 0.  pressure_weights:
                   exact integrals of pressure-space fields.
  manufactured     div u = 0, f = -nu Laplace u + grad p and u = 0 on the boundary
                   by finite differences; rhs and l2_errors by optimal L2 rates.
  transfer         coarse functions reproduced at random points; P^T A P equals
                   the coarse matrix with doubled penalty.
  multigrid        patches: sizes and disjointness per colour; local solvers:
                   exact on the single 2^3 patch, patch equilibrium after each
                   colour on 3^3 cells, Schur-CG = LU when converged and = the
                   brute-force Krylov energy minimiser after j steps; coarse
                   solve: exact for consistent b; FGMRES: brute-force least
                   squares over the Krylov vectors; V-cycle and solver: the
                   iteration counts of Sec. 3.3 and Table 2 (3D) and Table 1 (2D).
  planar           closed forms, symmetry, null space, coercivity, Galerkin
                   identity, one-patch exactness, Table 1.
Parity unpinned: only what the paper does not state (its manufactured
solution's sigma and mu, the 3D counts and errors of its lost figures).
"""
