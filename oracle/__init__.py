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

Parity status of each function is stated in its docstring; functions without
an independent pin say "parity unpinned".
"""
