/*
 * stokesmg.h - C ABI of a single-GPU (sm_103a) matrix-free multigrid solver for
 * the Stokes problem discretized with Raviart-Thomas RT_k velocity and DGQ_k
 * pressure on uniform Cartesian meshes of the unit cube.
 *
 * Method: Cui & Kanschat, "Multigrid methods for the Stokes problem on GPU
 * systems" (arXiv 2410.09497).  Each entry point cites the passage that
 * defines the operation it performs.
 *
 * Conventions shared by every call
 * --------------------------------
 *  Mesh:   n cells per side, h = 1/n, degree k in 1..5, m = n (k+1).
 *  Vector: [u_x | u_y | u_z | p], contiguous, N = 3 (m+1) m^2 + m^3 entries.
 *          Component c is an (E0, E1, E2) grid, x fastest, E_d = m+1 in
 *          direction c (its continuous, normal direction) and m otherwise;
 *          entry (i0, i1, i2) sits at i0 + E0 (i1 + E1 i2) within the block.
 *          p is an (m, m, m) grid.  Node a (0-based) of cell j in a direction
 *          has 1D index j (k+1) + a.  Support points: Gauss-Lobatto points in
 *          the continuous direction, Gauss points in the others and for p.
 *  Constraint: boundary normal entries (index 0 or m in direction c of u_c)
 *          are zero: operators ignore them on input and write 0 there.
 *  Levels: level 0 is the coarsest mesh (2 or 3 cells per side), the finest
 *          level is stk_num_levels() - 1 and has the n given to stk_setup.
 *  Memory: every vector argument is a DEVICE pointer unless the name says
 *          host; the caller owns it; it must be 16-byte aligned and not alias
 *          another argument of the same call unless stated.  The library
 *          keeps no pointer past the call.  All work is ordered on the stream
 *          given in stk_options (NULL = legacy default stream) and the calls
 *          return before it finishes, except where stated.
 *  dtype:  STK_F64 (double) or STK_F32 (float) vectors; the arithmetic is
 *          done in that precision.
 *  Errors: 0 = STK_OK; negative codes below.  No call aborts, throws or
 *          exits; stk_last_error() gives a message for the last failure.
 *  Threads: distinct problems may be used from different host threads at
 *          once (the shared coarse factors and launch attributes are
 *          synchronised), except that stk_smooth_static calls share one
 *          scratch array; one problem must not be used by two threads at
 *          once.  The messages read through stk_last_error(NULL) are kept
 *          per thread.
 */
#ifndef STOKESMG_H
#define STOKESMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STK_OK = 0,
  STK_EINVAL = -1,   /* bad argument: degree, size, level, dtype, null or misaligned pointer */
  STK_ECUDA = -2,    /* a CUDA call failed (message holds the CUDA error string)          */
  STK_ENOMEM = -3,   /* device or host allocation failed                                 */
  STK_ENOCONV = -4,  /* iteration limit reached before the tolerance                     */
  STK_ETIMEOUT = -5, /* a bounded device-side wait ran out (not returned: no kernel of
                        this library waits on another kernel or on a flag)              */
  STK_ESTATE = -6    /* call not valid in the current state                              */
};

enum { STK_F64 = 0, STK_F32 = 1 };
enum { STK_PREC_FP64 = 0, STK_PREC_MIXED = 1 };
/* Local solver of the patch smoother (Sec. 3.2): conjugate gradients on the
 * pressure Schur complement with a fixed number of steps, or until a relative
 * tolerance is met; or Direct (the paper's exact local solver, Sec. 3.2): the
 * inverse of the Schur complement of every patch type of a level is built
 * once in FP64 (on the level's first smoothing step, which is then
 * synchronous and allocates) and applied as one dense product per patch. */
enum { STK_CG_FIXED = 0, STK_CG_TOL = 1, STK_LOCAL_DIRECT = 2 };

typedef struct stk_options {
  int precision;         /* STK_PREC_FP64 or STK_PREC_MIXED (V-cycle in FP32, Sec. 4.3) */
  int gmres_restart;     /* restart length of the flexible GMRES, default 20           */
  int max_iter;          /* total GMRES iteration limit, default 200                    */
  int local_cg_mode;     /* STK_CG_FIXED (default), STK_CG_TOL or STK_LOCAL_DIRECT     */
  int local_cg_iters;    /* CG steps in FIXED mode, step limit in TOL mode; default 15 */
  double local_cg_tol;   /* relative CG residual in TOL mode, default 1e-8; FP32 smoothing
                          * uses max(local_cg_tol, 1e-6), the accuracy an FP32 CG reaches */
  double penalty_factor; /* gamma = penalty_factor (k+1)(k+2)/h, default 1             */
  void* stream;          /* cudaStream_t used by every call, NULL = default stream     */
  int use_graphs;        /* 1 (default): stk_solve replays its V-cycle as a captured
                            CUDA graph (needs a non-NULL stream); 0: direct launches */
  int fused_smoother;    /* 0 (default): each colour of the smoother first computes the
                            residual of the whole level (one operator apply), then the
                            patch kernel reads its patches' rows; 1: the patch kernel
                            computes its patch residual itself from the current x and b
                            (every coupling across the patch boundary kept).  Same
                            result up to rounding; on GB300 the default is faster for
                            every degree and precision (the patch kernel is bound by
                            shared-memory traffic, which the fused residual adds to). */
  int direct_gemm;       /* FP32 smoothing with the Direct local solver, on levels with
                            at least 512 interior patches per colour: 2 (default) the
                            product P = M R of all interior patches of a colour is one
                            GEMM on the tensor cores (cuBLAS, FP32 emulated by three
                            BF16 terms); 1 the same GEMM in plain FP32 on the CUDA
                            cores; 0 one product per patch inside the patch kernel. */
} stk_options;

typedef struct stk_problem stk_problem;

typedef struct stk_solve_info {
  int iterations;           /* GMRES iterations performed                               */
  int converged;            /* 1 if ||b - A x|| <= rtol ||b||                            */
  double relres;            /* final true relative residual                             */
  double nu;                /* fractional iteration count -8 / log10(rbar), Sec. 3.3    */
  double seconds;           /* wall time of the solve                                   */
  double residuals[256];    /* relative residual after each iteration, [0] = 1          */
} stk_solve_info;

/* Fill *opt with the defaults listed above: the solver settings of Sec. 3.3
 * (GMRES preconditioned by one V-cycle, about 15 local CG steps) where the
 * paper states them.  Returns STK_EINVAL if opt is NULL. */
int stk_default_options(stk_options* opt);

/* Build the mesh hierarchy and the 1D tables of every level (Sec. 2.3,
 * Sec. 3.2) for the unit cube with n cells per side, degree k and viscosity
 * nu (Sec. 2, eq. `model` and eq. `weak_form`).  n must be 2 or 3 times a
 * power of two (n >= 2) with m = n (k+1) <= 1200 (larger meshes: STK_EINVAL,
 * "mesh too large"; this keeps the operator's 32-bit per-CTA offsets in
 * range); k in 1..5; nu > 0.  opt may be NULL (defaults).  The
 * multigrid workspace of a dtype, the coarse factors and the Krylov basis are
 * allocated by the first call that needs them.  On success *out owns device
 * memory until stk_destroy.  Synchronous. */
int stk_setup(int n, int k, double nu, const stk_options* opt, stk_problem** out);

/* The same method on the unit square, for the two-dimensional results of
 * Table 1 (Sec. 3.3): RT_k x DGQ_k on n x n cells (n a power of two, n >= 2,
 * n (k+1) <= 8192), k in 1..8, vertex patches of 2 x 2 cells in four colours
 * (Sec. 3.1) with the exact ("Direct", Sec. 3.3) local solver, the embedding
 * and its transpose as transfers and the exact coarse solve on 2 x 2 cells.
 * Vector layout [u_x | u_y | p], x fastest: u_x on (m+1) x m nodes
 * (continuous in x), u_y on m x (m+1) (continuous in y), p on m x m,
 * m = n (k+1); normal entries on the boundary are constrained to zero.
 * Every entry point takes the returned problem: stk_layout (n_vel_component
 * = (m+1) m), stk_apply, stk_apply_stage, stk_residual, stk_prolongate_add,
 * stk_restrict, stk_smooth (four colours), stk_smooth_colour (colour 0..3),
 * stk_coarse_solve, stk_vcycle, stk_solve, stk_solve_batch and stk_rhs;
 * stk_smooth_batch, stk_smooth_static and stk_autotune are three-dimensional
 * only (STK_EINVAL).  The local_cg options are ignored (the local solver is
 * exact).  The patch inverses (one per boundary type, built on the host in
 * FP64, 16 types x (2 (2k+1)(2k+2) + (2k+2)^2)^2 entries in FP64 and FP32)
 * are shared by every problem of the process with the same device, degree,
 * viscosity and penalty factor.  Synchronous. */
int stk_setup_planar(int n, int k, double nu, const stk_options* opt, stk_problem** out);

/* L2 errors ||u - u_h|| and ||(-p) - p_h|| over the unit square of a
 * two-dimensional discrete solution x (finest level, FP64 device vector)
 * against the manufactured solution that stk_rhs builds from the same
 * coefficients (the discrete pressure approximates -p because the velocity
 * rows carry +(p, div v)), by the (k+3)^2-point Gauss rule of every cell: the
 * error measure of the paper's accuracy study (Sec. 3.3).  err_u and err_p are
 * host pointers.  Synchronous; allocates and frees a small device buffer.
 * STK_EINVAL for a three-dimensional problem or NULL arguments. */
int stk_planar_errors(stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq,
                      const double* p_amp, const double* x, double* err_u, double* err_p);

/* Release everything stk_setup allocated (bookkeeping, no counterpart in the
 * paper).  NULL is accepted. */
int stk_destroy(stk_problem* P);

/* Message of the last failed call on P (or of the last failed stk_setup when
 * P is NULL); error reporting has no counterpart in the paper.  The string
 * stays valid until the next call on P. */
const char* stk_last_error(const stk_problem* P);

/* Number of levels of the mesh hierarchy of the multigrid method (Sec. 3:
 * nested meshes obtained by uniform refinement of the coarsest one). */
int stk_num_levels(const stk_problem* P, int* nlevels);

/* Cells per side, per-velocity-component length, pressure length and total
 * length N of the vectors of one level: the DoF counts of the RT_k x DGQ_k
 * spaces (Sec. 2.1) in the layout described above. */
int stk_layout(const stk_problem* P, int level, int* n_cells, int64_t* n_vel_component,
               int64_t* n_pressure, int64_t* n_total);

/* The 1D fast-diagonalization data of the vertex-patch local solver (Sec. 3.2,
 * eq. `inverse2d` and eq. `fast_inverse`) exactly as stk_setup builds it for a
 * level of n cells per side, degree k, viscosity nu and penalty factor:
 * the generalized eigenpairs K S = M S diag(lambda), S^T M S = I, of one 1D
 * patch operator (K and M of the two cells of a patch; K without the factor nu).
 *   direction 0     the continuous direction of a velocity component: the
 *                   2k+1 patch-interior nodes, K the 1D stiffness, M the 1D
 *                   mass of the continuous basis;
 *   direction 1..4  a discontinuous direction of boundary type direction - 1
 *                   (0 interior patch, 1 patch on the lower mesh boundary,
 *                   2 on the upper one, 3 both): the 2k+2 nodes, K the 1D
 *                   interior-penalty operator with this level's penalty, M
 *                   the diagonal Gauss mass.
 * S (row-major dim x dim, eigenvectors in its columns) and lambda (dim) are
 * host arrays of the caller with room for (2k+2)^2 and 2k+2 doubles; *dim
 * receives 2k+1 or 2k+2 and *even_odd 1 when the columns are ordered with the
 * eigenvectors symmetric under the patch's reflection first and the
 * antisymmetric ones after (the kernels then transform lines in even-odd
 * form), else 0.  Host computation only: needs no GPU, touches no device and
 * keeps no state.  STK_EINVAL (message in stk_last_error(NULL)) for k outside
 * 1..5, n < 2, nu or penalty_factor not positive, direction outside 0..4 or a
 * NULL pointer; STK_ENOMEM if a host allocation fails. */
int stk_patch_eigen(int n, int k, double nu, double penalty_factor, int direction, double* S, double* lambda,
                    int* dim, int* even_odd);

/* The 1D cell matrices of the operator's Kronecker form (Sec. 2.3; the sums
 * of Kronecker products that the operator apply evaluates), exactly as
 * stk_setup builds them for a level of n cells per side, degree k, viscosity
 * nu and penalty factor.  With nc = k+2 and nd = k+1 they are written, all
 * row-major, one after another into the caller's host array out:
 *   KC  nc x nc      nu times the stiffness of one cell's continuous
 *                    (Gauss-Lobatto) basis;
 *   MC  nc x nc      the mass of that basis;
 *   D   nd x nc      D[a][i] = integral over the cell of psi_a phi_i', the
 *                    divergence factor (psi: Gauss basis, phi: Lobatto basis);
 *   LS  3 x nd x nd  diagonal block of nu times the 1D interior-penalty
 *                    operator of a discontinuous direction (eq. `bilinear` on
 *                    a line) for a cell inside the mesh (0), at its lower
 *                    boundary (1) and at its upper boundary (2);
 *   LLO nd x nd      its block coupling a cell's rows to the lower neighbour;
 *   LHI nd x nd      its block coupling a cell's rows to the upper neighbour;
 *   S   nd           the diagonal Gauss mass h w_a of a discontinuous direction;
 * 2 nc^2 + nd nc + 5 nd^2 + nd doubles in all.  Host computation only: needs
 * no GPU, touches no device and keeps no state.  STK_EINVAL (message in
 * stk_last_error(NULL)) for k outside 1..5, n < 2, nu or penalty_factor not
 * positive or out NULL; STK_ENOMEM if a host allocation fails. */
int stk_cell_tables(int n, int k, double nu, double penalty_factor, double* out);

/* The 1D child matrices of the level transfers (Sec. 3: the prolongation is
 * the canonical embedding of the nested spaces, the restriction its
 * transpose) exactly as stk_setup builds them for degree k: with nc = k+2,
 * nd = k+1 and zC / zD the Gauss-Lobatto / Gauss points of [0, 1],
 *   PC[ch][a][b] = lC_b((ch + zC_a) / 2)   ch = 0, 1; a, b < nc
 *   PD[ch][a][b] = lD_b((ch + zD_a) / 2)   ch = 0, 1; a, b < nd
 * (lC, lD the Lagrange bases of a coarse cell; ch the child, a the child's
 * node, b the coarse node), written row-major into the caller's host array
 * out, PC first: 2 nc^2 + 2 nd^2 doubles.  Host computation only: needs no
 * GPU, touches no device and keeps no state.  STK_EINVAL (message in
 * stk_last_error(NULL)) for k outside 1..5 or out NULL; STK_ENOMEM if a host
 * allocation fails. */
int stk_transfer_tables(int k, double* out);

/* y = A x on one level: the matrix-free Stokes operator of Algorithm 1 (cell,
 * interior-face and boundary-face loops of eq. `bilinear`, with the divergence
 * blocks of eq. `weak_form`), evaluated through its Kronecker form on the
 * Cartesian mesh (Sec. 2.3).  Velocity rows: nu a_h(u, v) + (p, div v);
 * pressure rows: (q, div u).  x and y must not alias. */
int stk_apply(stk_problem* P, int level, int dtype, const void* x, void* y);

/* One of the two kernels of stk_apply (Algorithm 1 split by test space): stage
 * 0 writes the velocity rows of y = A x, stage 1 the pressure rows; the other rows of y are left untouched.
 * Calling stage 0 then stage 1 is exactly stk_apply.  Lets a caller time the
 * two kernels separately on the library's stream. */
int stk_apply_stage(stk_problem* P, int level, int dtype, int stage, const void* x, void* y);

/* r = b - A x on one level (the residual of Algorithm 2).  r may alias b but
 * not x. */
int stk_residual(stk_problem* P, int level, int dtype, const void* x, const void* b, void* r);

/* xf += I^up xc: prolongation from level fine_level - 1 to fine_level by the
 * canonical embedding of the nested spaces X_{l-1} in X_l (Sec. 3).  xc has
 * the layout of the coarser level.  xc and xf must not alias. */
int stk_prolongate_add(stk_problem* P, int fine_level, int dtype, const void* xc, void* xf);

/* rc = I^down rf: residual restriction from fine_level to fine_level - 1, the
 * transpose of stk_prolongate_add (Sec. 3 calls it an l2-projection; the
 * transpose is the reading used here).  rc is overwritten. */
int stk_restrict(stk_problem* P, int fine_level, int dtype, const void* rf, void* rc);

/* One step x <- S_l(x, b) of the coloured vertex-patch multiplicative Schwarz
 * smoother (Algorithm 2, Sec. 3.1): for each of the 8 colours (ascending), the
 * residual r = b - A x, then on every patch of the colour in parallel the
 * local solve of Sec. 3.2 (Schur-complement CG with fast-diagonalization
 * A_j^{-1}; stk_options.local_cg_mode / local_cg_iters / local_cg_tol) and
 * x += R_j^T (U, P).  x is updated in place.  The first call for a dtype
 * allocates that dtype's multigrid workspace (three vectors per level). */
int stk_smooth(stk_problem* P, int level, int dtype, void* x, const void* b);

/* One colour of the smoothing step of Algorithm 2 (Sec. 3.1): r = b - A x
 * for the current x, then on every patch of colour `colour` (0..7, the
 * colour (i mod 2) + 2 (j mod 2) + 4 (l mod 2) of the patch's vertex (i, j, l))
 * the local solve of Sec. 3.2 and x += R_j^T (U, P).  Calling it for the
 * colours 0..7 in turn is exactly stk_smooth.  Same workspace, options and
 * errors as stk_smooth; STK_EINVAL for a colour outside 0..7. */
int stk_smooth_colour(stk_problem* P, int level, int dtype, int colour, void* x, const void* b);

/* One smoothing step (as stk_smooth: Algorithm 2, Sec. 3.1) of `count`
 * problems of the same degree k, batched (the merged launches have no
 * counterpart in the paper, which smooths one problem): per colour, every problem's colour residual, then ONE launch of
 * the patch kernel over that colour's patches of all the problems (64
 * problems per launch).  levels[i]: the level smoothed in problem i; x[i],
 * b[i]: its vectors, as in stk_smooth.  All work runs on problems[0]'s
 * stream, whose caller orders the other problems' streams before the call;
 * the local-solver options of problems[0] apply to all.  The result equals
 * `count` separate stk_smooth calls bitwise.  Errors: STK_EINVAL for NULL or
 * empty arguments, mixed degrees, a repeated problem, aliasing x[i] and b[i]
 * (stk_last_error(NULL) says which); nothing is launched then. */
int stk_smooth_batch(stk_problem* const* problems, int count, const int* levels, int dtype, void* const* x,
                     const void* const* b);

/* x = A_0^+ b on level 0 (the exact coarse solve P_0^{-1} = A_0^{-1} of
 * Sec. 3; the pressure null space is removed: the result is the
 * pseudo-inverse with mean-free pressure coefficients), always computed in
 * FP64.  On a 2^3 coarse mesh (n = 2^L) the first call builds the dense
 * pseudo-inverse (one exact patch solve per coarse DoF); on a 3^3 mesh
 * (n = 3 * 2^L) it builds dense inverses of the three velocity blocks and of
 * the pressure Schur complement (shared by every problem of the process with
 * the same device, degree, viscosity and penalty factor) and solves by block
 * elimination.  The first call is synchronous. */
int stk_coarse_solve(stk_problem* P, int dtype, const void* b, void* x);

/* x = P_L^{-1} b on the finest level: one V-cycle with x0 = 0, one pre- and
 * one post-smoothing step, residual restriction, exact coarse solve and
 * prolongation (Sec. 3).  Every level runs in dtype; the coarse solve always
 * runs in FP64.  The hierarchy ends on 2^3 (n = 2^L) or 3^3 (n = 3 * 2^L)
 * cells.  b and x must not alias. */
int stk_vcycle(stk_problem* P, int dtype, const void* b, void* x);

/* Solve A x = b to ||b - A x||_2 <= rtol ||b||_2 by flexible GMRES(restart)
 * right-preconditioned by one V-cycle, x0 = 0 (Sec. 3.3).  With
 * STK_PREC_MIXED the V-cycle runs in FP32 inside the FP64 Krylov method, with
 * conversions on entry and exit (Sec. 4.3).  b and x are FP64 device vectors;
 * the returned pressure has zero L2 mean.  Synchronous on the stream: the host
 * reads the Arnoldi coefficients every iteration.  info may be NULL.  Returns
 * STK_ENOCONV (x holds the last iterate, info filled) when max_iter is reached
 * first.  The first call allocates the Krylov basis (2 restart + 1 vectors). */
int stk_solve(stk_problem* P, const double* b, double* x, double rtol, stk_solve_info* info);

/* Solve `count` independent problems (each with its own setup, mesh, degree
 * and options) to ||b_i - A_i x_i|| <= rtol ||b_i||, by the same method as
 * stk_solve (Sec. 3.3; batching has no counterpart in the paper), with
 * bitwise the same results.  The host interleaves the
 * solves: it polls the problems' streams and, as soon as one has drained,
 * advances that problem's Krylov state and enqueues its next step, so
 * problems on distinct non-NULL streams run concurrently on the GPU (many
 * small problems fill the GPU that one alone cannot; the V-cycles replay
 * captured CUDA graphs).  b[i], x[i]: FP64 device vectors of problem i's finest level.
 * infos may be NULL, else count entries.  Synchronous.  Returns STK_OK,
 * STK_ENOCONV if any solve reached its max_iter, or the first other error;
 * stk_last_error(NULL) names the failing problem.  No problem may appear
 * twice and x[i] must not alias b[i] (STK_EINVAL before any launch). */
int stk_solve_batch(stk_problem* const* problems, int count, const double* const* b, double* const* x, double rtol,
                    stk_solve_info* infos);

/* Autotuner (no counterpart in the paper): for every level, time the operator
 * apply in `dtype` with each candidate run length of its velocity kernel's
 * persistent march (cells per run along the continuous direction: n, then
 * halving down to 2) on the problem's stream and keep the
 * fastest, then, on every level that is smoothed, one smoothing step in each
 * form (fused_smoother 0 and 1, with the problem's local solver) and keep
 * the faster, then, in that form, one step with the interior patches of a
 * colour in their own launch and one without, and keep the faster (levels
 * whose interior eigenbases are symmetric); every later apply, residual,
 * smoothing step and solve of that
 * dtype uses them (a V-cycle graph that an earlier solve captured in that
 * dtype is discarded, so the next solve captures the tuned launches).
 * Synchronous; allocates and frees two vectors per level (and builds the
 * Direct local inverses of a level if that is the local solver). */
int stk_autotune(stk_problem* P, int dtype);

/* The smoother form chosen by stk_autotune for a level and dtype: 0 split,
 * 1 fused, -1 not tuned (stk_options.fused_smoother applies); no counterpart
 * in the paper. */
int stk_tuned_smoother(const stk_problem* P, int level, int dtype, int* fused);

/* Whether stk_autotune put the interior patches of a colour in their own
 * launch on a level and dtype: 1 yes, 0 no, -1 not tuned (the built-in rule:
 * from 8192 interior patches per colour in FP64, 1024 in FP32);
 * no counterpart in the paper. */
int stk_tuned_split(const stk_problem* P, int level, int dtype, int* split);

/* The run length chosen by stk_autotune (or set by stk_set_tuning) for a
 * level and dtype (0 = not tuned: the built-in choice is used, whole columns
 * in FP64, about 8 CTAs per SM in FP32); no counterpart in the paper. */
int stk_tuning(const stk_problem* P, int level, int dtype, int* cells_per_run);

/* Set the run length of the apply's persistent march for a level and dtype
 * (cells per run along the continuous direction; 0 restores the built-in
 * choice; values above n act as n); for reusing a tuning found earlier.
 * Drops the problem's captured graphs of that dtype (synchronises its
 * stream).  STK_EINVAL for a bad level, dtype or a negative value; 2D
 * problems have no such tuning (STK_EINVAL); no counterpart in the paper. */
int stk_set_tuning(stk_problem* P, int level, int dtype, int cells_per_run);

/* b = right-hand side of a manufactured problem on the finest level
 * (Sec. 3.3): velocity rows (f, phi_i) with f = -nu Laplace(u) + grad p and
 * u = curl(psi), by the (k+3)-point Gauss rule of every cell; pressure rows
 * and constrained rows are 0.  HOST arrays: psi_freq[3][3][3] frequencies
 * (component, term, direction) in 1..8 and psi_amp[3][3] amplitudes of
 *   psi_c = sum_t psi_amp[c][t] G_a(x) G_b(y) G_c(z),  G_a(s) = s^2 (1-s)^2 sin(a pi s);
 * p_freq[3][3], p_amp[3] of  p = sum_t p_amp[t] cos(a pi x) cos(b pi y) cos(c pi z).
 * The discrete pressure approximates -p because the velocity rows carry
 * +(p, div v) (eq. `weak_form`).  b is a FP64 device vector, overwritten.
 * Two-dimensional problems use the first component's terms as the stream
 * function, psi = sum_t psi_amp[0][t] G_a(x) G_b(y) with (a, b) =
 * psi_freq[0][t][0..1], u = (d_y psi, -d_x psi), and p = sum_t p_amp[t]
 * cos(a pi x) cos(b pi y) with (a, b) = p_freq[t][0..1]: with one term a = b = 1
 * and p = cos(2 pi x) cos(2 pi y) this is the paper's 2D reference solution
 * (Sec. 3.3) with the bump G_1 in place of its unstated phi. */
int stk_rhs(stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq, const double* p_amp,
            double* b);

/* stk_smooth without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not call cudaMalloc, such as
 * a framework whose memory pool must own every device allocation (a foreign
 * cudaMalloc escapes its accounting and can fail once the pool holds the
 * memory), or a real-time loop that cannot absorb the device synchronisation
 * a cudaMalloc may cause.  Same kernels, same
 * order and same result as stk_smooth; the colour residual lives in a 32 MiB
 * array of device global memory built into the library (every GPU that loads
 * the library holds it until exit), so the level must have
 * N * sizeof(dtype) <= 33554432 bytes, else STK_EINVAL with a message.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race and must be ordered by
 * the caller.  Nothing in the array needs clearing between calls.  With the
 * Direct local solver the level's inverses must exist already (built by a
 * stk_smooth call on it), else STK_ESTATE. */
int stk_smooth_static(stk_problem* P, int level, int dtype, void* x, const void* b);

#ifdef __cplusplus
}
#endif

#endif /* STOKESMG_H */
