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
  STK_ETIMEOUT = -5, /* a bounded device-side wait ran out                               */
  STK_ESTATE = -6    /* call not valid in the current state                              */
};

enum { STK_F64 = 0, STK_F32 = 1 };
enum { STK_PREC_FP64 = 0, STK_PREC_MIXED = 1 };
/* Local solver of the patch smoother (Sec. 3.2): conjugate gradients on the
 * pressure Schur complement with a fixed number of steps, or until a relative
 * tolerance is met. */
enum { STK_CG_FIXED = 0, STK_CG_TOL = 1 };

typedef struct stk_options {
  int precision;         /* STK_PREC_FP64 or STK_PREC_MIXED (V-cycle in FP32, Sec. 4.3) */
  int gmres_restart;     /* restart length of the flexible GMRES, default 20           */
  int max_iter;          /* total GMRES iteration limit, default 200                    */
  int local_cg_mode;     /* STK_CG_FIXED (default) or STK_CG_TOL                       */
  int local_cg_iters;    /* CG steps in FIXED mode, step limit in TOL mode; default 15 */
  double local_cg_tol;   /* relative CG residual in TOL mode, default 1e-8              */
  double penalty_factor; /* gamma = penalty_factor (k+1)(k+2)/h, default 1             */
  void* stream;          /* cudaStream_t used by every call, NULL = default stream     */
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

/* Fill *opt with the defaults listed above.  Returns STK_EINVAL if opt is NULL. */
int stk_default_options(stk_options* opt);

/* Build the mesh hierarchy, the 1D tables of every level (Sec. 2.3, Sec. 3.2)
 * and all device workspace, for the unit cube with n cells per side, degree k
 * and viscosity nu (Sec. 2, eq. `model` and eq. `weak_form`).  n must be 2 or
 * 3 times a power of two (n >= 2); k in 1..5; nu > 0.  opt may be NULL
 * (defaults).  On success *out owns device memory until stk_destroy.
 * Synchronous. */
int stk_setup(int n, int k, double nu, const stk_options* opt, stk_problem** out);

/* Release everything stk_setup allocated.  NULL is accepted. */
int stk_destroy(stk_problem* P);

/* Message of the last failed call on P (or of the last failed stk_setup when
 * P is NULL).  The string stays valid until the next call on P. */
const char* stk_last_error(const stk_problem* P);

/* Number of levels of the hierarchy. */
int stk_num_levels(const stk_problem* P, int* nlevels);

/* Cells per side, per-velocity-component length, pressure length and total
 * length N of the vectors of one level. */
int stk_layout(const stk_problem* P, int level, int* n_cells, int64_t* n_vel_component,
               int64_t* n_pressure, int64_t* n_total);

/* y = A x on one level: the matrix-free Stokes operator of Algorithm 1 (cell,
 * interior-face and boundary-face loops of eq. `bilinear`, with the divergence
 * blocks of eq. `weak_form`), evaluated through its Kronecker form on the
 * Cartesian mesh (Sec. 2.3).  Velocity rows: nu a_h(u, v) + (p, div v);
 * pressure rows: (q, div u).  x and y must not alias. */
int stk_apply(stk_problem* P, int level, int dtype, const void* x, void* y);

/* One of the two kernels of stk_apply: stage 0 writes the velocity rows of
 * y = A x, stage 1 the pressure rows; the other rows of y are left untouched.
 * Calling stage 0 then stage 1 is exactly stk_apply.  Lets a caller time the
 * two kernels separately on the library's stream. */
int stk_apply_stage(stk_problem* P, int level, int dtype, int stage, const void* x, void* y);

/* r = b - A x on one level (the residual of Algorithm 2).  r may alias b but
 * not x. */
int stk_residual(stk_problem* P, int level, int dtype, const void* x, const void* b, void* r);

#ifdef __cplusplus
}
#endif

#endif /* STOKESMG_H */
