// Host orchestration of the multigrid method and the outer Krylov solver,
// plus the BLAS-1 kernels they need.
//
//  smooth  (Algorithm 2): for each colour, r = b - A x, then the patch kernel.
//  vcycle  (Sec. 3): pre-smooth, residual, restriction, recursion, exact
//          coarse solve on the 2^3 or 3^3 mesh, prolongation-add, post-smooth; x0 = 0.
//  solve   (Sec. 3.3, Sec. 4.3): flexible GMRES(restart), right preconditioned
//          by one V-cycle, x0 = 0, stopping at ||b - A x|| <= rtol ||b||.  In
//          mixed precision the V-cycle runs in FP32 and everything else in
//          FP64; vectors are converted on entry to and exit from the V-cycle.
//          Orthogonalization is classical Gram-Schmidt applied twice (one
//          batched dot kernel and one batched update per pass), equal to
//          modified Gram-Schmidt in exact arithmetic.
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>

#include "internal.h"

namespace stk {

constexpr int kRedBlocks = 2 * 152;
constexpr int kRedThreads = 256;
constexpr int kMaxBasis = 64;

// ------------------------------------------------------------------ kernels
template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

// partial[b] = block b's share of a . w (one scalar accumulator per thread)
__global__ void __launch_bounds__(kRedThreads) dot_kernel(const double* __restrict__ a, const double* __restrict__ w,
                                                          int64_t n, double* __restrict__ partial) {
  __shared__ double red[kRedThreads / 32];
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc += a[e] * w[e];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) s += red[q];
    partial[blockIdx.x] = s;
  }
}

// out[i] = sum_b partial[b * nv + i]  (fixed order: deterministic)
__global__ void finish_dot_kernel(const double* __restrict__ partial, int nblocks, int nv, double* __restrict__ out,
                                  int accumulate) {
  const int i = threadIdx.x;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * nv + i];
  out[i] = accumulate ? out[i] + s : s;
}

// sum_i W_i p_i and sum_i W_i over the pressure block (W = Gauss weight products)
__global__ void __launch_bounds__(kRedThreads) pressure_mean_partial(const double* __restrict__ p, int m, int nd,
                                                                      const double* __restrict__ S,
                                                                      double* __restrict__ partial) {
  __shared__ double red[2][kRedThreads / 32];
  const int64_t np = (int64_t)m * m * m;
  double a = 0.0, b = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(e % m), i1 = (int)((e / m) % m), i2 = (int)(e / ((int64_t)m * m));
    const double w = S[i0 % nd] * S[i1 % nd] * S[i2 % nd];
    a += w * p[e];
    b += w;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) s += red[threadIdx.x][q];
    partial[blockIdx.x * 2 + threadIdx.x] = s;
  }
}

__global__ void pressure_shift(double* __restrict__ p, int64_t np, const double* __restrict__ partial, int nblocks) {
  double a = 0.0, b = 0.0;
  for (int q = 0; q < nblocks; ++q) {
    a += partial[2 * q];
    b += partial[2 * q + 1];
  }
  const double mean = a / b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.x * blockDim.x)
    p[e] -= mean;
}

static int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 8); }

// --------------------------------------------------------------- workspace
static void free_all(std::vector<void*>& v) {
  for (void*& p : v)
    if (p) {
      cudaFree(p);
      p = nullptr;
    }
}

// A failed allocation leaves the workspace empty (nothing leaks, a later
// call starts over).
cudaError_t ensure_mg_workspace(stk_problem* P, int dtype) {
  MgWork& W = P->mg[dtype];
  if (W.ready) return cudaSuccess;
  const size_t es = dtype == STK_F64 ? 8 : 4;
  const int nl = (int)P->levels.size();
  W.r.assign(nl, nullptr);
  W.b.assign(nl, nullptr);
  W.x.assign(nl, nullptr);
  for (int l = 0; l < nl; ++l) {
    const size_t bytes = (size_t)P->levels[l].ntotal * es;
    cudaError_t e = dev_alloc(&W.r[l], bytes);
    if (e == cudaSuccess) e = dev_alloc(&W.b[l], bytes);
    if (e == cudaSuccess) e = dev_alloc(&W.x[l], bytes);
    if (e != cudaSuccess) {
      free_all(W.r);
      free_all(W.b);
      free_all(W.x);
      return e;
    }
  }
  W.ready = true;
  return cudaSuccess;
}

cudaError_t ensure_coarse(stk_problem* P) {
  if (P->dim == 2) return cudaSuccess;  // the 2D coarse solve uses the patch inverses built at setup
  if (P->levels[0].n != 2) {
    // 3^3 coarse mesh: FP64 vectors and the dense block factors
    if (P->coarse3f) return cudaSuccess;
    const size_t bytes = sizeof(double) * (size_t)P->levels[0].ntotal;
    for (int i = 0; i < 3; ++i) {
      if (P->coarse3[i]) continue;
      cudaError_t e = dev_alloc(&P->coarse3[i], bytes);
      if (e != cudaSuccess) return e;
    }
    return acquire_coarse3(P);
  }
  if (P->coarse_inv) return cudaSuccess;
  const int NL = patch_local_size(P->k);
  cudaError_t e = dev_alloc(&P->coarse_inv, sizeof(double) * (size_t)NL * NL);
  if (e != cudaSuccess) return e;
  // every free coarse DoF's pseudo-inverse column: CG on the Schur complement to 1e-14
  e = launch_coarse_columns(P, P->coarse_inv, 2000, 1e-14);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) {  // no half-built inverse survives a failure
    cudaFree(P->coarse_inv);
    P->coarse_inv = nullptr;
  }
  return e;
}

// ---------------------------------------------------------------- smoother
// Algorithm 2 on one level.  Split form: per colour, r = b - A x over the
// whole level, then the colour's patch kernel reads R_j r.  Fused form
// (opt.fused_smoother): the patch kernel computes R_j (b - A x) itself; since
// all patches of a colour must see the x from before the colour, the colours
// alternate between x and the level's residual buffer as input and output
// (x -> tmp -> x ... : eight colours end in x), and the entries no patch of
// the colour owns are copied across.
cudaError_t run_smooth(stk_problem* P, int level, int dtype, void* x, const void* b) {
  cudaError_t e = ensure_mg_workspace(P, dtype);
  if (P->dim == 2) {  // four colours, exact local solver, split form
    if (e != cudaSuccess) return e;
    void* r = P->mg[dtype].r[level];
    for (int colour = 0; colour < 4 && e == cudaSuccess; ++colour) {
      e = launch_apply(P, level, dtype, x, b, r, -1.0);
      if (e == cudaSuccess) e = launch_patch_colour_planar(P, level, dtype, colour, r, x);
    }
    return e;
  }
  if (e == cudaSuccess && P->opt.local_cg_mode == STK_LOCAL_DIRECT) e = ensure_direct(P, level);
  if (e != cudaSuccess) return e;
  void* r = P->mg[dtype].r[level];
  const int pick = P->levels[level].fused_pick[dtype];
  const bool fused = pick >= 0 ? pick == 1 : P->opt.fused_smoother != 0;
  for (int colour = 0; colour < 8; ++colour) {
    if (fused) {
      void* xin = (colour % 2 == 0) ? x : r;
      void* xout = (colour % 2 == 0) ? r : x;
      e = launch_copy_unowned(P, level, dtype, colour, xin, xout);
      if (e == cudaSuccess) e = launch_patch_colour_fused(P, level, dtype, colour, xin, b, xout);
    } else {
      e = launch_apply(P, level, dtype, x, b, r, -1.0);
      if (e == cudaSuccess) e = launch_patch_colour(P, level, dtype, colour, r, x);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One colour of Algorithm 2: r = b - A x, then the colour's patch solves
// (fused form: x is copied to the residual buffer, which is the colour's input).
cudaError_t run_smooth_colour(stk_problem* P, int level, int dtype, int colour, void* x, const void* b) {
  cudaError_t e = ensure_mg_workspace(P, dtype);
  if (P->dim == 2) {
    if (e != cudaSuccess) return e;
    void* r2 = P->mg[dtype].r[level];
    e = launch_apply(P, level, dtype, x, b, r2, -1.0);
    if (e == cudaSuccess) e = launch_patch_colour_planar(P, level, dtype, colour, r2, x);
    return e;
  }
  if (e == cudaSuccess && P->opt.local_cg_mode == STK_LOCAL_DIRECT) e = ensure_direct(P, level);
  if (e != cudaSuccess) return e;
  void* r = P->mg[dtype].r[level];
  if (P->opt.fused_smoother) {
    const size_t bytes = (size_t)P->levels[level].ntotal * (dtype == STK_F64 ? 8 : 4);
    e = cudaMemcpyAsync(r, x, bytes, cudaMemcpyDeviceToDevice, P->stream);
    if (e == cudaSuccess) e = launch_patch_colour_fused(P, level, dtype, colour, r, b, x);
    return e;
  }
  e = launch_apply(P, level, dtype, x, b, r, -1.0);
  if (e == cudaSuccess) e = launch_patch_colour(P, level, dtype, colour, r, x);
  return e;
}

// One smoothing step of several problems of the same degree, all on the first
// problem's stream: per colour, every problem's colour residual, then one
// patch launch over the colour's patches of all of them.
cudaError_t run_smooth_batch(stk_problem* const* Ps, const int* levels, int count, int dtype, void* const* x,
                             const void* const* b) {
  const cudaStream_t s = Ps[0]->stream;
  if (Ps[0]->opt.local_cg_mode == STK_LOCAL_DIRECT) {
    // the Direct local inverses belong to each problem's level: one launch per problem
    for (int i = 0; i < count; ++i) {
      stk_problem* P = Ps[i];
      const cudaStream_t own = P->stream;
      P->stream = s;
      const cudaError_t e = run_smooth(P, levels[i], dtype, x[i], b[i]);
      P->stream = own;
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  std::vector<void*> r(count);
  for (int i = 0; i < count; ++i) {
    cudaError_t e = ensure_mg_workspace(Ps[i], dtype);
    if (e != cudaSuccess) return e;
    r[i] = Ps[i]->mg[dtype].r[levels[i]];
  }
  for (int colour = 0; colour < 8; ++colour) {
    for (int i = 0; i < count; ++i) {
      cudaError_t e = launch_apply_on(Ps[i], levels[i], dtype, x[i], b[i], r[i], -1.0, 3, s);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_patch_colour_multi(Ps, levels, count, dtype, colour, r.data(), x, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Coarse solve P_0^{-1} (Sec. 3), exact in FP64 whatever the V-cycle's
// precision.  On the 2^3 mesh: the dense pseudo-inverse.  On a 3^3 mesh
// (n = 3 * 2^L): block elimination with dense factors of the velocity blocks
// and of the pressure Schur complement (coarse3.cu), after the pressure rows
// of the right-hand side are made to sum to zero.
template <typename S, typename D>
__global__ void copy_convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

// Remove the mean of the pressure rows (one CTA; the coarse pressure block is
// small): the bordered coarse system maps the right-hand side's pressure
// mean to its multiplier, so the block elimination sees a consistent system.
__global__ void __launch_bounds__(256) remove_pressure_sum(double* __restrict__ p, int64_t np) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) s += p[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < 8; ++w) t += red[w];
  const double mean = t / (double)np;
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) p[i] -= mean;
}

static cudaError_t coarse_level_solve(stk_problem* P, int dtype, const void* b, void* x) {
  if (P->dim == 2) return launch_coarse_solve_planar(P, dtype, b, x);
  if (P->levels[0].n == 2) return launch_coarse_solve(P, dtype, b, x);
  const int64_t n = P->levels[0].ntotal;
  double *cb = P->coarse3[0], *cx = P->coarse3[1];
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 1024);
  if (dtype == STK_F64)
    copy_convert_kernel<double, double><<<grid, 256, 0, P->stream>>>((const double*)b, cb, n);
  else
    copy_convert_kernel<float, double><<<grid, 256, 0, P->stream>>>((const float*)b, cb, n);
  remove_pressure_sum<<<1, 256, 0, P->stream>>>(cb + 3 * P->levels[0].nvel, P->levels[0].npress);
  cudaError_t e = coarse3_solve(P);
  if (e != cudaSuccess) return e;
  if (dtype == STK_F64)
    copy_convert_kernel<double, double><<<grid, 256, 0, P->stream>>>(cx, (double*)x, n);
  else
    copy_convert_kernel<double, float><<<grid, 256, 0, P->stream>>>(cx, (float*)x, n);
  return cudaGetLastError();
}

static cudaError_t vcycle_rec(stk_problem* P, int level, int dtype, const void* b, void* x) {
  cudaError_t e;
  if (level == 0) return coarse_level_solve(P, dtype, b, x);
  const size_t es = dtype == STK_F64 ? 8 : 4;
  MgWork& W = P->mg[dtype];
  e = cudaMemsetAsync(x, 0, (size_t)P->levels[level].ntotal * es, P->stream);
  if (e == cudaSuccess) e = run_smooth(P, level, dtype, x, b);
  if (e == cudaSuccess) e = launch_apply(P, level, dtype, x, b, W.r[level], -1.0);
  if (e == cudaSuccess) e = launch_restrict(P, level, dtype, W.r[level], W.b[level - 1]);
  if (e == cudaSuccess) e = vcycle_rec(P, level - 1, dtype, W.b[level - 1], W.x[level - 1]);
  if (e == cudaSuccess) e = launch_prolongate_add(P, level, dtype, W.x[level - 1], x);
  if (e == cudaSuccess) e = run_smooth(P, level, dtype, x, b);
  return e;
}

cudaError_t run_vcycle(stk_problem* P, int dtype, const void* b, void* x) {
  cudaError_t e = ensure_mg_workspace(P, dtype);
  if (e == cudaSuccess) e = ensure_coarse(P);
  if (e != cudaSuccess) return e;
  return vcycle_rec(P, (int)P->levels.size() - 1, dtype, b, x);
}

cudaError_t run_coarse_solve(stk_problem* P, int dtype, const void* b, void* x) {
  cudaError_t e = ensure_coarse(P);
  if (e != cudaSuccess) return e;
  return coarse_level_solve(P, dtype, b, x);
}

// -------------------------------------------------------------------- FGMRES
// Flexible GMRES(restart), right preconditioned by one V-cycle, x0 = 0
// (Sec. 3.3), with its whole scalar recurrence on the device: the Arnoldi
// coefficients, the Givens rotations, the least-squares update and the
// stopping tests live in a GmresState in device memory and are advanced by
// single-thread kernels, and every kernel that depends on the step j reads it
// from there.  So the same launch sequence runs two ways: driven by the host,
// which reads a few flags after each step (no stream, or graphs off), or as
// one CUDA graph per solve whose two loops are conditional WHILE nodes set by
// those kernels: a solve is then one graph launch and one read at the end.
// Both ways run the same kernels in the same order: bitwise the same result.

struct GmresState {
  // flags the host reads while it drives the loop (first 64 bytes)
  int j;          // current Arnoldi step of the cycle
  int its;        // steps so far
  int jdone;      // steps of the current cycle
  int stop;       // the cycle ends after this step
  int converged;  // true residual below rtol ||b||
  int more;       // another cycle follows
  int m, max_iter;
  double bnorm, beta, hn, rtol;
  double H[(kMaxBasis + 1) * kMaxBasis];  // H[i * kMaxBasis + col]
  double cs[kMaxBasis], sn[kMaxBasis], g[kMaxBasis + 1], y[kMaxBasis];
  double res[256];  // relative residual estimate after each step, res[0] = 1
};
constexpr size_t kStateFlags = 64;

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, unsigned v) {
  if (use) cudaGraphSetConditional(h, v);
}

// bnorm = ||b|| from h[0]; start of the first cycle
__global__ void gm_start_kernel(GmresState* st, const double* __restrict__ h, double rtol, int m, int max_iter,
                                cudaGraphConditionalHandle hout, int use) {
  st->m = m;
  st->max_iter = max_iter;
  st->rtol = rtol;
  st->bnorm = sqrt(h[0]);
  st->beta = st->bnorm;
  st->its = 0;
  st->j = 0;
  st->jdone = 0;
  st->stop = 0;
  st->converged = st->bnorm == 0.0;
  st->more = !st->converged;
  st->res[0] = 1.0;
  set_cond(hout, use, st->more ? 1u : 0u);
}

// dst = src / beta (V_0 of a cycle); nothing when no cycle follows
__global__ void gm_scale_kernel(const double* __restrict__ src, double* __restrict__ dst, const GmresState* st,
                                int64_t n) {
  if (!st->more) return;
  const double inv = 1.0 / st->beta;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e] * inv;
}

__global__ void gm_cycle_begin_kernel(GmresState* st, cudaGraphConditionalHandle hin, int use) {
  st->j = 0;
  st->stop = 0;
  for (int i = 0; i < (kMaxBasis + 1) * kMaxBasis; ++i) st->H[i] = 0.0;
  for (int i = 0; i <= kMaxBasis; ++i) st->g[i] = 0.0;
  st->g[0] = st->beta;
  set_cond(hin, use, 1u);
}

// dst = (T) V_j
template <typename T>
__global__ void gm_copy_in_kernel(const double* __restrict__ V, const GmresState* st, int64_t n, T* __restrict__ dst) {
  const double* v = V + (int64_t)st->j * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (T)v[e];
}

// Z_j = z (and zbuf = z, the apply's fixed input, when z is FP32)
template <typename T>
__global__ void gm_copy_out_kernel(const T* __restrict__ z, double* __restrict__ Z, const GmresState* st, int64_t n,
                                   double* __restrict__ zbuf) {
  double* zj = Z + (int64_t)st->j * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)z[e];
    zj[e] = v;
    if (zbuf) zbuf[e] = v;
  }
}

// partial[b * nv + i] = block b's share of V_i . w, i <= j (nv = j + 1 from the state)
__global__ void __launch_bounds__(kRedThreads) gm_multidot_kernel(const double* __restrict__ V, const GmresState* st,
                                                                   const double* __restrict__ w, int64_t n,
                                                                   double* __restrict__ partial) {
  __shared__ double red[kRedThreads / 32][kMaxBasis];
  const int nv = st->j + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // the basis vectors in chunks of 8 accumulators per thread (registers, no local array)
  for (int i0 = 0; i0 < nv; i0 += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const double we = w[e];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u < nv) acc[u] += V[(int64_t)(i0 + u) * n + e] * we;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double v = acc[u];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && i0 + u < nv) red[wid][i0 + u] = v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) s += red[q][i];
    partial[(int64_t)blockIdx.x * kMaxBasis + i] = s;
  }
}

// out[i] = sum over blocks, fixed order (deterministic); nv = j + 1, or 1 when `one`
__global__ void gm_finish_dot_kernel(const double* __restrict__ partial, int nblocks, const GmresState* st, int one,
                                     double* __restrict__ out) {
  const int nv = one ? 1 : st->j + 1;
  const int i = threadIdx.x;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * kMaxBasis + i];
  out[i] = s;
}

// w -= sum_{i <= j} h[i] V_i
__global__ void gm_axpy_kernel(double* __restrict__ w, const double* __restrict__ V, const GmresState* st,
                               const double* __restrict__ h, int64_t n) {
  __shared__ double hs[kMaxBasis];
  const int nv = st->j + 1;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = w[e];
    for (int i = 0; i < nv; ++i) s -= hs[i] * V[(int64_t)i * n + e];
    w[e] = s;
  }
}

// one Arnoldi step on the device: column j of H from the two Gram-Schmidt
// passes (h[i] + h[kMaxBasis + i]) and the norm (h[2 kMaxBasis]), the earlier
// Givens rotations, a new one, the residual estimate and the stopping test
__global__ void gm_arnoldi_kernel(GmresState* st, const double* __restrict__ h, cudaGraphConditionalHandle hin,
                                  int use) {
  const int j = st->j, m = st->m;
  double* H = st->H;
  for (int i = 0; i <= j; ++i) H[i * kMaxBasis + j] = h[i] + h[kMaxBasis + i];
  const double hn = sqrt(h[2 * kMaxBasis]);
  H[(j + 1) * kMaxBasis + j] = hn;
  st->hn = hn;
  for (int i = 0; i < j; ++i) {
    const double t = st->cs[i] * H[i * kMaxBasis + j] + st->sn[i] * H[(i + 1) * kMaxBasis + j];
    H[(i + 1) * kMaxBasis + j] = -st->sn[i] * H[i * kMaxBasis + j] + st->cs[i] * H[(i + 1) * kMaxBasis + j];
    H[i * kMaxBasis + j] = t;
  }
  const double den = hypot(H[j * kMaxBasis + j], H[(j + 1) * kMaxBasis + j]);
  st->cs[j] = H[j * kMaxBasis + j] / den;
  st->sn[j] = H[(j + 1) * kMaxBasis + j] / den;
  H[j * kMaxBasis + j] = den;
  H[(j + 1) * kMaxBasis + j] = 0.0;
  st->g[j + 1] = -st->sn[j] * st->g[j];
  st->g[j] = st->cs[j] * st->g[j];
  st->its += 1;
  st->jdone = j + 1;
  if (st->its < 256) st->res[st->its] = fabs(st->g[j + 1]) / st->bnorm;
  const int stop = fabs(st->g[j + 1]) <= st->rtol * st->bnorm || st->its >= st->max_iter || j + 1 == m;
  st->stop = stop;
  if (!stop) st->j = j + 1;
  set_cond(hin, use, stop ? 0u : 1u);
}

// V_{jdone} = w / hn (the next basis vector; harmless when the cycle stops)
__global__ void gm_normalize_kernel(double* __restrict__ V, const double* __restrict__ w, const GmresState* st,
                                    int64_t n) {
  double* v = V + (int64_t)st->jdone * n;
  const double inv = 1.0 / st->hn;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    v[e] = w[e] * inv;
}

// y = H^{-1} g on the cycle's jdone steps (upper triangular)
__global__ void gm_solve_y_kernel(GmresState* st) {
  const int jd = st->jdone;
  for (int i = jd - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int l = i + 1; l < jd; ++l) s -= st->H[i * kMaxBasis + l] * st->y[l];
    st->y[i] = s / st->H[i * kMaxBasis + i];
  }
}

// x += sum_{i < jdone} y_i Z_i
__global__ void gm_update_x_kernel(double* __restrict__ x, const double* __restrict__ Z, const GmresState* st,
                                   int64_t n) {
  __shared__ double ys[kMaxBasis];
  const int jd = st->jdone;
  for (int i = threadIdx.x; i < jd; i += blockDim.x) ys[i] = st->y[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = x[e];
    for (int i = 0; i < jd; ++i) s += ys[i] * Z[(int64_t)i * n + e];
    x[e] = s;
  }
}

// the true residual's norm (h[0]) decides: converged, or another cycle
__global__ void gm_restart_kernel(GmresState* st, const double* __restrict__ h, cudaGraphConditionalHandle hout,
                                  int use) {
  st->beta = sqrt(h[0]);
  st->converged = st->beta <= st->rtol * st->bnorm;
  st->more = !st->converged && st->its < st->max_iter;
  set_cond(hout, use, st->more ? 1u : 0u);
}

cudaError_t ensure_krylov(stk_problem* P) {
  KrylovWork& K = P->kry;
  const int m = P->opt.gmres_restart;
  if (K.ready) return cudaSuccess;
  const int64_t n = P->levels.back().ntotal;
  cudaError_t e = dev_alloc(&K.V, sizeof(double) * (size_t)(m + 1) * n);
  if (e == cudaSuccess) e = dev_alloc(&K.Z, sizeof(double) * (size_t)m * n);
  if (e == cudaSuccess) e = dev_alloc(&K.w, sizeof(double) * (size_t)n);
  if (e == cudaSuccess && P->opt.precision == STK_PREC_MIXED) e = dev_alloc(&K.zbuf, sizeof(double) * (size_t)n);
  if (e == cudaSuccess) e = dev_alloc(&K.partial, sizeof(double) * (size_t)kRedBlocks * kMaxBasis);
  if (e == cudaSuccess) e = dev_alloc(&K.h, sizeof(double) * (2 * kMaxBasis + 2));
  if (e == cudaSuccess) e = dev_alloc(&K.state, sizeof(GmresState));
  if (e == cudaSuccess) e = host_alloc_pinned(&K.state_host, sizeof(GmresState));
  if (e != cudaSuccess) {  // leave nothing half allocated
    for (double** d : {&K.V, &K.Z, &K.w, &K.zbuf, &K.partial, &K.h})
      if (*d) {
        cudaFree(*d);
        *d = nullptr;
      }
    if (K.state) cudaFree(K.state);
    K.state = nullptr;
    if (K.state_host) cudaFreeHost(K.state_host);
    K.state_host = nullptr;
    return e;
  }
  K.ready = true;
  return cudaSuccess;
}

// *out = a . w (deterministic two-stage reduction)
static cudaError_t dot(stk_problem* P, const double* a, const double* w, int64_t n, double* out) {
  dot_kernel<<<kRedBlocks, kRedThreads, 0, P->stream>>>(a, w, n, P->kry.partial);
  finish_dot_kernel<<<1, 32, 0, P->stream>>>(P->kry.partial, kRedBlocks, 1, out, 0);
  return cudaGetLastError();
}

// One V-cycle on the finest-level buffers of the workspace (fixed pointers):
// the first call runs it directly (setting kernel attributes and building the
// coarse pseudo-inverse), the second captures it into a CUDA graph, later
// calls replay the graph.  Graphs need a non-default stream and opt.use_graphs.
static cudaError_t fixed_vcycle(stk_problem* P, int dtype) {
  const int L = (int)P->levels.size() - 1;
  MgWork& W = P->mg[dtype];
  const bool graphs = P->opt.use_graphs && P->stream != nullptr;
  if (!graphs || W.vcycle_runs == 0) {
    ++W.vcycle_runs;
    return run_vcycle(P, dtype, W.b[L], W.x[L]);
  }
  if (!W.graph) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e1 = vcycle_rec(P, L, dtype, W.b[L], W.x[L]);
    e = cudaStreamEndCapture(P->stream, &g);
    if (e1 != cudaSuccess) e = e1;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&W.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      W.graph = nullptr;
      return e;
    }
  }
  return cudaGraphLaunch(W.graph, P->stream);
}

cudaError_t project_pressure_mean(stk_problem* P, double* x) {
  if (P->dim == 2) return launch_pressure_mean_planar(P, x, P->kry.partial, kRedBlocks);
  const Level& L = P->levels.back();
  double* p = x + 3 * L.nvel;
  pressure_mean_partial<<<kRedBlocks, kRedThreads, 0, P->stream>>>(p, L.m, P->k + 1, P->pmean_w, P->kry.partial);
  pressure_shift<<<grid_for(L.npress), 256, 0, P->stream>>>(p, L.npress, P->kry.partial, kRedBlocks);
  return cudaGetLastError();
}

// --- the launch sequence of the solve, shared by both drivers.  `use` 1:
// the kernels set the conditional handles (graph); 0: the host drives.
static int mixed(const stk_problem* P) { return P->opt.precision == STK_PREC_MIXED; }

static cudaError_t issue_start(stk_problem* P, const double* b, double* x, double rtol, cudaGraphConditionalHandle hout,
                               int use) {
  KrylovWork& K = P->kry;
  const int64_t N = P->levels.back().ntotal;
  GmresState* st = static_cast<GmresState*>(K.state);
  cudaError_t e = dot(P, b, b, N, K.h);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, sizeof(double) * N, P->stream);
  if (e != cudaSuccess) return e;
  gm_start_kernel<<<1, 1, 0, P->stream>>>(st, K.h, rtol, P->opt.gmres_restart, P->opt.max_iter, hout, use);
  gm_scale_kernel<<<grid_for(N), 256, 0, P->stream>>>(b, K.V, st, N);
  return cudaGetLastError();
}

// one Arnoldi step: z = M^{-1} V_j (the V-cycle inline, or its own graph when
// `vcycle_graph`), w = A z, two Gram-Schmidt passes, the norm, the device
// step and V_{j+1}
static cudaError_t issue_iter(stk_problem* P, cudaGraphConditionalHandle hin, int use, bool vcycle_graph) {
  KrylovWork& K = P->kry;
  const int L = (int)P->levels.size() - 1;
  const int64_t N = P->levels[L].ntotal;
  GmresState* st = static_cast<GmresState*>(K.state);
  const int dt = mixed(P) ? STK_F32 : STK_F64;
  MgWork& W = P->mg[dt];
  cudaError_t e = cudaSuccess;
  if (dt == STK_F32)
    gm_copy_in_kernel<float><<<grid_for(N), 256, 0, P->stream>>>(K.V, st, N, (float*)W.b[L]);
  else
    gm_copy_in_kernel<double><<<grid_for(N), 256, 0, P->stream>>>(K.V, st, N, (double*)W.b[L]);
  e = vcycle_graph ? fixed_vcycle(P, dt) : vcycle_rec(P, L, dt, W.b[L], W.x[L]);
  if (e != cudaSuccess) return e;
  const double* z = nullptr;
  if (dt == STK_F32) {
    gm_copy_out_kernel<float><<<grid_for(N), 256, 0, P->stream>>>((const float*)W.x[L], K.Z, st, N, K.zbuf);
    z = K.zbuf;
  } else {
    gm_copy_out_kernel<double><<<grid_for(N), 256, 0, P->stream>>>((const double*)W.x[L], K.Z, st, N, nullptr);
    z = (const double*)W.x[L];
  }
  e = launch_apply(P, L, STK_F64, z, nullptr, K.w, 1.0);
  if (e != cudaSuccess) return e;
  for (int pass = 0; pass < 2; ++pass) {
    double* hp = K.h + pass * kMaxBasis;
    gm_multidot_kernel<<<kRedBlocks, kRedThreads, 0, P->stream>>>(K.V, st, K.w, N, K.partial);
    gm_finish_dot_kernel<<<1, kMaxBasis, 0, P->stream>>>(K.partial, kRedBlocks, st, 0, hp);
    gm_axpy_kernel<<<grid_for(N), 256, 0, P->stream>>>(K.w, K.V, st, hp, N);
  }
  e = dot(P, K.w, K.w, N, K.h + 2 * kMaxBasis);
  if (e != cudaSuccess) return e;
  gm_arnoldi_kernel<<<1, 1, 0, P->stream>>>(st, K.h, hin, use);
  gm_normalize_kernel<<<grid_for(N), 256, 0, P->stream>>>(K.V, K.w, st, N);
  return cudaGetLastError();
}

// end of a cycle: x += Z y, the true residual into V_m and its norm, the
// restart decision and V_0 of the next cycle
static cudaError_t issue_cycle_end(stk_problem* P, const double* b, double* x, cudaGraphConditionalHandle hout,
                                   int use) {
  KrylovWork& K = P->kry;
  const int L = (int)P->levels.size() - 1;
  const int64_t N = P->levels[L].ntotal;
  GmresState* st = static_cast<GmresState*>(K.state);
  double* rtmp = K.V + (size_t)P->opt.gmres_restart * N;
  gm_solve_y_kernel<<<1, 1, 0, P->stream>>>(st);
  gm_update_x_kernel<<<grid_for(N), 256, 0, P->stream>>>(x, K.Z, st, N);
  cudaError_t e = launch_apply(P, L, STK_F64, x, b, rtmp, -1.0);
  if (e == cudaSuccess) e = dot(P, rtmp, rtmp, N, K.h);
  if (e != cudaSuccess) return e;
  gm_restart_kernel<<<1, 1, 0, P->stream>>>(st, K.h, hout, use);
  gm_scale_kernel<<<grid_for(N), 256, 0, P->stream>>>(rtmp, K.V, st, N);
  return cudaGetLastError();
}

// the step of the last solve launch that failed (for the error message)
thread_local const char* g_solve_step = "";

static cudaError_t read_state(stk_problem* P, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(P->kry.state_host, P->kry.state, bytes, cudaMemcpyDeviceToHost, P->stream);
  return e == cudaSuccess ? cudaStreamSynchronize(P->stream) : e;
}

// Everything a solve needs, set up before any capture: the Krylov basis, the
// multigrid workspace, the coarse solver, the Direct inverses and the kernel
// attributes (one V-cycle and one FP64 apply run directly the first time).
static cudaError_t prepare_solve(stk_problem* P) {
  cudaError_t e = ensure_krylov(P);
  const int dt = mixed(P) ? STK_F32 : STK_F64;
  if (e == cudaSuccess) e = ensure_mg_workspace(P, dt);
  if (e == cudaSuccess) e = ensure_coarse(P);
  if (e != cudaSuccess) return e;
  MgWork& W = P->mg[dt];
  if (W.vcycle_runs == 0) {
    const int L = (int)P->levels.size() - 1;
    const size_t es = dt == STK_F64 ? 8 : 4;
    e = cudaMemsetAsync(W.b[L], 0, (size_t)P->levels[L].ntotal * es, P->stream);
    if (e == cudaSuccess) e = fixed_vcycle(P, dt);
    // both forms of the FP64 apply (kernel attributes are set outside any capture)
    if (e == cudaSuccess) e = launch_apply(P, L, STK_F64, P->kry.w, nullptr, P->kry.V, 1.0);
    if (e == cudaSuccess) e = launch_apply(P, L, STK_F64, P->kry.w, P->kry.V, P->kry.Z, -1.0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  }
  return e;
}

// The whole solve as one graph: start, WHILE (another cycle) { cycle begin,
// WHILE (another step) { Arnoldi step }, cycle end }, pressure mean, state
// to the host.  The loop bodies are captured on two side streams into the
// conditional nodes' graphs; the loop conditions are set by the kernels before
// each test (gm_start / gm_restart for the outer loop, gm_cycle_begin /
// gm_arnoldi for the inner one).
static cudaError_t add_while(cudaStream_t s, cudaGraphConditionalHandle* h, cudaGraph_t* body, bool create_handle) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t r = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (r == cudaSuccess && create_handle) r = cudaGraphConditionalHandleCreate(h, g, 0, 0);
  if (r != cudaSuccess) return r;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = *h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  r = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
  if (r != cudaSuccess) return r;
  *body = cp.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

static cudaError_t build_solve_graph(stk_problem* P, const double* b, double* x, double rtol) {
  KrylovWork& K = P->kry;
  for (int i = 0; i < 2; ++i)
    if (!K.side[i]) {
      cudaError_t e = cudaStreamCreateWithFlags(&K.side[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
  const cudaStream_t main = P->stream;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaError_t e = cudaStreamBeginCapture(main, mode);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = cudaSuccess;
  cudaGraphConditionalHandle hout = 0, hin = 0;
  cudaGraph_t top = nullptr, outer = nullptr, inner = nullptr;
  {
    cudaStreamCaptureStatus cs;
    e1 = cudaStreamGetCaptureInfo(main, &cs, nullptr, &top, nullptr, nullptr, nullptr);
    if (e1 == cudaSuccess) e1 = cudaGraphConditionalHandleCreate(&hout, top, 0, 0);
  }
  if (e1 == cudaSuccess) e1 = issue_start(P, b, x, rtol, hout, 1);
  if (e1 == cudaSuccess) e1 = add_while(main, &hout, &outer, false);
  if (e1 != cudaSuccess) g_solve_step = "graph build: start and outer loop";
  if (e1 == cudaSuccess) {
    // outer body on side stream 0
    e1 = cudaStreamBeginCaptureToGraph(K.side[0], outer, nullptr, nullptr, 0, mode);
    if (e1 == cudaSuccess) {
      P->stream = K.side[0];
      cudaError_t eb = cudaGraphConditionalHandleCreate(&hin, outer, 0, 0);
      if (eb == cudaSuccess) {
        gm_cycle_begin_kernel<<<1, 1, 0, P->stream>>>(static_cast<GmresState*>(K.state), hin, 1);
        eb = cudaGetLastError();
      }
      if (eb == cudaSuccess) eb = add_while(K.side[0], &hin, &inner, false);
      if (eb == cudaSuccess) {
        // inner body on side stream 1: one Arnoldi step with the V-cycle inline
        eb = cudaStreamBeginCaptureToGraph(K.side[1], inner, nullptr, nullptr, 0, mode);
        if (eb == cudaSuccess) {
          P->stream = K.side[1];
          cudaError_t ei = issue_iter(P, hin, 1, false);
          cudaGraph_t got = nullptr;
          eb = cudaStreamEndCapture(K.side[1], &got);
          if (ei != cudaSuccess) eb = ei;
          if (eb != cudaSuccess) g_solve_step = "graph build: Arnoldi step body";
          P->stream = K.side[0];
        }
      }
      if (eb == cudaSuccess) eb = issue_cycle_end(P, b, x, hout, 1);
      cudaGraph_t got = nullptr;
      cudaError_t ee = cudaStreamEndCapture(K.side[0], &got);
      e1 = eb != cudaSuccess ? eb : ee;
      P->stream = main;
    }
  }
  if (e1 == cudaSuccess) e1 = project_pressure_mean(P, x);
  if (e1 == cudaSuccess)
    e1 = cudaMemcpyAsync(K.state_host, K.state, sizeof(GmresState), cudaMemcpyDeviceToHost, main);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(main, &graph);
  P->stream = main;
  if (e1 != cudaSuccess) e = e1;
  if (e == cudaSuccess) {
    if (K.solve_graph) cudaGraphExecDestroy(K.solve_graph);
    K.solve_graph = nullptr;
    e = cudaGraphInstantiate(&K.solve_graph, graph, 0);
    if (e != cudaSuccess) {
      K.solve_graph = nullptr;
      g_solve_step = "graph instantiate";
      cudaGetLastError();  // a refused instantiation is not a sticky error: do not leave it for later calls
    }
  }
  if (graph) cudaGraphDestroy(graph);
  if (e == cudaSuccess) {
    K.key_b = b;
    K.key_x = x;
    K.key_rtol = rtol;
  }
  return e;
}

// The whole solve is one graph when the problem has a stream and graphs are
// on, except when its FP32 Direct smoother runs the interior patches'
// products as cuBLAS GEMMs: the library's kernels cannot sit in a
// conditional node's body (instantiation is refused), so those solves are
// driven by the host, with the V-cycle replayed as its own graph.
static bool use_solve_graph(const stk_problem* P) {
  if (!P->opt.use_graphs || P->stream == nullptr) return false;
  if (P->opt.precision == STK_PREC_MIXED && P->opt.local_cg_mode == STK_LOCAL_DIRECT && P->opt.direct_gemm)
    for (const Level& L : P->levels)
      if (L.gemm_cap > 0) return false;
  return true;
}

// Start a solve: the graph is (re)built for new b, x or rtol and launched;
// without graphs the host drives the same launches, reading the state's flags
// after each step.  Returns after the GPU work is enqueued (graph) or done.
static cudaError_t solve_launch(stk_problem* P, const double* b, double* x, double rtol) {
  g_solve_step = "setup";
  cudaError_t e = prepare_solve(P);
  if (e != cudaSuccess) return e;
  KrylovWork& K = P->kry;
  if (use_solve_graph(P)) {
    g_solve_step = "graph build";
    if (!K.solve_graph || K.key_b != b || K.key_x != x || K.key_rtol != rtol) e = build_solve_graph(P, b, x, rtol);
    if (e == cudaSuccess) {
      g_solve_step = "graph launch";
      e = cudaGraphLaunch(K.solve_graph, P->stream);
    }
    return e;
  }
  g_solve_step = "host-driven steps";
  GmresState* st = static_cast<GmresState*>(K.state);
  const GmresState* sh = static_cast<const GmresState*>(K.state_host);
  e = issue_start(P, b, x, rtol, 0, 0);
  if (e == cudaSuccess) e = read_state(P, kStateFlags);
  while (e == cudaSuccess && sh->more) {
    gm_cycle_begin_kernel<<<1, 1, 0, P->stream>>>(st, 0, 0);
    do {
      e = issue_iter(P, 0, 0, true);
      if (e == cudaSuccess) e = read_state(P, kStateFlags);
    } while (e == cudaSuccess && !sh->stop);
    if (e == cudaSuccess) e = issue_cycle_end(P, b, x, 0, 0);
    if (e == cudaSuccess) e = read_state(P, kStateFlags);
  }
  if (e == cudaSuccess) e = project_pressure_mean(P, x);
  if (e == cudaSuccess) e = read_state(P, sizeof(GmresState));
  return e;
}

// After the stream has finished: the info from the state copied to the host.
static int solve_finish(stk_problem* P, double t0_seconds, stk_solve_info* info, std::string& err) {
  const GmresState* sh = static_cast<const GmresState*>(P->kry.state_host);
  stk_solve_info local{};
  stk_solve_info& I = info ? *info : local;
  std::memset(&I, 0, sizeof(stk_solve_info));
  I.iterations = sh->its;
  I.converged = sh->converged ? 1 : 0;
  I.relres = sh->bnorm > 0 ? sh->beta / sh->bnorm : 0.0;
  const int nres = std::min(sh->its, 255);
  for (int i = 0; i <= nres; ++i) I.residuals[i] = sh->res[i];
  I.residuals[0] = 1.0;
  const double last = sh->its > 0 && sh->its < 256 ? sh->res[sh->its] : I.relres;
  I.nu = (sh->its > 0 && last > 0) ? -8.0 / std::log10(std::pow(last, 1.0 / sh->its)) : 0.0;
  I.seconds = t0_seconds;
  if (!sh->converged) {
    err = "GMRES reached max_iter before the tolerance";
    return STK_ENOCONV;
  }
  return STK_OK;
}

static int cuda_status(cudaError_t e, const char* what, std::string& err) {
  err = std::string(what) + " (" + g_solve_step + "): " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA;
}

int run_solve(stk_problem* P, const double* b, double* x, double rtol, stk_solve_info* info, std::string& err) {
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = solve_launch(P, b, x, rtol);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_status(e, "solve", err);
  return solve_finish(P, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(), info, err);
}

// Many problems: every solve is launched (as one graph on the problem's own
// stream where it has one: the solves then run concurrently, with no host
// work between their steps), then all streams are waited for.
int run_solve_batch(stk_problem* const* Ps, int count, const double* const* b, double* const* x, double rtol,
                    stk_solve_info* infos, std::string& err) {
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<cudaError_t> status(count, cudaSuccess);
  for (int i = 0; i < count; ++i) status[i] = solve_launch(Ps[i], b[i], x[i], rtol);
  for (int i = 0; i < count; ++i)
    if (status[i] == cudaSuccess) status[i] = cudaStreamSynchronize(Ps[i]->stream);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = STK_OK;
  for (int i = 0; i < count; ++i) {
    std::string e1;
    const int rc = status[i] == cudaSuccess ? solve_finish(Ps[i], secs, infos ? &infos[i] : nullptr, e1)
                                            : cuda_status(status[i], "solve", e1);
    if (rc != STK_OK && (worst == STK_OK || rc != STK_ENOCONV)) {
      worst = rc;
      err = "problem " + std::to_string(i) + ": " + e1;
    }
  }
  return worst;
}

}  // namespace stk
