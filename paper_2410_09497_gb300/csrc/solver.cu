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

// partial[b * nv + i] = sum over block b's share of V_i . w   (V_i = V + i * n)
__global__ void __launch_bounds__(kRedThreads) multidot_kernel(const double* __restrict__ V, int nv,
                                                                const double* __restrict__ w, int64_t n,
                                                                double* __restrict__ partial) {
  __shared__ double red[kRedThreads / 32][kMaxBasis];
  double acc[kMaxBasis];
  for (int i = 0; i < nv; ++i) acc[i] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double we = w[e];
    for (int i = 0; i < nv; ++i) acc[i] += V[(int64_t)i * n + e] * we;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) s += red[q][i];
    partial[(int64_t)blockIdx.x * nv + i] = s;
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

// w -= sum_i h[i] V_i
__global__ void multi_axpy_kernel(double* __restrict__ w, const double* __restrict__ V, int nv,
                                  const double* __restrict__ h, int64_t n) {
  __shared__ double hs[kMaxBasis];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = w[e];
    for (int i = 0; i < nv; ++i) s -= hs[i] * V[(int64_t)i * n + e];
    w[e] = s;
  }
}

// dst = src / *scale   (scale on the device)
__global__ void scale_kernel(const double* __restrict__ src, double* __restrict__ dst, const double* __restrict__ s,
                             int64_t n) {
  const double inv = 1.0 / *s;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e] * inv;
}

struct Coeffs {
  double y[kMaxBasis];
};

// x += sum_i y_i Z_i
__global__ void update_x_kernel(double* __restrict__ x, const double* __restrict__ Z, int nz, Coeffs c, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = x[e];
    for (int i = 0; i < nz; ++i) s += c.y[i] * Z[(int64_t)i * n + e];
    x[e] = s;
  }
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
cudaError_t ensure_krylov(stk_problem* P) {
  KrylovWork& K = P->kry;
  const int m = P->opt.gmres_restart;
  if (K.ready) return cudaSuccess;
  const int64_t n = P->levels.back().ntotal;
  cudaError_t e = dev_alloc(&K.V, sizeof(double) * (size_t)(m + 1) * n);
  if (e == cudaSuccess) e = dev_alloc(&K.Z, sizeof(double) * (size_t)m * n);
  if (e == cudaSuccess) e = dev_alloc(&K.partial, sizeof(double) * (size_t)kRedBlocks * kMaxBasis);
  if (e == cudaSuccess) e = dev_alloc(&K.h, sizeof(double) * 2 * kMaxBasis);
  if (e == cudaSuccess) e = host_alloc_pinned(&K.h_host, sizeof(double) * 2 * kMaxBasis);
  if (e != cudaSuccess) {  // leave nothing half allocated
    for (double** d : {&K.V, &K.Z, &K.partial, &K.h})
      if (*d) {
        cudaFree(*d);
        *d = nullptr;
      }
    if (K.h_host) cudaFreeHost(K.h_host);
    K.h_host = nullptr;
    return e;
  }
  K.ready = true;
  return cudaSuccess;
}

static cudaError_t dots(stk_problem* P, const double* V, int nv, const double* w, int64_t n, double* out,
                        int accumulate) {
  multidot_kernel<<<kRedBlocks, kRedThreads, 0, P->stream>>>(V, nv, w, n, P->kry.partial);
  finish_dot_kernel<<<1, kMaxBasis, 0, P->stream>>>(P->kry.partial, kRedBlocks, nv, out, accumulate);
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

static cudaError_t precondition(stk_problem* P, const double* v, double* z) {
  const int L = (int)P->levels.size() - 1;
  const int64_t n = P->levels[L].ntotal;
  if (P->opt.precision == STK_PREC_MIXED) {
    MgWork& W = P->mg[STK_F32];
    convert_kernel<double, float><<<grid_for(n), 256, 0, P->stream>>>(v, (float*)W.b[L], n);
    cudaError_t e = fixed_vcycle(P, STK_F32);
    if (e != cudaSuccess) return e;
    convert_kernel<float, double><<<grid_for(n), 256, 0, P->stream>>>((const float*)W.x[L], z, n);
    return cudaGetLastError();
  }
  MgWork& W = P->mg[STK_F64];
  cudaError_t e = cudaMemcpyAsync(W.b[L], v, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream);
  if (e == cudaSuccess) e = fixed_vcycle(P, STK_F64);
  if (e == cudaSuccess) e = cudaMemcpyAsync(z, W.x[L], sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream);
  return e;
}

cudaError_t project_pressure_mean(stk_problem* P, double* x) {
  if (P->dim == 2) return launch_pressure_mean_planar(P, x, P->kry.partial, kRedBlocks);
  const Level& L = P->levels.back();
  double* p = x + 3 * L.nvel;
  pressure_mean_partial<<<kRedBlocks, kRedThreads, 0, P->stream>>>(p, L.m, P->k + 1, P->pmean_w, P->kry.partial);
  pressure_shift<<<grid_for(L.npress), 256, 0, P->stream>>>(p, L.npress, P->kry.partial, kRedBlocks);
  return cudaGetLastError();
}

// dst = src * s (host scalar)
__global__ void scale_by_kernel(const double* __restrict__ src, double* __restrict__ dst, double s, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e] * s;
}

// Flexible GMRES(restart) as a resumable state machine: issue() enqueues the
// GPU work of the current phase on the problem's stream and ends with a copy
// of the scalars the host needs; complete() runs after the stream is idle and
// decides the next phase.  stk_solve drives one machine; stk_solve_batch
// interleaves many, one stream each, so their kernels overlap on the GPU.
struct SolveMachine {
  enum Phase { START, ITER, CYCLE_END, FINISH, DONE };
  stk_problem* P = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  double rtol = 0;
  stk_solve_info* info = nullptr;
  stk_solve_info local{};
  Phase phase = START;
  int status = STK_OK;
  std::string err;
  double bnorm = 0, beta = 0, hn_prev = 1.0;
  int its = 0, j = 0, jdone = 0;
  bool converged = false, need_normalize = false;
  std::vector<double> H, cs, sn, g;
  std::chrono::steady_clock::time_point t0;

  stk_solve_info& I() { return info ? *info : local; }
  int m() const { return P->opt.gmres_restart; }
  int64_t n() const { return P->levels.back().ntotal; }
  cudaStream_t s() const { return P->stream; }

  int prepare() {
    t0 = std::chrono::steady_clock::now();
    cudaError_t e = ensure_krylov(P);
    if (e == cudaSuccess) e = ensure_mg_workspace(P, P->opt.precision == STK_PREC_MIXED ? STK_F32 : STK_F64);
    if (e == cudaSuccess) e = ensure_coarse(P);
    if (e != cudaSuccess) return fail_cuda(e, "solve setup");
    std::memset(&I(), 0, sizeof(stk_solve_info));
    I().residuals[0] = 1.0;
    H.assign((m() + 1) * m(), 0.0);
    cs.assign(m(), 0.0);
    sn.assign(m(), 0.0);
    g.assign(m() + 1, 0.0);
    return STK_OK;
  }

  int fail_cuda(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    status = e == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA;
    phase = DONE;
    return status;
  }

  // enqueue the work of the current phase
  int issue() {
    KrylovWork& K = P->kry;
    const int64_t N = n();
    cudaError_t e = cudaSuccess;
    switch (phase) {
      case START:
        e = dots(P, b, 1, b, N, K.h, 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, sizeof(double) * N, s());
        break;
      case ITER: {
        double* Vj = K.V + (size_t)j * N;
        double* Zj = K.Z + (size_t)j * N;
        double* w = K.V + (size_t)(j + 1) * N;
        if (j == 0) {
          // V_0 = r / beta (r = b when x0 = 0, else the last true residual in V_m)
          const double* r = (its == 0) ? b : K.V + (size_t)m() * N;
          scale_by_kernel<<<grid_for(N), 256, 0, s()>>>(r, K.V, 1.0 / beta, N);
        } else if (need_normalize) {
          scale_by_kernel<<<grid_for(N), 256, 0, s()>>>(Vj, Vj, 1.0 / hn_prev, N);
        }
        e = precondition(P, Vj, Zj);
        if (e == cudaSuccess) e = launch_apply(P, (int)P->levels.size() - 1, STK_F64, Zj, nullptr, w, 1.0);
        if (e != cudaSuccess) break;
        // two passes of classical Gram-Schmidt
        dots(P, K.V, j + 1, w, N, K.h, 0);
        multi_axpy_kernel<<<grid_for(N), 256, 0, s()>>>(w, K.V, j + 1, K.h, N);
        dots(P, K.V, j + 1, w, N, K.h + kMaxBasis, 0);
        multi_axpy_kernel<<<grid_for(N), 256, 0, s()>>>(w, K.V, j + 1, K.h + kMaxBasis, N);
        e = dots(P, w, 1, w, N, K.h + kMaxBasis + j + 1, 0);
        break;
      }
      case CYCLE_END: {
        // y = H^{-1} g (upper triangular), x += Z y, true residual into V_m
        Coeffs c{};
        const int mm = m();
        for (int i = jdone - 1; i >= 0; --i) {
          double sum = g[i];
          for (int l = i + 1; l < jdone; ++l) sum -= H[i * mm + l] * c.y[l];
          c.y[i] = sum / H[i * mm + i];
        }
        update_x_kernel<<<grid_for(N), 256, 0, s()>>>(x, K.Z, jdone, c, N);
        double* rtmp = K.V + (size_t)mm * N;
        e = launch_apply(P, (int)P->levels.size() - 1, STK_F64, x, b, rtmp, -1.0);
        if (e == cudaSuccess) e = dots(P, rtmp, 1, rtmp, N, K.h, 0);
        break;
      }
      case FINISH:
        e = project_pressure_mean(P, x);
        break;
      case DONE:
        return status;
    }
    if (e == cudaSuccess && phase != FINISH)
      e = cudaMemcpyAsync(K.h_host, K.h, sizeof(double) * 2 * kMaxBasis, cudaMemcpyDeviceToHost, s());
    if (e != cudaSuccess) return fail_cuda(e, "solve");
    return STK_OK;
  }

  // host side of the current phase, after the stream has finished
  void complete() {
    KrylovWork& K = P->kry;
    const int mm = m();
    switch (phase) {
      case START:
        bnorm = std::sqrt(K.h_host[0]);
        beta = bnorm;
        converged = bnorm == 0.0;
        j = 0;
        phase = converged ? FINISH : ITER;
        break;
      case ITER: {
        for (int i = 0; i <= j; ++i) H[i * mm + j] = K.h_host[i] + K.h_host[kMaxBasis + i];
        const double hn = std::sqrt(K.h_host[kMaxBasis + j + 1]);
        H[(j + 1) * mm + j] = hn;
        hn_prev = hn;
        need_normalize = true;
        if (j == 0) std::fill(g.begin(), g.end(), 0.0), g[0] = beta;
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * H[i * mm + j] + sn[i] * H[(i + 1) * mm + j];
          H[(i + 1) * mm + j] = -sn[i] * H[i * mm + j] + cs[i] * H[(i + 1) * mm + j];
          H[i * mm + j] = t;
        }
        const double den = std::hypot(H[j * mm + j], H[(j + 1) * mm + j]);
        cs[j] = H[j * mm + j] / den;
        sn[j] = H[(j + 1) * mm + j] / den;
        H[j * mm + j] = den;
        H[(j + 1) * mm + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++its;
        jdone = j + 1;
        if (its < 256) I().residuals[its] = std::fabs(g[j + 1]) / bnorm;
        if (std::fabs(g[j + 1]) <= rtol * bnorm || its >= P->opt.max_iter || j + 1 == mm)
          phase = CYCLE_END;
        else
          ++j;
        break;
      }
      case CYCLE_END:
        beta = std::sqrt(K.h_host[0]);
        converged = beta <= rtol * bnorm;
        if (converged || its >= P->opt.max_iter) {
          phase = FINISH;
        } else {
          j = 0;
          need_normalize = false;
          std::fill(H.begin(), H.end(), 0.0);
          phase = ITER;
        }
        break;
      case FINISH: {
        stk_solve_info& In = I();
        In.iterations = its;
        In.converged = converged ? 1 : 0;
        In.relres = bnorm > 0 ? beta / bnorm : 0.0;
        const double last = its > 0 && its < 256 ? In.residuals[its] : In.relres;
        In.nu = (its > 0 && last > 0) ? -8.0 / std::log10(std::pow(last, 1.0 / its)) : 0.0;
        In.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (!converged) {
          err = "GMRES reached max_iter before the tolerance";
          status = STK_ENOCONV;
        }
        phase = DONE;
        break;
      }
      case DONE:
        break;
    }
  }
};

int run_solve(stk_problem* P, const double* b, double* x, double rtol, stk_solve_info* info, std::string& err) {
  SolveMachine M;
  M.P = P;
  M.b = b;
  M.x = x;
  M.rtol = rtol;
  M.info = info;
  if (M.prepare() != STK_OK) {
    err = M.err;
    return M.status;
  }
  while (M.phase != SolveMachine::DONE) {
    if (M.issue() != STK_OK) break;
    cudaError_t e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) {
      M.fail_cuda(e, "solve");
      break;
    }
    M.complete();
  }
  err = M.err;
  return M.status;
}

int run_solve_batch(stk_problem* const* Ps, int count, const double* const* b, double* const* x, double rtol,
                    stk_solve_info* infos, std::string& err) {
  std::vector<SolveMachine> M(count);
  for (int i = 0; i < count; ++i) {
    M[i].P = Ps[i];
    M[i].b = b[i];
    M[i].x = x[i];
    M[i].rtol = rtol;
    M[i].info = infos ? &infos[i] : nullptr;
    if (M[i].prepare() != STK_OK) {
      err = "problem " + std::to_string(i) + ": " + M[i].err;
      return M[i].status;
    }
  }
  // Each solve advances on its own: whenever its stream has drained, its
  // phase is completed on the host and the next one issued at once, so a
  // short phase of a small problem never waits for a long phase of a large
  // one.  The loop polls the streams (cudaStreamQuery) until all are done.
  int active = 0;
  for (auto& m : M) {
    m.issue();
    if (m.phase != SolveMachine::DONE) ++active;
  }
  while (active > 0) {
    bool progressed = false;
    for (int i = 0; i < count; ++i) {
      SolveMachine& m = M[i];
      if (m.phase == SolveMachine::DONE) continue;
      const cudaError_t q = cudaStreamQuery(m.s());
      if (q == cudaErrorNotReady) continue;
      progressed = true;
      if (q != cudaSuccess) {
        m.fail_cuda(q, "solve");
      } else {
        m.complete();
        if (m.phase != SolveMachine::DONE) m.issue();
      }
      if (m.phase == SolveMachine::DONE) --active;
    }
    if (!progressed) std::this_thread::yield();
  }
  int worst = STK_OK;
  for (int i = 0; i < count; ++i)
    if (M[i].status != STK_OK && (worst == STK_OK || M[i].status != STK_ENOCONV)) {
      worst = M[i].status;
      err = "problem " + std::to_string(i) + ": " + M[i].err;
    }
  return worst;
}

}  // namespace stk
