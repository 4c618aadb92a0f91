// Host orchestration of the multigrid method and the outer Krylov solver,
// plus the BLAS-1 kernels they need.
//
//  smooth  (Algorithm 2): for each colour, r = b - A x, then the patch kernel.
//  vcycle  (Sec. 3): pre-smooth, residual, restriction, recursion, exact
//          coarse solve on the 2^3 mesh, prolongation-add, post-smooth; x0 = 0.
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
static cudaError_t dmalloc(void** p, size_t bytes) { return cudaMalloc(p, bytes); }

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
    cudaError_t e = dmalloc(&W.r[l], bytes);
    if (e == cudaSuccess) e = dmalloc(&W.b[l], bytes);
    if (e == cudaSuccess) e = dmalloc(&W.x[l], bytes);
    if (e != cudaSuccess) return e;
  }
  W.ready = true;
  return cudaSuccess;
}

cudaError_t ensure_coarse(stk_problem* P) {
  if (P->coarse_inv) return cudaSuccess;
  const int NL = patch_local_size(P->k);
  cudaError_t e = cudaMalloc(&P->coarse_inv, sizeof(double) * (size_t)NL * NL);
  if (e != cudaSuccess) return e;
  // every free coarse DoF's pseudo-inverse column: CG on the Schur complement to 1e-14
  e = launch_coarse_columns(P, P->coarse_inv, 2000, 1e-14);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(P->stream);
}

// ---------------------------------------------------------------- smoother
cudaError_t run_smooth(stk_problem* P, int level, int dtype, void* x, const void* b) {
  cudaError_t e = ensure_mg_workspace(P, dtype);
  if (e != cudaSuccess) return e;
  void* r = P->mg[dtype].r[level];
  for (int colour = 0; colour < 8; ++colour) {
    e = launch_apply(P, level, dtype, x, b, r, -1.0);
    if (e != cudaSuccess) return e;
    e = launch_patch_colour(P, level, dtype, colour, r, x);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t vcycle_rec(stk_problem* P, int level, int dtype, const void* b, void* x) {
  cudaError_t e;
  if (level == 0) return launch_coarse_solve(P, dtype, b, x);
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
  return launch_coarse_solve(P, dtype, b, x);
}

// -------------------------------------------------------------------- FGMRES
cudaError_t ensure_krylov(stk_problem* P) {
  KrylovWork& K = P->kry;
  const int m = P->opt.gmres_restart;
  if (K.ready) return cudaSuccess;
  const int64_t n = P->levels.back().ntotal;
  cudaError_t e = cudaMalloc(&K.V, sizeof(double) * (size_t)(m + 1) * n);
  if (e == cudaSuccess) e = cudaMalloc(&K.Z, sizeof(double) * (size_t)m * n);
  if (e == cudaSuccess) e = cudaMalloc(&K.partial, sizeof(double) * (size_t)kRedBlocks * kMaxBasis);
  if (e == cudaSuccess) e = cudaMalloc(&K.h, sizeof(double) * 2 * kMaxBasis);
  if (e == cudaSuccess) e = cudaMallocHost(&K.h_host, sizeof(double) * 2 * kMaxBasis);
  if (e != cudaSuccess) return e;
  K.ready = true;
  return cudaSuccess;
}

static cudaError_t dots(stk_problem* P, const double* V, int nv, const double* w, int64_t n, double* out,
                        int accumulate) {
  multidot_kernel<<<kRedBlocks, kRedThreads, 0, P->stream>>>(V, nv, w, n, P->kry.partial);
  finish_dot_kernel<<<1, kMaxBasis, 0, P->stream>>>(P->kry.partial, kRedBlocks, nv, out, accumulate);
  return cudaGetLastError();
}

static cudaError_t precondition(stk_problem* P, const double* v, double* z) {
  const int L = (int)P->levels.size() - 1;
  const int64_t n = P->levels[L].ntotal;
  if (P->opt.precision == STK_PREC_MIXED) {
    cudaError_t e = ensure_mg_workspace(P, STK_F32);
    if (e != cudaSuccess) return e;
    float* b32 = (float*)P->mixed_b;
    float* x32 = (float*)P->mixed_x;
    convert_kernel<double, float><<<grid_for(n), 256, 0, P->stream>>>(v, b32, n);
    e = run_vcycle(P, STK_F32, b32, x32);
    if (e != cudaSuccess) return e;
    convert_kernel<float, double><<<grid_for(n), 256, 0, P->stream>>>(x32, z, n);
    return cudaGetLastError();
  }
  return run_vcycle(P, STK_F64, v, z);
}

cudaError_t project_pressure_mean(stk_problem* P, double* x) {
  const Level& L = P->levels.back();
  double* p = x + 3 * L.nvel;
  pressure_mean_partial<<<kRedBlocks, kRedThreads, 0, P->stream>>>(p, L.m, P->k + 1, P->pmean_w, P->kry.partial);
  pressure_shift<<<grid_for(L.npress), 256, 0, P->stream>>>(p, L.npress, P->kry.partial, kRedBlocks);
  return cudaGetLastError();
}

int run_solve(stk_problem* P, const double* b, double* x, double rtol, stk_solve_info* info, std::string& err) {
  auto t0 = std::chrono::steady_clock::now();
  const int m = P->opt.gmres_restart;
  const int L = (int)P->levels.size() - 1;
  const int64_t n = P->levels[L].ntotal;
  cudaStream_t s = P->stream;
  cudaError_t e = ensure_krylov(P);
  if (e == cudaSuccess && P->opt.precision == STK_PREC_MIXED && !P->mixed_b) {
    e = cudaMalloc(&P->mixed_b, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->mixed_x, sizeof(float) * n);
  }
  if (e == cudaSuccess) e = ensure_mg_workspace(P, P->opt.precision == STK_PREC_MIXED ? STK_F32 : STK_F64);
  if (e == cudaSuccess) e = ensure_coarse(P);
  if (e != cudaSuccess) {
    err = std::string("solve setup: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA;
  }
  KrylovWork& K = P->kry;
  stk_solve_info local{};
  stk_solve_info& I = info ? *info : local;
  std::memset(&I, 0, sizeof(I));
  I.residuals[0] = 1.0;
  // ||b||
  dots(P, b, 1, b, n, K.h, 0);
  cudaMemcpyAsync(K.h_host, K.h, sizeof(double), cudaMemcpyDeviceToHost, s);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
    err = std::string("solve: ") + cudaGetErrorString(e);
    return STK_ECUDA;
  }
  const double bnorm = std::sqrt(K.h_host[0]);
  cudaMemsetAsync(x, 0, sizeof(double) * n, s);
  int its = 0;
  bool converged = bnorm == 0.0;
  double beta = bnorm;
  // r0 = b (x0 = 0) into V_0 after scaling
  const double* rsrc = b;
  double* rtmp = K.V + (size_t)m * n;  // the last basis slot doubles as residual storage
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1);
  while (!converged && its < P->opt.max_iter) {
    // V_0 = r / beta
    K.h_host[0] = beta;
    cudaMemcpyAsync(K.h, K.h_host, sizeof(double), cudaMemcpyHostToDevice, s);
    scale_kernel<<<grid_for(n), 256, 0, s>>>(rsrc, K.V, K.h, n);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double* Vj = K.V + (size_t)j * n;
      double* Zj = K.Z + (size_t)j * n;
      double* w = K.V + (size_t)(j + 1) * n;
      if ((e = precondition(P, Vj, Zj)) != cudaSuccess) break;
      if ((e = launch_apply(P, L, STK_F64, Zj, nullptr, w, 1.0)) != cudaSuccess) break;
      // two passes of classical Gram-Schmidt
      dots(P, K.V, j + 1, w, n, K.h, 0);
      multi_axpy_kernel<<<grid_for(n), 256, 0, s>>>(w, K.V, j + 1, K.h, n);
      dots(P, K.V, j + 1, w, n, K.h + kMaxBasis, 0);
      multi_axpy_kernel<<<grid_for(n), 256, 0, s>>>(w, K.V, j + 1, K.h + kMaxBasis, n);
      dots(P, w, 1, w, n, K.h + kMaxBasis + j + 1, 0);
      cudaMemcpyAsync(K.h_host, K.h, sizeof(double) * 2 * kMaxBasis, cudaMemcpyDeviceToHost, s);
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
      for (int i = 0; i <= j; ++i) H[i * m + j] = K.h_host[i] + K.h_host[kMaxBasis + i];
      const double hn = std::sqrt(K.h_host[kMaxBasis + j + 1]);
      H[(j + 1) * m + j] = hn;
      K.h_host[0] = hn;
      cudaMemcpyAsync(K.h, K.h_host, sizeof(double), cudaMemcpyHostToDevice, s);
      scale_kernel<<<grid_for(n), 256, 0, s>>>(w, w, K.h, n);
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      cs[j] = H[j * m + j] / den;
      sn[j] = H[(j + 1) * m + j] / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      jdone = j + 1;
      if (its < 256) I.residuals[its] = std::fabs(g[j + 1]) / bnorm;
      if (std::fabs(g[j + 1]) <= rtol * bnorm || its >= P->opt.max_iter) break;
    }
    if (e != cudaSuccess) break;
    // y = H^{-1} g (upper triangular), x += Z y
    Coeffs c{};
    for (int i = jdone - 1; i >= 0; --i) {
      double sum = g[i];
      for (int l = i + 1; l < jdone; ++l) sum -= H[i * m + l] * c.y[l];
      c.y[i] = sum / H[i * m + i];
    }
    update_x_kernel<<<grid_for(n), 256, 0, s>>>(x, K.Z, jdone, c, n);
    // true residual
    if ((e = launch_apply(P, L, STK_F64, x, b, rtmp, -1.0)) != cudaSuccess) break;
    dots(P, rtmp, 1, rtmp, n, K.h, 0);
    cudaMemcpyAsync(K.h_host, K.h, sizeof(double), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    beta = std::sqrt(K.h_host[0]);
    rsrc = rtmp;
    converged = beta <= rtol * bnorm;
  }
  if (e != cudaSuccess) {
    err = std::string("solve: ") + cudaGetErrorString(e);
    return STK_ECUDA;
  }
  if ((e = project_pressure_mean(P, x)) == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = std::string("solve: ") + cudaGetErrorString(e);
    return STK_ECUDA;
  }
  I.iterations = its;
  I.converged = converged ? 1 : 0;
  I.relres = bnorm > 0 ? beta / bnorm : 0.0;
  const double last = its > 0 && its < 256 ? I.residuals[its] : I.relres;
  I.nu = (its > 0 && last > 0) ? -8.0 / std::log10(std::pow(last, 1.0 / its)) : 0.0;
  I.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (!converged) {
    err = "GMRES reached max_iter before the tolerance";
    return STK_ENOCONV;
  }
  return STK_OK;
}

}  // namespace stk
