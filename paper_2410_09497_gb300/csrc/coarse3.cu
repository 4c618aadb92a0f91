// Exact coarse solve on the 3^3 mesh that ends an n = 3 * 2^L hierarchy
// (Sec. 3: the V-cycle's coarsest correction is the exact solve A_0^{-1}).
//
// The coarse system [[A, B^T], [B, 0]] [u; p] = [f; g] is solved by block
// elimination with dense FP64 factors built once:
//   A = diag(A_0, A_1, A_2) is block diagonal over the velocity components
//   (the viscous form acts on each component separately), each A_c symmetric
//   positive definite on the free DoFs; S = B A^{-1} B^T is the pressure
//   Schur complement, whose null space is the constant coefficient vector 1
//   (B^T 1 = 0).  With alpha > 0,
//     t = A^{-1} f,   p = (S + alpha 1 1^T)^{-1} (B t - g),   u = A^{-1} (f - B^T p).
// The right-hand side's pressure rows are first made to sum to zero (the
// bordered system maps that sum to its multiplier); then 1^T p = 0, the
// normalization of the 2^3 pseudo-inverse.  The velocity is computed as
// u = t + A^{-1} (f - A t - B^T p), one refinement step that costs nothing
// extra since the residual kernel forms A t and B^T p together.
//
// Build.  Columns of A_c are the operator kernels applied to unit vectors
// (one unit per component at a time), so the factors use exactly the operator
// of the V-cycle.  Constrained (boundary normal) DoFs have zero rows and
// columns; they get a unit diagonal for the elimination and a zero one
// afterwards, so the solve returns 0 there.  Columns of S are
// B (A^{-1} (B^T e_q)) with the sparse B^T e_q combined from rows of the
// inverse.  Each A_c and S + alpha 1 1^T (alpha = trace(S) / n_p^2, which puts
// the constant mode at S's mean eigenvalue) is inverted in place by
// Gauss-Jordan elimination without pivoting, which is stable for symmetric
// positive definite matrices.  A probed column j is stored as row j, so the
// stored inverse is the transpose of the inverse; the matrices are symmetric
// up to rounding and the solve uses the stored rows directly.
//
// The factors depend only on (device, k, nu, penalty factor): problems share
// them through a process-wide cache.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace stk {

namespace {

constexpr int kGjRows = 8;  // rows of one Gauss-Jordan CTA

// Row j-1 of the three matrices M_c <- y_c (the column probed last); the unit
// entries of x move from j-1 to j (j == n only stores).
__global__ void probe_velocity_step(double* __restrict__ x, double* __restrict__ M, const double* __restrict__ y,
                                    int64_t n, int64_t ld, int64_t j) {
  const int c = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > 0 && i < n) M[((int64_t)c * n + (j - 1)) * ld + i] = y[c * n + i];
  if (i == 0) {
    if (j > 0) x[c * n + j - 1] = 0.0;
    if (j < n) x[c * n + j] = 1.0;
  }
}

// Row q-1 of S <- y_p; the unit pressure entry of x moves from q-1 to q.
__global__ void probe_pressure_step(double* __restrict__ xp, double* __restrict__ S, const double* __restrict__ yp,
                                    int64_t n, int64_t ld, int64_t q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q > 0 && i < n) S[(q - 1) * ld + i] = yp[i];
  if (i == 0) {
    if (q > 0) xp[q - 1] = 0.0;
    if (q < n) xp[q] = 1.0;
  }
}

// A zero diagonal marks a constrained DoF (the operator ignores its input and
// writes 0 to its row); it gets a unit diagonal for the elimination.
__global__ void mark_constrained(double* __restrict__ M, int64_t n, int64_t ld, int nmat,
                                 unsigned char* __restrict__ flag) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n * nmat) return;
  const int64_t mat = r / n, i = r % n;
  double& d = M[(mat * n + i) * ld + i];
  flag[r] = d == 0.0;
  if (d == 0.0) d = 1.0;
}

__global__ void clear_constrained(double* __restrict__ M, int64_t n, int64_t ld, int nmat,
                                  const unsigned char* __restrict__ flag) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n * nmat) return;
  const int64_t mat = r / n, i = r % n;
  if (flag[r]) M[(mat * n + i) * ld + i] = 0.0;
}

// Row and column buffers of pivot step s (double buffered):
//   row(s, mat) = buf + ((s & 1) * nmat + mat) * 2 * ld,  col = row + ld.
__device__ __forceinline__ double* gj_row(double* buf, int s, int nmat, int mat, int64_t ld) {
  return buf + ((int64_t)((s & 1) * nmat + mat) * 2) * ld;
}

__global__ void gj_init(const double* __restrict__ M, int64_t n, int64_t ld, int nmat, double* __restrict__ buf) {
  const int mat = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* A = M + (int64_t)mat * n * ld;
  double* row = gj_row(buf, 0, nmat, mat, ld);
  row[i] = A[i];           // row 0
  row[ld + i] = A[i * ld];  // column 0
}

// One Gauss-Jordan pivot step on column kp of nmat matrices (in place):
//   M[k][k] <- 1/p,  M[k][j] <- M[k][j]/p,  M[i][k] <- -M[i][k]/p,
//   M[i][j] <- M[i][j] - M[i][k] M[k][j] / p   (i, j != k).
// Row and column kp are read from the step's buffers, so every entry is read
// and written by one thread only; the new row and column kp+1 go to the next
// step's buffers.
__global__ void __launch_bounds__(256) gj_step(double* __restrict__ M, int64_t n, int64_t ld, int nmat,
                                               double* __restrict__ buf, int kp) {
  const int mat = blockIdx.y;
  double* A = M + (int64_t)mat * n * ld;
  const double* rk = gj_row(buf, kp, nmat, mat, ld);
  const double* ck = rk + ld;
  double* rn = gj_row(buf, kp + 1, nmat, mat, ld);
  double* cn = rn + ld;
  const double inv_p = 1.0 / rk[kp];
  const int64_t i0 = (int64_t)blockIdx.x * kGjRows;
  for (int r = 0; r < kGjRows; ++r) {
    const int64_t i = i0 + r;
    if (i >= n) break;
    const double cik = ck[i] * inv_p;
    double* Ai = A + i * ld;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      double v;
      if (i == kp)
        v = j == kp ? inv_p : rk[j] * inv_p;
      else if (j == kp)
        v = -cik;
      else
        v = fma(-cik, rk[j], Ai[j]);
      Ai[j] = v;
      if (i == kp + 1) rn[j] = v;
      if (j == kp + 1) cn[i] = v;
    }
  }
}

// t_c = M_c^T y_c over the nonzeros of y_c only (B^T e_q has 3 (k+2) of them):
// t_c[i] = sum_{j: y_c[j] != 0} M_c[j][i] y_c[j], in ascending j.  Each CTA
// compacts the nonzeros of y_c chunk by chunk into shared memory (warp
// ballots, so the order is fixed), then accumulates.
__global__ void __launch_bounds__(256) sparse_combine(const double* __restrict__ M, int64_t n, int64_t ld,
                                                      const double* __restrict__ y, double* __restrict__ t) {
  __shared__ int sj[256];
  __shared__ double sv[256];
  __shared__ int wcount[8];
  const int c = blockIdx.y;
  const double* Mc = M + (int64_t)c * n * ld;
  const double* yc = y + c * n;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += 256) {
    const int64_t j = j0 + threadIdx.x;
    const double v = j < n ? yc[j] : 0.0;
    const unsigned nz = __ballot_sync(0xffffffffu, v != 0.0);
    if (lane == 0) wcount[wid] = __popc(nz);
    __syncthreads();
    int base = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
      base += w < wid ? wcount[w] : 0;
      total += wcount[w];
    }
    if (v != 0.0) {
      const int slot = base + __popc(nz & ((1u << lane) - 1u));
      sj[slot] = (int)j;
      sv[slot] = v;
    }
    __syncthreads();
    if (i < n)
      for (int s = 0; s < total; ++s) acc = fma(Mc[(int64_t)sj[s] * ld + i], sv[s], acc);
    __syncthreads();
  }
  if (i < n) t[c * n + i] = acc;
}

// alpha = trace(S) / n^2 (one CTA, fixed order)
__global__ void __launch_bounds__(256) schur_shift(const double* __restrict__ S, int64_t n, int64_t ld,
                                                   double* __restrict__ alpha) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += S[i * ld + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *alpha = t / ((double)n * (double)n);
  }
}

__global__ void add_shift(double* __restrict__ S, int64_t n, int64_t ld, const double* __restrict__ alpha) {
  const double a = *alpha;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x)
    S[(e / n) * ld + e % n] += a;
}

// y_mat = alpha M_mat x_mat (+ y_mat if accumulate), one warp per row; x and y
// are nmat consecutive segments of length n, M_mat row-major with stride ld
// (ld even, rows 16-byte aligned).
__global__ void __launch_bounds__(256) gemv_blocks(const double* __restrict__ M, int64_t n, int64_t ld, int nmat,
                                                   const double* __restrict__ x, double* __restrict__ y,
                                                   double alpha, int accumulate) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n * nmat) return;
  const int64_t mat = row / n;
  const double* Mr = M + row * ld;
  const double* xs = x + mat * n;
  double a0 = 0.0, a1 = 0.0;
  int64_t j = 2 * lane;
  for (; j + 1 < n; j += 64) {
    const double2 m = *reinterpret_cast<const double2*>(Mr + j);
    a0 = fma(m.x, __ldg(xs + j), a0);
    a1 = fma(m.y, __ldg(xs + j + 1), a1);
  }
  if (j < n) a0 = fma(Mr[j], __ldg(xs + j), a0);
  double s = a0 + a1;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = alpha * s + (accumulate ? y[row] : 0.0);
}

int64_t round_ld(int64_t n) { return (n + 3) & ~int64_t(3); }

cudaError_t gemv(const double* M, int64_t n, int64_t ld, int nmat, const double* x, double* y, double alpha,
                 int accumulate, cudaStream_t s) {
  const int64_t rows = n * nmat;
  gemv_blocks<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(M, n, ld, nmat, x, y, alpha, accumulate);
  return cudaGetLastError();
}

// In-place Gauss-Jordan inverse of nmat matrices (n x n, stride ld).
cudaError_t gauss_jordan(double* M, int64_t n, int64_t ld, int nmat, cudaStream_t s) {
  double* buf = nullptr;
  cudaError_t e = dev_alloc_async(&buf, sizeof(double) * 4 * (size_t)nmat * ld, s);
  if (e != cudaSuccess) return e;
  gj_init<<<dim3((unsigned)((n + 255) / 256), nmat), 256, 0, s>>>(M, n, ld, nmat, buf);
  const dim3 grid((unsigned)((n + kGjRows - 1) / kGjRows), nmat);
  for (int kp = 0; kp < n; ++kp) gj_step<<<grid, 256, 0, s>>>(M, n, ld, nmat, buf, kp);
  e = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(buf, s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace

struct Coarse3Factors {
  int64_t nc = 0, np = 0, ldA = 0, ldS = 0;
  double* Ainv = nullptr;  // 3 blocks of nc rows, stride ldA
  double* Sinv = nullptr;  // np rows, stride ldS
  ~Coarse3Factors() {
    if (Ainv) cudaFree(Ainv);
    if (Sinv) cudaFree(Sinv);
  }
};

namespace {

using Key = std::tuple<int, int, uint64_t, uint64_t>;
std::mutex g_mu;
std::map<Key, std::weak_ptr<Coarse3Factors>> g_cache;

uint64_t bits(double v) {
  uint64_t b;
  std::memcpy(&b, &v, sizeof b);
  return b;
}

cudaError_t fill_factors(stk_problem* P, Coarse3Factors& F, unsigned char* flag);

// Builds the factors on the problem's stream with its coarse FP64 vectors
// (x = coarse3[1], y = coarse3[2]) as probes; synchronizes at the end.
cudaError_t build_factors(stk_problem* P, Coarse3Factors& F) {
  const Level& L = P->levels[0];
  const cudaStream_t s = P->stream;
  const int64_t nc = L.nvel, np = L.npress;
  F.nc = nc;
  F.np = np;
  F.ldA = round_ld(nc);
  F.ldS = round_ld(np);
  cudaError_t e = dev_alloc(&F.Ainv, sizeof(double) * 3 * (size_t)nc * F.ldA);
  if (e == cudaSuccess) e = dev_alloc(&F.Sinv, sizeof(double) * (size_t)np * F.ldS);
  if (e != cudaSuccess) return e;
  unsigned char* flag = nullptr;
  e = dev_alloc_async(&flag, 3 * (size_t)nc, s);
  if (e != cudaSuccess) return e;
  e = fill_factors(P, F, flag);
  const cudaError_t e2 = cudaFreeAsync(flag, s);  // on every path
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// The probes, eliminations and shift of build_factors; flag: 3 n_c bytes of
// device scratch.
cudaError_t fill_factors(stk_problem* P, Coarse3Factors& F, unsigned char* flag) {
  const Level& L = P->levels[0];
  const cudaStream_t s = P->stream;
  const int64_t nc = L.nvel, np = L.npress, N = L.ntotal;
  double *x = P->coarse3[1], *y = P->coarse3[2], *t = P->coarse3[0];
  cudaError_t e = cudaMemsetAsync(F.Ainv, 0, sizeof(double) * 3 * (size_t)nc * F.ldA, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(F.Sinv, 0, sizeof(double) * (size_t)np * F.ldS, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, sizeof(double) * N, s);
  if (e != cudaSuccess) return e;

  // A_c: unit vectors in all three components at once (A is block diagonal)
  const dim3 gv((unsigned)((nc + 255) / 256), 3);
  for (int64_t j = 0; j <= nc && e == cudaSuccess; ++j) {
    probe_velocity_step<<<gv, 256, 0, s>>>(x, F.Ainv, y, nc, F.ldA, j);
    if (j < nc) e = launch_apply(P, 0, STK_F64, x, nullptr, y, 1.0, 1);
  }
  if (e != cudaSuccess) return e;
  mark_constrained<<<(unsigned)((3 * nc + 255) / 256), 256, 0, s>>>(F.Ainv, nc, F.ldA, 3, flag);
  e = gauss_jordan(F.Ainv, nc, F.ldA, 3, s);
  if (e != cudaSuccess) return e;
  clear_constrained<<<(unsigned)((3 * nc + 255) / 256), 256, 0, s>>>(F.Ainv, nc, F.ldA, 3, flag);

  // S = B A^{-1} B^T, column q from the unit pressure vector e_q (velocity part of x is zero again)
  double* xp = x + 3 * nc;
  const unsigned gp = (unsigned)((np + 255) / 256);
  for (int64_t q = 0; q <= np && e == cudaSuccess; ++q) {
    probe_pressure_step<<<gp, 256, 0, s>>>(xp, F.Sinv, y + 3 * nc, np, F.ldS, q);
    if (q == np) break;
    e = launch_apply(P, 0, STK_F64, x, nullptr, y, 1.0, 1);  // y_u = B^T e_q
    if (e != cudaSuccess) break;
    sparse_combine<<<gv, 256, 0, s>>>(F.Ainv, nc, F.ldA, y, t);  // t_u = A^{-1} B^T e_q
    e = launch_apply(P, 0, STK_F64, t, nullptr, y, 1.0, 2);      // y_p = B t_u
  }
  if (e != cudaSuccess) return e;
  double* alpha = reinterpret_cast<double*>(flag);  // 3 nc >= 8 bytes, flags no longer needed
  schur_shift<<<1, 256, 0, s>>>(F.Sinv, np, F.ldS, alpha);
  add_shift<<<(unsigned)std::min<int64_t>((np * np + 255) / 256, 4096), 256, 0, s>>>(F.Sinv, np, F.ldS, alpha);
  return gauss_jordan(F.Sinv, np, F.ldS, 1, s);
}

}  // namespace

cudaError_t invert_shifted(double* M, int64_t n, int64_t ld, cudaStream_t s) {
  double* alpha = nullptr;
  cudaError_t e = dev_alloc_async(&alpha, sizeof(double), s);
  if (e != cudaSuccess) return e;
  schur_shift<<<1, 256, 0, s>>>(M, n, ld, alpha);
  add_shift<<<(unsigned)std::min<int64_t>((n * n + 255) / 256, 4096), 256, 0, s>>>(M, n, ld, alpha);
  e = gauss_jordan(M, n, ld, 1, s);
  const cudaError_t e2 = cudaFreeAsync(alpha, s);
  return e != cudaSuccess ? e : e2;
}

cudaError_t acquire_coarse3(stk_problem* P) {
  if (P->coarse3f) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const Key key{dev, P->k, bits(P->nu), bits(P->opt.penalty_factor)};
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_cache.find(key);
  if (it != g_cache.end())
    if (auto f = it->second.lock()) {
      P->coarse3f = f;
      return cudaSuccess;
    }
  auto f = std::make_shared<Coarse3Factors>();
  e = build_factors(P, *f);
  if (e != cudaSuccess) return e;
  g_cache[key] = f;
  P->coarse3f = f;
  return cudaSuccess;
}

// x = A_0^{-1} b on the 3^3 mesh, FP64 in P->coarse3 (b in [0], x in [1],
// scratch in [2]); b's pressure rows must already sum to zero.
cudaError_t coarse3_solve(stk_problem* P) {
  const Coarse3Factors& F = *P->coarse3f;
  const cudaStream_t s = P->stream;
  const int64_t nv = 3 * F.nc;
  double *b = P->coarse3[0], *x = P->coarse3[1], *r = P->coarse3[2];
  cudaError_t e = gemv(F.Ainv, F.nc, F.ldA, 3, b, x, 1.0, 0, s);         // t = A^{-1} f
  if (e == cudaSuccess) e = launch_apply(P, 0, STK_F64, x, b, r, -1.0, 2);  // r_p = g - B t
  if (e == cudaSuccess) e = gemv(F.Sinv, F.np, F.ldS, 1, r + nv, x + nv, -1.0, 0, s);  // p
  if (e == cudaSuccess) e = launch_apply(P, 0, STK_F64, x, b, r, -1.0, 1);  // r_u = f - A t - B^T p
  if (e == cudaSuccess) e = gemv(F.Ainv, F.nc, F.ldA, 3, r, x, 1.0, 1, s);  // u = t + A^{-1} r_u
  return e;
}

}  // namespace stk
