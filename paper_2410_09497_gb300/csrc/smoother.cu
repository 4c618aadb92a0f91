// Coloured vertex-patch multiplicative Schwarz smoother (Algorithm 2) with the
// Schur-complement local solver built on the fast diagonalization method
// (Sec. 3.2).
//
// Algorithm 2 on one level: for each of the 8 colours, r = b - A x (the
// residual kernel of apply.cu), then one CTA per patch of the colour:
//   gather  F = R_j r (velocity, patch-boundary normal nodes excluded),
//           G = pressure part of R_j r
//   solve   S P = B A^{-1} F - G  by CG on mean-free pressures,
//           S = B A^{-1} B^T, then U = A^{-1} (F - B^T P)
//   scatter x += R_j^T (U, P)
// The patches of one colour share no DoF, so the scatter needs no atomics.
// A^{-1} of each velocity component is applied as
//   (1/nu) (S_x (x) S_y (x) S_z) diag(1 / (lam_x + lam_y + lam_z)) (S_x (x) S_y (x) S_z)^T
// (eq. `inverse2d` in 3D): three forward line transforms, a diagonal scale,
// three backward line transforms, all in shared memory.  B and B^T are the
// local divergence factor D_loc along the component's continuous direction
// scaled by the diagonal Gauss masses of the other two (eq. `b`).
//
// The same kernel, with the right-hand side set to unit vectors, builds the
// dense pseudo-inverse of the coarse problem at setup: on a 2^3 mesh the one
// vertex patch holds every free DoF.
#include <algorithm>

#include "internal.h"

namespace stk {

template <int K>
struct PatchCfg {
  static constexpr int ND = K + 1, NPC = 2 * K + 1, NPD = 2 * K + 2;
  static constexpr int NV1 = NPC * NPD * NPD;  // one velocity component
  static constexpr int NV = 3 * NV1;
  static constexpr int NP = NPD * NPD * NPD;
  static constexpr int NT = (K <= 2) ? 128 : 256;
  static constexpr int NW = NT / 32;
};

template <typename T>
struct PatchArgs {
  const T* r;     // colour residual (mode 0)
  T* x;           // solution, updated in place (mode 0)
  double* cols;   // mode 1: column-major output, N_p x N_p
  const PatchTables<T>* tab;
  int n, m;
  int colour;
  int cnt[3];     // patches of the colour per direction
  int mode;       // 0: smoother colour, 1: coarse pseudo-inverse columns
  int cg_iters;   // FIXED: exact count; TOL: limit
  int cg_tol_mode;
  T cg_tol;
};

template <typename T, int NW>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
#pragma unroll
  for (int i = 0; i < NW; ++i) s += red[i];
  return s;
}

// Extents of velocity component c on the patch: NPC along c, NPD otherwise.
template <int K>
__device__ __forceinline__ int vext(int c, int d) {
  return (c == d) ? PatchCfg<K>::NPC : PatchCfg<K>::NPD;
}

// Line transforms of all three velocity components along direction d.
// forward: out_j = sum_i S[i][j] in_i  (S^T), backward: out_i = sum_j S[i][j] in_j.
template <int K, typename T>
__device__ void transform_dir(const T* __restrict__ in, T* __restrict__ out, int d, bool forward,
                              const PatchTables<T>& tb, const int* type) {
  using C = PatchCfg<K>;
  constexpr int NMAX = C::NPD;
  // lines per component: NV1 / extent along d
  const int lines_c0 = C::NV1 / vext<K>(0, d);
  const int lines_c1 = C::NV1 / vext<K>(1, d);
  const int total = lines_c0 + lines_c1 + C::NV1 / vext<K>(2, d);
  for (int L = threadIdx.x; L < total; L += C::NT) {
    int c, l;
    if (L < lines_c0) {
      c = 0;
      l = L;
    } else if (L < lines_c0 + lines_c1) {
      c = 1;
      l = L - lines_c0;
    } else {
      c = 2;
      l = L - lines_c0 - lines_c1;
    }
    const int e0 = vext<K>(c, 0), e1 = vext<K>(c, 1);
    const int n = vext<K>(c, d);
    int base, stride;
    if (d == 0) {
      base = l * e0;
      stride = 1;
    } else if (d == 1) {
      const int i0 = l % e0, i2 = l / e0;
      base = i0 + e0 * e1 * i2;
      stride = e0;
    } else {
      base = l;
      stride = e0 * e1;
    }
    base += c * C::NV1;
    const T* S = (d == c) ? tb.SC : tb.SD[type[d]];
    T v[NMAX];
#pragma unroll
    for (int i = 0; i < NMAX; ++i) v[i] = (i < n) ? in[base + i * stride] : T(0);
    if (forward) {
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        if (j >= n) break;
        T acc = T(0);
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
          if (i < n) acc += S[i * n + j] * v[i];
        out[base + j * stride] = acc;
      }
    } else {
#pragma unroll
      for (int i = 0; i < NMAX; ++i) {
        if (i >= n) break;
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
          if (j < n) acc += S[i * n + j] * v[j];
        out[base + i * stride] = acc;
      }
    }
  }
  __syncthreads();
}

// Y = A^{-1} X for the three velocity components; A is scratch, X may equal Y.
template <int K, typename T>
__device__ void fdm_inverse(const T* X, T* Abuf, T* Y, const PatchTables<T>& tb, const int* type) {
  using C = PatchCfg<K>;
  transform_dir<K, T>(X, Abuf, 0, true, tb, type);
  transform_dir<K, T>(Abuf, Y, 1, true, tb, type);
  transform_dir<K, T>(Y, Abuf, 2, true, tb, type);
  for (int i = threadIdx.x; i < C::NV; i += C::NT) {
    const int c = i / C::NV1, li = i - c * C::NV1;
    const int e0 = vext<K>(c, 0), e1 = vext<K>(c, 1);
    const int i0 = li % e0, i1 = (li / e0) % e1, i2 = li / (e0 * e1);
    const T l0 = (c == 0) ? tb.LC[i0] : tb.LD[type[0]][i0];
    const T l1 = (c == 1) ? tb.LC[i1] : tb.LD[type[1]][i1];
    const T l2 = (c == 2) ? tb.LC[i2] : tb.LD[type[2]][i2];
    Abuf[i] *= tb.inv_nu / (l0 + l1 + l2);
  }
  __syncthreads();
  transform_dir<K, T>(Abuf, Y, 2, false, tb, type);
  transform_dir<K, T>(Y, Abuf, 1, false, tb, type);
  transform_dir<K, T>(Abuf, Y, 0, false, tb, type);
}

// Gout = B V (pressure nodes)
template <int K, typename T>
__device__ void apply_B(const T* V, T* Gout, const PatchTables<T>& tb) {
  using C = PatchCfg<K>;
  for (int q = threadIdx.x; q < C::NP; q += C::NT) {
    const int q0 = q % C::NPD, q1 = (q / C::NPD) % C::NPD, q2 = q / (C::NPD * C::NPD);
    T acc = T(0);
    {  // component x: D along x, masses along y, z
      const T* v = V + 0 * C::NV1 + C::NPC * (q1 + C::NPD * q2);
      T s = T(0);
#pragma unroll
      for (int a = 0; a < C::NPC; ++a) s += tb.DL[q0 * C::NPC + a] * v[a];
      acc += tb.W[q1] * tb.W[q2] * s;
    }
    {  // component y
      const T* v = V + 1 * C::NV1 + q0 + C::NPD * C::NPC * q2;
      T s = T(0);
#pragma unroll
      for (int a = 0; a < C::NPC; ++a) s += tb.DL[q1 * C::NPC + a] * v[a * C::NPD];
      acc += tb.W[q0] * tb.W[q2] * s;
    }
    {  // component z
      const T* v = V + 2 * C::NV1 + q0 + C::NPD * q1;
      T s = T(0);
#pragma unroll
      for (int a = 0; a < C::NPC; ++a) s += tb.DL[q2 * C::NPC + a] * v[a * C::NPD * C::NPD];
      acc += tb.W[q0] * tb.W[q1] * s;
    }
    Gout[q] = acc;
  }
  __syncthreads();
}

// Vout = B^T P (velocity nodes)
template <int K, typename T>
__device__ void apply_BT(const T* Pin, T* Vout, const PatchTables<T>& tb) {
  using C = PatchCfg<K>;
  for (int i = threadIdx.x; i < C::NV; i += C::NT) {
    const int c = i / C::NV1, li = i - c * C::NV1;
    const int e0 = vext<K>(c, 0), e1 = vext<K>(c, 1);
    const int i0 = li % e0, i1 = (li / e0) % e1, i2 = li / (e0 * e1);
    const int ii[3] = {i0, i1, i2};
    const int a = ii[c];
    // pressure index with q_c running, others fixed
    int pbase, pstride;
    if (c == 0) {
      pbase = C::NPD * (i1 + C::NPD * i2);
      pstride = 1;
    } else if (c == 1) {
      pbase = i0 + C::NPD * C::NPD * i2;
      pstride = C::NPD;
    } else {
      pbase = i0 + C::NPD * i1;
      pstride = C::NPD * C::NPD;
    }
    T s = T(0);
#pragma unroll
    for (int q = 0; q < C::NPD; ++q) s += tb.DL[q * C::NPC + a] * Pin[pbase + q * pstride];
    const int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
    Vout[i] = tb.W[ii[d1]] * tb.W[ii[d2]] * s;
  }
  __syncthreads();
}

// global index of patch-local DoF j (velocity components then pressure)
template <int K>
__device__ __forceinline__ int64_t patch_global(int j, const int* v, int m) {
  using C = PatchCfg<K>;
  constexpr int ND = C::ND;
  const int64_t nvel = (int64_t)(m + 1) * m * m;
  if (j < C::NV) {
    const int c = j / C::NV1, li = j - c * C::NV1;
    const int e0 = vext<K>(c, 0), e1 = vext<K>(c, 1);
    const int ii[3] = {li % e0, (li / e0) % e1, li / (e0 * e1)};
    int64_t g[3];
    for (int d = 0; d < 3; ++d) g[d] = (int64_t)(v[d] - 1) * ND + ii[d] + (d == c ? 1 : 0);
    const int64_t E0 = (c == 0) ? m + 1 : m, E1 = (c == 1) ? m + 1 : m;
    return c * nvel + g[0] + E0 * (g[1] + E1 * g[2]);
  }
  const int q = j - C::NV;
  const int qq[3] = {q % C::NPD, (q / C::NPD) % C::NPD, q / (C::NPD * C::NPD)};
  int64_t g[3];
  for (int d = 0; d < 3; ++d) g[d] = (int64_t)(v[d] - 1) * ND + qq[d];
  return 3 * nvel + g[0] + (int64_t)m * (g[1] + (int64_t)m * g[2]);
}

template <int K, typename T>
__global__ void __launch_bounds__(PatchCfg<K>::NT) patch_kernel(PatchArgs<T> A) {
  using C = PatchCfg<K>;
  __shared__ PatchTables<T> tb;
  __shared__ T red[C::NW];
  extern __shared__ __align__(16) unsigned char patch_smem[];
  T* Fv = reinterpret_cast<T*>(patch_smem);  // velocity rhs F, later F - B^T P
  T* V1 = Fv + C::NV;
  T* V2 = V1 + C::NV;
  T* G = V2 + C::NV;
  T* Pp = G + C::NP;
  T* R = Pp + C::NP;
  T* Dd = R + C::NP;
  T* Sd = Dd + C::NP;

  const int tid = threadIdx.x;
  for (int i = tid; i < (int)(sizeof(PatchTables<T>) / sizeof(T)); i += C::NT)
    reinterpret_cast<T*>(&tb)[i] = reinterpret_cast<const T*>(A.tab)[i];

  int v[3];
  if (A.mode == 0) {
    int p = blockIdx.x;
    for (int d = 0; d < 3; ++d) {
      const int t = p % A.cnt[d];
      p /= A.cnt[d];
      const int bit = (A.colour >> d) & 1;
      v[d] = bit ? 2 * t + 1 : 2 * t + 2;
    }
  } else {
    v[0] = v[1] = v[2] = 1;
  }
  int type[3];
  for (int d = 0; d < 3; ++d) type[d] = (v[d] == 1 ? 1 : 0) | (v[d] == A.n - 1 ? 2 : 0);

  // ---- gather the local right-hand side
  for (int j = tid; j < C::NV + C::NP; j += C::NT) {
    T val;
    if (A.mode == 0)
      val = A.r[patch_global<K>(j, v, A.m)];
    else
      val = (j == (int)blockIdx.x) ? T(1) : T(0);
    if (j < C::NV)
      Fv[j] = val;
    else
      G[j - C::NV] = val;
  }
  __syncthreads();

  // ---- rhs of the Schur system: B A^{-1} F - G, projected to mean zero
  fdm_inverse<K, T>(Fv, V2, V1, tb, type);  // V1 = A^{-1} F
  apply_B<K, T>(V1, R, tb);
  T part = T(0);
  for (int q = tid; q < C::NP; q += C::NT) {
    R[q] -= G[q];
    part += R[q];
  }
  T mean = block_sum<T, C::NW>(part, red) / T(C::NP);
  part = T(0);
  for (int q = tid; q < C::NP; q += C::NT) {
    const T rv = R[q] - mean;
    R[q] = rv;
    Dd[q] = rv;
    Pp[q] = T(0);
    part += rv * rv;
  }
  T rr = block_sum<T, C::NW>(part, red);
  const T rr0 = rr;
  // ---- conjugate gradients on the Schur complement
  for (int it = 0; it < A.cg_iters; ++it) {
    if (A.cg_tol_mode && rr <= A.cg_tol * A.cg_tol * rr0) break;
    if (!(rr > T(0))) break;
    apply_BT<K, T>(Dd, V1, tb);
    fdm_inverse<K, T>(V1, V2, V1, tb, type);
    apply_B<K, T>(V1, Sd, tb);
    part = T(0);
    for (int q = tid; q < C::NP; q += C::NT) part += Dd[q] * Sd[q];
    const T dSd = block_sum<T, C::NW>(part, red);
    if (!(dSd > T(0))) break;
    const T alpha = rr / dSd;
    part = T(0);
    for (int q = tid; q < C::NP; q += C::NT) {
      Pp[q] += alpha * Dd[q];
      const T rv = R[q] - alpha * Sd[q];
      R[q] = rv;
      part += rv;
    }
    mean = block_sum<T, C::NW>(part, red) / T(C::NP);
    part = T(0);
    for (int q = tid; q < C::NP; q += C::NT) {
      const T rv = R[q] - mean;
      R[q] = rv;
      part += rv * rv;
    }
    const T rr_new = block_sum<T, C::NW>(part, red);
    const T beta = rr_new / rr;
    for (int q = tid; q < C::NP; q += C::NT) Dd[q] = R[q] + beta * Dd[q];
    rr = rr_new;
    __syncthreads();
  }
  // ---- velocity: U = A^{-1} (F - B^T P)
  apply_BT<K, T>(Pp, V1, tb);
  for (int i = tid; i < C::NV; i += C::NT) Fv[i] -= V1[i];
  __syncthreads();
  fdm_inverse<K, T>(Fv, V2, V1, tb, type);  // V1 = U
  // ---- scatter
  for (int j = tid; j < C::NV + C::NP; j += C::NT) {
    const T val = (j < C::NV) ? V1[j] : Pp[j - C::NV];
    if (A.mode == 0)
      A.x[patch_global<K>(j, v, A.m)] += val;
    else
      A.cols[(int64_t)blockIdx.x * (C::NV + C::NP) + j] = (double)val;
  }
}

template <int K>
size_t patch_smem_bytes(size_t esize) {
  using C = PatchCfg<K>;
  return esize * (3 * C::NV + 5 * C::NP);
}

template <int K, typename T>
static cudaError_t launch_patch_k(PatchArgs<T> a, int nblocks, cudaStream_t s) {
  using C = PatchCfg<K>;
  const size_t smem = patch_smem_bytes<K>(sizeof(T));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(patch_kernel<K, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (nblocks > 0) patch_kernel<K, T><<<nblocks, C::NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch_patch(int k, PatchArgs<T> a, int nblocks, cudaStream_t s) {
  switch (k) {
    case 1: return launch_patch_k<1, T>(a, nblocks, s);
    case 2: return launch_patch_k<2, T>(a, nblocks, s);
    case 3: return launch_patch_k<3, T>(a, nblocks, s);
    case 4: return launch_patch_k<4, T>(a, nblocks, s);
    case 5: return launch_patch_k<5, T>(a, nblocks, s);
  }
  return cudaErrorInvalidValue;
}

static void colour_counts(int n, int colour, int* cnt) {
  for (int d = 0; d < 3; ++d) {
    const int bit = (colour >> d) & 1;
    cnt[d] = bit ? n / 2 : (n - 1) / 2;  // odd vertices 1,3,..; even vertices 2,4,.. within [1, n-1]
  }
}

template <typename T>
static void fill_common(const stk_problem* P, const Level& L, PatchArgs<T>& a) {
  a.n = L.n;
  a.m = L.m;
  a.cg_iters = P->opt.local_cg_iters;
  a.cg_tol_mode = P->opt.local_cg_mode == STK_CG_TOL;
  a.cg_tol = (T)P->opt.local_cg_tol;
  a.cols = nullptr;
}

cudaError_t launch_patch_colour(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x) {
  const Level& L = P->levels[level];
  int cnt[3];
  colour_counts(L.n, colour, cnt);
  const int nb = cnt[0] * cnt[1] * cnt[2];
  if (dtype == STK_F64) {
    PatchArgs<double> a;
    fill_common(P, L, a);
    a.r = (const double*)r;
    a.x = (double*)x;
    a.tab = L.ptab64;
    a.colour = colour;
    for (int d = 0; d < 3; ++d) a.cnt[d] = cnt[d];
    a.mode = 0;
    return dispatch_patch<double>(P->k, a, nb, P->stream);
  }
  PatchArgs<float> a;
  fill_common(P, L, a);
  a.r = (const float*)r;
  a.x = (float*)x;
  a.tab = L.ptab32;
  a.colour = colour;
  for (int d = 0; d < 3; ++d) a.cnt[d] = cnt[d];
  a.mode = 0;
  return dispatch_patch<float>(P->k, a, nb, P->stream);
}

int patch_local_size(int k) {
  const int npc = 2 * k + 1, npd = 2 * k + 2;
  return 3 * npc * npd * npd + npd * npd * npd;
}

cudaError_t launch_coarse_columns(const stk_problem* P, double* cols, int max_iter, double tol) {
  const Level& L = P->levels[0];
  PatchArgs<double> a;
  fill_common(P, L, a);
  a.r = nullptr;
  a.x = nullptr;
  a.cols = cols;
  a.tab = L.ptab64;
  a.colour = 7;
  a.cnt[0] = a.cnt[1] = a.cnt[2] = 1;
  a.mode = 1;
  a.cg_iters = max_iter;
  a.cg_tol_mode = 1;
  a.cg_tol = tol;
  return dispatch_patch<double>(P->k, a, patch_local_size(P->k), P->stream);
}

// ---------------------------------------------------------------- coarse solve
// x = C b on the 2^3 coarse mesh, C the dense pseudo-inverse in patch-local
// order (column-major, FP64), b and x in the level's global layout.
template <int K, typename T>
__global__ void __launch_bounds__(256) coarse_solve_kernel(const double* __restrict__ Cm, const T* __restrict__ b,
                                                            T* __restrict__ x, int m) {
  using C = PatchCfg<K>;
  constexpr int NL = C::NV + C::NP;
  extern __shared__ __align__(16) unsigned char cs_smem[];
  double* bl = reinterpret_cast<double*>(cs_smem);
  const int v[3] = {1, 1, 1};
  for (int j = threadIdx.x; j < NL; j += blockDim.x) bl[j] = (double)b[patch_global<K>(j, v, m)];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NL) return;
  double acc = 0.0;
  for (int j = 0; j < NL; ++j) acc += Cm[(int64_t)j * NL + i] * bl[j];
  x[patch_global<K>(i, v, m)] = (T)acc;
}

cudaError_t launch_coarse_solve(const stk_problem* P, int dtype, const void* b, void* x) {
  const Level& L = P->levels[0];
  const int NL = patch_local_size(P->k);
  const size_t esize = dtype == STK_F64 ? 8 : 4;
  cudaError_t e = cudaMemsetAsync(x, 0, (size_t)L.ntotal * esize, P->stream);
  if (e != cudaSuccess) return e;
  const int blocks = (NL + 255) / 256;
  const size_t smem = sizeof(double) * NL;
#define STK_CS_CASE(KK)                                                                                       \
  case KK: {                                                                                                  \
    static bool attr64 = false, attr32 = false;                                                               \
    if (dtype == STK_F64) {                                                                                   \
      if (!attr64) {                                                                                          \
        e = cudaFuncSetAttribute(coarse_solve_kernel<KK, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                                  \
        if (e != cudaSuccess) return e;                                                                       \
        attr64 = true;                                                                                        \
      }                                                                                                       \
      coarse_solve_kernel<KK, double><<<blocks, 256, smem, P->stream>>>(P->coarse_inv, (const double*)b,      \
                                                                          (double*)x, L.m);                  \
    } else {                                                                                                  \
      if (!attr32) {                                                                                          \
        e = cudaFuncSetAttribute(coarse_solve_kernel<KK, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 (int)smem);                                                                  \
        if (e != cudaSuccess) return e;                                                                       \
        attr32 = true;                                                                                        \
      }                                                                                                       \
      coarse_solve_kernel<KK, float><<<blocks, 256, smem, P->stream>>>(P->coarse_inv, (const float*)b,        \
                                                                         (float*)x, L.m);                    \
    }                                                                                                         \
    break;                                                                                                    \
  }
  switch (P->k) {
    STK_CS_CASE(1)
    STK_CS_CASE(2)
    STK_CS_CASE(3)
    STK_CS_CASE(4)
    STK_CS_CASE(5)
    default:
      return cudaErrorInvalidValue;
  }
#undef STK_CS_CASE
  return cudaGetLastError();
}

}  // namespace stk
