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
//
// This file holds the host side: colour counts, the interior/boundary
// launch split, the Direct local inverses, the coarse pseudo-inverse
// columns and the 2^3 coarse solve.  The patch kernels (gather, Schur-CG
// or Direct local solve by fast diagonalization, scatter) are in
// patch_kernel.cuh.
#include <cublas_v2.h>

#include <algorithm>

#include "patch_kernel.cuh"

namespace stk {

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

template <typename T>
static cudaError_t dispatch_patch_multi(int k, const PatchArgs<T>& a, const PatchJobs<T>& J, int nblocks,
                                        cudaStream_t s) {
  switch (k) {
    case 1: return launch_patch_multi_k<1, T>(a, J, nblocks, s);
    case 2: return launch_patch_multi_k<2, T>(a, J, nblocks, s);
    case 3: return launch_patch_multi_k<3, T>(a, J, nblocks, s);
    case 4: return launch_patch_multi_k<4, T>(a, J, nblocks, s);
    case 5: return launch_patch_multi_k<5, T>(a, J, nblocks, s);
  }
  return cudaErrorInvalidValue;
}

static void colour_counts(int n, int colour, int* cnt) {
  for (int d = 0; d < 3; ++d) {
    const int bit = (colour >> d) & 1;
    cnt[d] = bit ? n / 2 : (n - 1) / 2;  // odd vertices 1,3,..; even vertices 2,4,.. within [1, n-1]
  }
}

// An FP32 CG stagnates near 1e-6 relative; below that a TOL-mode local solve
// would run to its step limit and spoil the smoother.
constexpr double kMinTolF32 = 1e-6;

template <typename T>
static T local_tol(double tol) {
  return (T)(sizeof(T) == 4 ? std::max(tol, kMinTolF32) : tol);
}

template <typename T>
static void fill_common(const stk_problem* P, const Level& L, PatchArgs<T>& a) {
  a.n = L.n;
  a.m = L.m;
  a.cg_iters = P->opt.local_cg_iters;
  a.cg_tol_mode = P->opt.local_cg_mode == STK_CG_TOL;
  a.cg_tol = local_tol<T>(P->opt.local_cg_tol);
  a.cols = nullptr;
  a.xin = nullptr;
  a.b = nullptr;
  a.ctab = nullptr;
  a.part = 0;
  a.dir = nullptr;
  a.gemm_phase = 0;
  a.rout = nullptr;
  a.pin = nullptr;
  if constexpr (sizeof(T) == 8)
    a.htab = &L.hptab64;
  else
    a.htab = &L.hptab32;
  for (int d = 0; d < 3; ++d) a.tlo[d] = a.cint[d] = a.btype[d] = 0;
}

constexpr int kGemmMinPatches = 512;  // interior patches per colour from which the Direct product is a GEMM

// The cuBLAS handle and workspace of a problem (first call outside any
// capture: the smoothing step that builds the Direct inverses makes it).
static cudaError_t ensure_blas(stk_problem* P, size_t ws_bytes) {
  if (!P->blas) {
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    P->blas = h;
  }
  if (P->blas_ws_bytes < ws_bytes) {
    if (P->blas_ws) cudaFree(P->blas_ws);
    P->blas_ws = nullptr;
    P->blas_ws_bytes = 0;
    cudaError_t e = dev_alloc(&P->blas_ws, ws_bytes);
    if (e != cudaSuccess) return e;
    P->blas_ws_bytes = ws_bytes;
  }
  cublasHandle_t h = static_cast<cublasHandle_t>(P->blas);
  if (cublasSetWorkspace(h, P->blas_ws, P->blas_ws_bytes) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  return cudaSuccess;
}

// P = M R for the `ni` interior patches of a colour: C (np x ni) = M (np x np)
// R (np x ni), column-major; M symmetric, the type-0 inverse of the level
static cudaError_t direct_gemm(const stk_problem* P, const Level& L, int ni) {
  const int np = (2 * P->k + 2) * (2 * P->k + 2) * (2 * P->k + 2);
  cublasHandle_t h = static_cast<cublasHandle_t>(P->blas);
  if (cublasSetStream(h, P->stream) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  const float one = 1.0f, zero = 0.0f;
  const cublasComputeType_t ct =
      P->opt.direct_gemm == 2 ? CUBLAS_COMPUTE_32F_EMULATED_16BFX9 : CUBLAS_COMPUTE_32F_PEDANTIC;
  const cublasStatus_t st = cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, np, ni, np, &one, L.dir32_host[0], CUDA_R_32F,
                                         np, L.gemmR, CUDA_R_32F, np, &zero, L.gemmP, CUDA_R_32F, np, ct,
                                         CUBLAS_GEMM_DEFAULT);
  return st == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

constexpr int kSplitInterior = 8192;  // interior patches per colour from which they get their own launch
constexpr int kSplitInteriorF32 = 1024;  // FP32, whose interior kernel reads its matrices from the constant bank

// The interior patches of a colour (2 <= v <= n-2 in every direction) form a
// box of the colour's patch grid: t in [tlo, tlo + cint) per direction.
static void interior_box(int n, int colour, const int* cnt, int* tlo, int* cint) {
  for (int d = 0; d < 3; ++d) {
    const int bit = (colour >> d) & 1;
    int lo = cnt[d], hi = 0;
    for (int t = 0; t < cnt[d]; ++t) {
      const int v = bit ? 2 * t + 1 : 2 * t + 2;
      if (v >= 2 && v <= n - 2) {
        lo = std::min(lo, t);
        hi = std::max(hi, t + 1);
      }
    }
    tlo[d] = lo;
    cint[d] = std::max(0, hi - lo);
  }
}

// One colour of patch solves.  xin == NULL: the patch residuals are read from
// r (mode 0) and x is updated in place; else they are computed in the kernel
// from xin and b (mode 3, r is the right-hand side b) and x receives
// xin + the corrections at the patch DoFs.
template <typename T>
static cudaError_t patch_colour(const stk_problem* P, const Level& L, const PatchTables<T>* tab, int colour,
                                const void* r, void* x, int cg_tol_mode, int cg_iters, double cg_tol,
                                const void* xin = nullptr) {
  int cnt[3];
  colour_counts(L.n, colour, cnt);
  const int nb = cnt[0] * cnt[1] * cnt[2];
  PatchArgs<T> a;
  fill_common(P, L, a);
  a.r = (const T*)r;
  a.x = (T*)x;
  a.tab = tab;
  a.colour = colour;
  for (int d = 0; d < 3; ++d) a.cnt[d] = cnt[d];
  a.mode = 0;
  if (xin) {
    a.mode = 3;
    a.r = nullptr;
    a.xin = (const T*)xin;
    a.b = (const T*)r;
    if constexpr (sizeof(T) == 8)
      a.ctab = L.tab64;
    else
      a.ctab = L.tab32;
  }
  a.cg_tol_mode = cg_tol_mode;
  a.cg_iters = cg_iters;
  a.cg_tol = local_tol<T>(cg_tol);
  if (P->opt.local_cg_mode == STK_LOCAL_DIRECT && L.dir_ready) {
    if constexpr (sizeof(T) == 8)
      a.dir = L.dirtab64;
    else
      a.dir = L.dirtab32;
  }
  interior_box(L.n, colour, cnt, a.tlo, a.cint);
  const int ni = a.cint[0] * a.cint[1] * a.cint[2];
  // FP32 Direct: the interior patches' products as one GEMM (M read once per
  // colour instead of once per patch), then the boundary patches as usual
  if constexpr (sizeof(T) == 4) {
    if (a.dir && !xin && P->opt.direct_gemm && L.eo_interior && ni >= kGemmMinPatches && L.gemm_cap >= ni &&
        P->blas && L.dir32_host[0]) {
      a.part = 1;
      a.gemm_phase = 1;
      a.rout = L.gemmR;
      cudaError_t e = dispatch_patch<T>(P->k, a, ni, P->stream);
      if (e == cudaSuccess) e = direct_gemm(P, L, ni);
      if (e != cudaSuccess) return e;
      a.gemm_phase = 2;
      a.rout = nullptr;
      a.pin = L.gemmP;
      e = dispatch_patch<T>(P->k, a, ni, P->stream);
      if (e != cudaSuccess || ni == nb) return e;
      a.gemm_phase = 0;
      a.pin = nullptr;
      a.part = 2;
      return dispatch_patch<T>(P->k, a, nb, P->stream);
    }
  }
  // Interior patches in their own launch (no dense transforms compiled in),
  // then the rest: 3-9 % faster per smoothing step at 64^3 (k = 2..4); at
  // 32^3 and below the second launch and its serialized tail cost as much,
  // except in FP32, whose interior kernel is ~20 % faster than the general
  // one (6 % faster smoothing at 32^3, k = 3).  stk_autotune may have timed
  // both per level.
  const int pick = L.split_pick[sizeof(T) == 8 ? STK_F64 : STK_F32];
  const int thr = sizeof(T) == 4 ? kSplitInteriorF32 : kSplitInterior;
  const bool split = L.eo_interior && ni > 0 && (pick >= 0 ? pick == 1 : ni >= thr);
  if (!split) return dispatch_patch<T>(P->k, a, nb, P->stream);
  a.part = 1;
  cudaError_t e = dispatch_patch<T>(P->k, a, ni, P->stream);
  if (e != cudaSuccess || ni == nb) return e;
  a.part = 2;
  return dispatch_patch<T>(P->k, a, nb, P->stream);
}

cudaError_t launch_patch_colour_cg(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x,
                                   int cg_tol_mode, int cg_iters, double cg_tol) {
  const Level& L = P->levels[level];
  if (dtype == STK_F64) return patch_colour<double>(P, L, L.ptab64, colour, r, x, cg_tol_mode, cg_iters, cg_tol);
  return patch_colour<float>(P, L, L.ptab32, colour, r, x, cg_tol_mode, cg_iters, cg_tol);
}

cudaError_t launch_patch_colour(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x) {
  return launch_patch_colour_cg(P, level, dtype, colour, r, x, P->opt.local_cg_mode == STK_CG_TOL,
                                P->opt.local_cg_iters, P->opt.local_cg_tol);
}

cudaError_t launch_patch_colour_fused(const stk_problem* P, int level, int dtype, int colour, const void* xin,
                                      const void* b, void* xout) {
  const Level& L = P->levels[level];
  const int tolm = P->opt.local_cg_mode == STK_CG_TOL;
  if (dtype == STK_F64)
    return patch_colour<double>(P, L, L.ptab64, colour, b, xout, tolm, P->opt.local_cg_iters, P->opt.local_cg_tol,
                                xin);
  return patch_colour<float>(P, L, L.ptab32, colour, b, xout, tolm, P->opt.local_cg_iters, P->opt.local_cg_tol, xin);
}

// x_out = x_in at every entry that no patch of the colour owns: the normal
// nodes on the patch boundaries, the cells no patch of the colour covers and
// the constrained entries (the fused colour writes only the patch DoFs).  A
// cell j along a direction is covered when a vertex v of the colour (v in
// [1, n-1], v = bit mod 2) has j in {v-1, v}; a continuous-direction node on
// the cell boundary w is owned only when w is such a vertex (the patch's
// middle node).
template <typename T>
__global__ void copy_unowned_kernel(const T* __restrict__ xin, T* __restrict__ xout, int n, int k, int colour) {
  const int nd = k + 1, m = n * nd;
  const int64_t nvel = (int64_t)(m + 1) * m * m, N = 3 * nvel + (int64_t)m * m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    int c = 3;
    int64_t loc = e - 3 * nvel;
    if (e < 3 * nvel) {
      c = (int)(e / nvel);
      loc = e - c * nvel;
    }
    const int64_t E0 = (c == 0) ? m + 1 : m, E1 = (c == 1) ? m + 1 : m;
    const int idx[3] = {(int)(loc % E0), (int)((loc / E0) % E1), (int)(loc / (E0 * E1))};
    bool owned = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int bit = (colour >> d) & 1, i = idx[d];
      if (d == c) {
        if (i % nd == 0) {
          const int w = i / nd;
          owned = owned && w >= 1 && w <= n - 1 && (w & 1) == bit;
          continue;
        }
      }
      const int j = min(i / nd, n - 1);
      const bool cov = (j >= 1 && ((j & 1) == bit)) || (j + 1 <= n - 1 && (((j + 1) & 1) == bit));
      owned = owned && cov;
    }
    if (!owned) xout[e] = xin[e];
  }
}

cudaError_t launch_copy_unowned(const stk_problem* P, int level, int dtype, int colour, const void* xin, void* xout) {
  const Level& L = P->levels[level];
  const int blocks = (int)std::min<int64_t>((L.ntotal + 255) / 256, 152 * 8);
  if (dtype == STK_F64)
    copy_unowned_kernel<double><<<blocks, 256, 0, P->stream>>>((const double*)xin, (double*)xout, L.n, P->k, colour);
  else
    copy_unowned_kernel<float><<<blocks, 256, 0, P->stream>>>((const float*)xin, (float*)xout, L.n, P->k, colour);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t patch_colour_multi(const stk_problem* const* Ps, const int* levels, int count, int colour,
                                      void* const* r, void* const* x, cudaStream_t stream) {
  for (int i0 = 0; i0 < count; i0 += kMaxPatchJobs) {
    const int nj = std::min(kMaxPatchJobs, count - i0);
    PatchArgs<T> a;
    fill_common(Ps[0], Ps[0]->levels[levels[0]], a);
    a.r = nullptr;
    a.x = nullptr;
    a.tab = nullptr;
    a.colour = colour;
    a.mode = 0;
    PatchJobs<T> J{};
    J.count = nj;
    int total = 0;
    for (int j = 0; j < nj; ++j) {
      const stk_problem* P = Ps[i0 + j];
      const Level& L = P->levels[levels[i0 + j]];
      int cnt[3];
      colour_counts(L.n, colour, cnt);
      J.first[j] = total;
      J.r[j] = (const T*)r[i0 + j];
      J.x[j] = (T*)x[i0 + j];
      if constexpr (sizeof(T) == 8)
        J.tab[j] = L.ptab64;
      else
        J.tab[j] = L.ptab32;
      J.n[j] = L.n;
      J.m[j] = L.m;
      for (int d = 0; d < 3; ++d) J.cnt[j][d] = cnt[d];
      total += cnt[0] * cnt[1] * cnt[2];
    }
    cudaError_t e = dispatch_patch_multi<T>(Ps[0]->k, a, J, total, stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_patch_colour_multi(const stk_problem* const* Ps, const int* levels, int count, int dtype,
                                      int colour, void* const* r, void* const* x, cudaStream_t stream) {
  if (dtype == STK_F64) return patch_colour_multi<double>(Ps, levels, count, colour, r, x, stream);
  return patch_colour_multi<float>(Ps, levels, count, colour, r, x, stream);
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// The Direct local solver of a level: for every patch type (t0, t1, t2) that
// occurs, the columns S e_q of its Schur complement (patch kernel, mode 2,
// FP64), then (S + a 1 1^T)^{-1} in place, plus an FP32 copy.  Built once,
// synchronously; a failure leaves nothing allocated.
cudaError_t ensure_direct(stk_problem* P, int level) {
  Level& L = P->levels[level];
  if (L.dir_ready) return cudaSuccess;
  const int npd = 2 * P->k + 2;
  const int64_t np = (int64_t)npd * npd * npd, nn = np * np;
  bool present[4] = {false, false, false, false};
  for (int v = 1; v <= L.n - 1; ++v) present[(v == 1 ? 1 : 0) | (v == L.n - 1 ? 2 : 0)] = true;
  std::vector<int> combos;
  for (int t2 = 0; t2 < 4; ++t2)
    for (int t1 = 0; t1 < 4; ++t1)
      for (int t0 = 0; t0 < 4; ++t0)
        if (present[t0] && present[t1] && present[t2]) combos.push_back(t0 + 4 * t1 + 16 * t2);
  const int nc = (int)combos.size();
  cudaError_t e = dev_alloc(&L.dirM64, sizeof(double) * nn * nc);
  if (e == cudaSuccess) e = dev_alloc(&L.dirM32, sizeof(float) * nn * nc);
  if (e == cudaSuccess) e = dev_alloc(&L.dirtab64, sizeof(double*) * 64);
  if (e == cudaSuccess) e = dev_alloc(&L.dirtab32, sizeof(float*) * 64);
  std::vector<const double*> t64(64, nullptr);
  std::vector<const float*> t32(64, nullptr);
  for (int i = 0; e == cudaSuccess && i < nc; ++i) {
    const int c = combos[i];
    double* S = L.dirM64 + nn * i;
    PatchArgs<double> a;
    fill_common(P, L, a);
    a.r = nullptr;
    a.x = nullptr;
    a.cols = S;
    a.tab = L.ptab64;
    a.colour = 0;
    a.cnt[0] = a.cnt[1] = a.cnt[2] = 1;
    a.mode = 2;
    a.btype[0] = c % 4;
    a.btype[1] = (c / 4) % 4;
    a.btype[2] = c / 16;
    e = dispatch_patch<double>(P->k, a, (int)np, P->stream);
    if (e == cudaSuccess) e = invert_shifted(S, np, np, P->stream);
    if (e == cudaSuccess) {
      to_float_kernel<<<(unsigned)std::min<int64_t>((nn + 255) / 256, 4096), 256, 0, P->stream>>>(
          S, L.dirM32 + nn * i, nn);
      e = cudaGetLastError();
    }
    t64[c] = S;
    t32[c] = L.dirM32 + nn * i;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.dirtab64, t64.data(), sizeof(double*) * 64, cudaMemcpyHostToDevice, P->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.dirtab32, t32.data(), sizeof(float*) * 64, cudaMemcpyHostToDevice, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  // the GEMM form of the FP32 product: R and P of the most interior patches
  // any colour has, and the cuBLAS handle (never during a capture: the first
  // smoothing step of the level runs this)
  int64_t ni_max = 0;
  for (int colour = 0; colour < 8; ++colour) {
    int cnt[3], tlo[3], cint[3];
    colour_counts(L.n, colour, cnt);
    interior_box(L.n, colour, cnt, tlo, cint);
    ni_max = std::max<int64_t>(ni_max, (int64_t)cint[0] * cint[1] * cint[2]);
  }
  if (e == cudaSuccess && P->opt.direct_gemm && L.eo_interior && ni_max >= kGemmMinPatches && present[0]) {
    e = dev_alloc(&L.gemmR, sizeof(float) * (size_t)(ni_max * np));
    if (e == cudaSuccess) e = dev_alloc(&L.gemmP, sizeof(float) * (size_t)(ni_max * np));
    if (e == cudaSuccess) e = ensure_blas(P, std::max<size_t>(size_t(64) << 20, sizeof(float) * 3 * (size_t)(ni_max * np)));
    if (e == cudaSuccess) L.gemm_cap = ni_max;
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(P->stream);
    for (void* p : {(void*)L.dirM64, (void*)L.dirM32, (void*)L.dirtab64, (void*)L.dirtab32, (void*)L.gemmR, (void*)L.gemmP})
      if (p) cudaFree(p);
    L.dirM64 = nullptr;
    L.dirM32 = nullptr;
    L.dirtab64 = nullptr;
    L.dirtab32 = nullptr;
    L.gemmR = nullptr;
    L.gemmP = nullptr;
    L.gemm_cap = 0;
    return e;
  }
  for (int c = 0; c < 64; ++c) L.dir32_host[c] = t32[c];
  L.dir_ready = true;
  return cudaSuccess;
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
    static std::atomic<unsigned long long> set64{0}, set32{0};                                               \
    if (dtype == STK_F64) {                                                                                   \
      e = allow_dynamic_smem(coarse_solve_kernel<KK, double>, smem, set64);                                   \
      if (e != cudaSuccess) return e;                                                                         \
      coarse_solve_kernel<KK, double><<<blocks, 256, smem, P->stream>>>(P->coarse_inv, (const double*)b,      \
                                                                          (double*)x, L.m);                  \
    } else {                                                                                                  \
      e = allow_dynamic_smem(coarse_solve_kernel<KK, float>, smem, set32);                                    \
      if (e != cudaSuccess) return e;                                                                         \
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
