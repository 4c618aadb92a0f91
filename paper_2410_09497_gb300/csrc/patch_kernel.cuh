// Device side of the coloured vertex-patch smoother: the patch kernels.
//
// Fast diagonalization (eq. `inverse2d`, eq. `fast_inverse` in 3D): per
// velocity component c,  A_c^{-1} = (1/nu) S_c Lam_c^{-1} S_c^T  with
// S_c = S_x (x) S_y (x) S_z (continuous-direction eigenvectors along c,
// discontinuous ones along the other two).  Because B_c = D (x) W (x) W
// (eq. `b`) is a Kronecker product too, so is  B_c S_c = (D S) (x) (W S) (x) (W S),
// and the Schur operator is  S = (1/nu) sum_c (B_c S_c) Lam_c^{-1} (B_c S_c)^T.
// One CG step is therefore six passes of batched 1D line transforms (three
// from pressure space to the scaled eigen-coefficients, three back) over all
// three components, instead of B^T, A^{-1} (six passes) and B separately;
// for k <= 3 the two middle ones run as one pass in registers.  Symmetric
// 1D eigenbases (the continuous direction, interior patches) transform lines
// in even-odd form: half the products and matrix loads.
//   start:  Ft_c = S_c^T F_c,  R = sum_c (B_c S_c) Lam_c^{-1} Ft_c / nu - G
//   end:    U_c = S_c Lam_c^{-1} (Ft_c - (B_c S_c)^T P) / nu
// Every patch tensor lives in shared memory in a (2k+3) x (2k+2) x (2k+2)
// box (odd x stride: strided line accesses hit distinct banks).
//
// The same kernel, with the right-hand side set to unit vectors, builds the
// dense pseudo-inverse of the coarse problem at setup: on a 2^3 mesh the one
// vertex patch holds every free DoF.  Two more kernels share the patch
// solve: one for the interior patches of a large level (no dense transforms
// compiled in) and one for a colour of several problems in one launch.
//
// Included by the patch_k<K>.cu files, one per degree, so that the
// degrees compile in parallel, and by smoother.cu for the argument types
// and the patch-local numbering of the coarse solve.
#pragma once

#include "internal.h"

namespace stk {

template <int K>
struct PatchCfg {
  static constexpr int ND = K + 1, NPC = 2 * K + 1, NPD = 2 * K + 2;
  static constexpr int NV1 = NPC * NPD * NPD;  // one velocity component (unpadded)
  static constexpr int NV = 3 * NV1;
  static constexpr int NP = NPD * NPD * NPD;
  static constexpr int BX = NPD + 1;           // padded x extent of every patch tensor
  static constexpr int BOX = BX * NPD * NPD;   // one padded tensor
  static constexpr int LPC = NPD * NPD;       // lines of one component along a direction
};

// Threads of a patch CTA.  A pass transforms LPC lines of each component.  W
// warps serve one component (warp-uniform component: no divergence) and each
// thread transforms R lines with every matrix entry it loads: the broadcast
// loads of the transform matrices are what the shared-memory pipe spends most
// of its wavefronts on.  FP32 at k = 3: two warps per component (one line per
// thread, twice the warps per SM to hide the latency of the passes) measured
// 5 % faster per smoothing step than one; FP64 at k = 3 measured 5 % slower
// that way (register spills at 3 CTAs per SM).
template <int K, typename T>
struct PatchThreads {
  static constexpr int W = sizeof(T) == 4 ? ((K <= 2) ? 1 : (K <= 4 ? 2 : 3)) : ((K <= 3) ? 1 : (K == 4 ? 2 : 3));
  static constexpr int TPC = 32 * W;
  static constexpr int R = (PatchCfg<K>::LPC + TPC - 1) / TPC;
  static constexpr int NT = 3 * TPC;
  static constexpr int NW = NT / 32;
};

// The four transform matrices of an interior patch (every 1D basis of type
// 0: SC, SD[0], EC, FM[0]), passed to the interior-patch kernel by value.
// Their warp-uniform reads at compile-time offsets come from the constant
// bank as FMA operands instead of shared-memory broadcasts, which the
// shared-memory pipe (the interior kernel's bound) no longer has to serve.
template <int K, typename T>
struct InteriorMats {
  static constexpr int NPD = 2 * K + 2;
  static constexpr int NE = sizeof(T) == 4 ? NPD * kRowStride : 1;  // FP64 reads its shared tables
  T SC[NE], SD[NE], EC[NE], FM[NE];
};

// Resident CTAs per SM the register budget must allow: as many as the shared
// memory of one patch (13 padded tensors + tables) permits, except FP32 at
// k = 3, where 5 CTAs of 6 warps (68 registers a thread) measured 3 % faster
// than the 6 shared memory allows (56 registers, with spills).
template <int K, typename T>
struct PatchOcc {
  static constexpr int value = sizeof(T) == 4 ? ((K == 1) ? 12 : (K == 2) ? 8 : (K == 3) ? 5 : (K == 4) ? 3 : 2)
                                              : ((K == 1) ? 8 : (K == 2) ? 4 : (K == 3) ? 3 : 1);
};

template <typename T>
struct PatchArgs {
  const T* r;     // colour residual (mode 0)
  T* x;           // solution, updated in place (mode 0); the output x_out (mode 3)
  const T* xin;   // mode 3: the solution before the colour (x_in), read only
  const T* b;     // mode 3: right-hand side
  const CellTables<T>* ctab;  // mode 3: the level's 1D cell matrices
  double* cols;   // mode 1: column-major output, N_p x N_p
  const PatchTables<T>* tab;
  const PatchTables<T>* htab;  // host copy of *tab: the launcher passes the interior matrices from it
  int n, m;
  int colour;
  int cnt[3];     // patches of the colour per direction
  int part;       // mode 0: 0 every patch, 1 interior patches only, 2 boundary patches only
  int tlo[3], cint[3];  // the interior patches: t in [tlo, tlo + cint) per direction
  int mode;       // 0: smoother colour, 1: coarse pseudo-inverse columns, 2: Schur complement columns,
                  // 3: smoother colour with the patch residual computed in the kernel (fused)
  const T* const* dir;  // mode 0: (S + a 1 1^T)^{-1} per patch type t0 + 4 t1 + 16 t2 (NULL: CG)
  int btype[3];   // mode 2: the patch type in each direction
  int cg_iters;   // FIXED: exact count; TOL: limit
  int cg_tol_mode;
  T cg_tol;
  // Direct local solver as one GEMM per colour (mode 0, interior launch):
  // phase 1 writes each patch's mean-free Schur right-hand side R to
  // rout[blk * NP ...] and stops; phase 2 reads the solution P = M R from
  // pin[blk * NP ...] and finishes the patch (0: the product in the kernel)
  int gemm_phase;
  T* rout;
  const T* pin;
};

// Per-problem fields of a multi-problem colour launch (passed by value).
template <typename T>
struct PatchJobs {
  int count;
  int first[kMaxPatchJobs];  // first CTA of each problem
  const T* r[kMaxPatchJobs];
  T* x[kMaxPatchJobs];
  const PatchTables<T>* tab[kMaxPatchJobs];
  int n[kMaxPatchJobs], m[kMaxPatchJobs];
  int cnt[kMaxPatchJobs][3];
};

// Block-wide sums with one barrier: callers alternate between two red
// buffers, so the previous reads of a buffer are always separated from its
// next writes by at least one barrier.
template <typename T, int NW>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
#pragma unroll
  for (int i = 0; i < NW; ++i) s += red[i];
  return s;
}

// two sums at once
template <typename T, int NW>
__device__ __forceinline__ void block_sum2(T& a, T& b, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[w] = a;
    red[NW + w] = b;
  }
  __syncthreads();
  a = T(0);
  b = T(0);
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    a += red[i];
    b += red[NW + i];
  }
}

__device__ __forceinline__ int box_stride(int d, int bx, int npd) { return d == 0 ? 1 : (d == 1 ? bx : bx * npd); }

// 16-byte vector of a matrix row
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int width = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int width = 2;
};
__device__ __forceinline__ void vec_fma(float* r, const float4& w, float s) {
  r[0] += w.x * s;
  r[1] += w.y * s;
  r[2] += w.z * s;
  r[3] += w.w * s;
}
__device__ __forceinline__ void vec_fma(double* r, const double2& w, double s) {
  r[0] += w.x * s;
  r[1] += w.y * s;
}
__device__ __forceinline__ float vget(const float4& w, int e) { return e == 0 ? w.x : e == 1 ? w.y : e == 2 ? w.z : w.w; }
__device__ __forceinline__ double vget(const double2& w, int e) { return e == 0 ? w.x : w.y; }

// VW consecutive entries of a transform matrix row, from M + off: one 16-byte
// shared-memory load, or (SCAL) VW scalar reads, which the compiler takes
// straight from the constant bank as FMA operands when M is a kernel
// parameter and off is known at compile time.
template <bool SCAL, typename T>
__device__ __forceinline__ typename Vec16<T>::type mat_vec(const T* __restrict__ M, int off) {
  if constexpr (SCAL) {
    if constexpr (sizeof(T) == 4)
      return make_float4(M[off], M[off + 1], M[off + 2], M[off + 3]);
    else
      return make_double2(M[off], M[off + 1]);
  } else {
    return *reinterpret_cast<const typename Vec16<T>::type*>(M + off);
  }
}

// Even-odd line transforms (Kronbichler-style symmetry of a 1D eigenbasis).
// The rows of M are indexed by nodes paired by the patch reflection
// i <-> NR-1-i (P pairs, plus a centre node P when CEN, NR = 2P+1); the
// columns are eigenvectors, HE even ones then HO odd ones, and
// M[NR-1-i][j] = SIG s_j M[i][j] with s_j = +1 (even) / -1 (odd).
// Forward: out_j = sum_i M[i][j] v_i over rows; backward: out_i = sum_j
// M[i][j] v_j.  Each needs only the first P (+1) rows and half the products.
// Outputs past the real extent are zero.
template <int N, int NR, int P, bool CEN, int SIG, int HE, int HO, int R, typename T, bool SCAL = false>
__device__ __forceinline__ void eo_fwd(const T* __restrict__ M, const T (&v)[R][N], T (&res)[R][N]) {
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::width;
  constexpr int NCOL = HE + HO, NVEC = (NCOL + VW - 1) / VW;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < N; ++j) res[r][j] = T(0);
#pragma unroll
  for (int i = 0; i < P; ++i) {
    T a[R], b[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const T x = v[r][i], y = v[r][NR - 1 - i];
      a[r] = SIG > 0 ? x + y : x - y;  // feeds the even columns
      b[r] = SIG > 0 ? x - y : x + y;  // feeds the odd columns
    }
#pragma unroll
    for (int q = 0; q < NVEC; ++q) {
      const V w = mat_vec<SCAL, T>(M, i * kRowStride + q * VW);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int j = q * VW + e;
        if (j < NCOL)
#pragma unroll
          for (int r = 0; r < R; ++r) res[r][j] = fma(vget(w, e), j < HE ? a[r] : b[r], res[r][j]);
      }
    }
  }
  if (CEN) {
#pragma unroll
    for (int q = 0; q < (HE + VW - 1) / VW; ++q) {
      const V w = mat_vec<SCAL, T>(M, P * kRowStride + q * VW);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int j = q * VW + e;
        if (j < HE)
#pragma unroll
          for (int r = 0; r < R; ++r) res[r][j] = fma(vget(w, e), v[r][P], res[r][j]);
      }
    }
  }
}

template <int N, int NR, int P, bool CEN, int SIG, int HE, int HO, int R, typename T, bool SCAL = false>
__device__ __forceinline__ void eo_bwd(const T* __restrict__ M, const T (&v)[R][N], T (&res)[R][N]) {
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::width;
  constexpr int NCOL = HE + HO, NVEC = (NCOL + VW - 1) / VW;
#pragma unroll
  for (int i = 0; i < P + (CEN ? 1 : 0); ++i) {
    T E[R], O[R];
#pragma unroll
    for (int r = 0; r < R; ++r) E[r] = O[r] = T(0);
#pragma unroll
    for (int q = 0; q < NVEC; ++q) {
      const V w = mat_vec<SCAL, T>(M, i * kRowStride + q * VW);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int j = q * VW + e;
        if (j < HE) {
#pragma unroll
          for (int r = 0; r < R; ++r) E[r] = fma(vget(w, e), v[r][j], E[r]);
        } else if (j < NCOL && i < P) {
#pragma unroll
          for (int r = 0; r < R; ++r) O[r] = fma(vget(w, e), v[r][j], O[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (i < P) {
        res[r][i] = E[r] + O[r];
        res[r][NR - 1 - i] = SIG > 0 ? E[r] - O[r] : O[r] - E[r];
      } else {
        res[r][i] = E[r];  // centre node: odd eigenvectors vanish there
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = NR; j < N; ++j) res[r][j] = T(0);
}

__device__ __forceinline__ float vec_dot_acc(const float4& w, const float* v, float acc) {
  acc = fmaf(w.x, v[0], acc);
  acc = fmaf(w.y, v[1], acc);
  acc = fmaf(w.z, v[2], acc);
  return fmaf(w.w, v[3], acc);
}
__device__ __forceinline__ double vec_dot_acc(const double2& w, const double* v, double acc) {
  return fma(w.y, v[1], fma(w.x, v[0], acc));
}

// pass kinds: velocity eigen-transform (S^T: VEL_FWD, S: VEL_BWD), pressure to
// eigen-coefficients ((B S)^T: BT), eigen-coefficients to pressure (B S: BF)
enum { VEL_FWD = 0, VEL_BWD = 1, BT = 2, BF = 3, BTBF = 4 };
// epilogues of a pass
enum { EPI_NONE = 0, EPI_SCALE = 1, EPI_FT_AND_SCALE = 2, EPI_SUB_SCALE = 3 };

struct PatchGeo {
  int type[3];
  __device__ __forceinline__ int t(int d) const { return d == 0 ? type[0] : (d == 1 ? type[1] : type[2]); }
};

// One pass: every line along direction d of the three component tensors.
// Every tensor is handled as (2k+2)^3 in its padded box: the continuous
// direction of a velocity component has 2k+1 nodes, the extra node holds zero
// (zero rows / columns of SC and EC), so all lines have the same length and
// compile-time loop bounds.  Thread u of component c (warps c W .. c W + W-1)
// owns lines u, u + TPC, ... of that component.  in_shared: all components
// read the same (pressure) box.  Epilogues scale by
// inv_nu / (lam_0 + lam_1 + lam_2) of the output node (the last pass of a
// chain toward eigen-coefficients).
// inv_nu / lam: FP32 epilogues use the hardware reciprocal (2 ulp), FP64 the
// correctly rounded division.
__device__ __forceinline__ float scale_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double scale_div(double a, double b) { return a / b; }

// R lines through one 1D transform: FWD out_j = sum_i M[i][j] v_i (S^T, (B S)^T),
// otherwise out_i = sum_j M[i][j] v_j (S, B S).  VELM: velocity eigenvectors
// (SC / SD[t]) or the divergence / mass factors in the eigenbasis (EC / FM[t]).
template <int K, typename T, bool FWD, bool VELM, int R, bool EO_ALL, bool SCAL = false>
__device__ __forceinline__ void line_transform(const T* __restrict__ M, bool eo, bool along_c,
                                               const T (&v)[R][PatchCfg<K>::NPD], T (&res)[R][PatchCfg<K>::NPD]) {
  using C = PatchCfg<K>;
  constexpr int N = C::NPD, NPC = C::NPC;
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::width;
  constexpr int NV = N / VW, TAIL = N - NV * VW;  // N is even: TAIL is 0 or (FP32) 2
  if (EO_ALL || eo) {
    if (along_c) {
      if (VELM) {
        if (FWD)
          eo_fwd<N, NPC, K, true, 1, K + 1, K, R, T, SCAL>(M, v, res);
        else
          eo_bwd<N, NPC, K, true, 1, K + 1, K, R, T, SCAL>(M, v, res);
      } else {
        if (FWD)
          eo_fwd<N, N, K + 1, false, -1, K + 1, K, R, T, SCAL>(M, v, res);
        else
          eo_bwd<N, N, K + 1, false, -1, K + 1, K, R, T, SCAL>(M, v, res);
      }
    } else {
      if (FWD)
        eo_fwd<N, N, K + 1, false, 1, K + 1, K + 1, R, T, SCAL>(M, v, res);
      else
        eo_bwd<N, N, K + 1, false, 1, K + 1, K + 1, R, T, SCAL>(M, v, res);
    }
  } else if (FWD) {
    // one vector load feeds VW outputs of R lines
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int j = 0; j < N; ++j) res[r][j] = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const T* row = M + i * kRowStride;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const V w = reinterpret_cast<const V*>(row)[q];
#pragma unroll
        for (int r = 0; r < R; ++r) vec_fma(res[r] + q * VW, w, v[r][i]);
      }
      if (TAIL) {
        const float2 w = *reinterpret_cast<const float2*>(row + NV * VW);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          res[r][NV * VW] = fma((T)w.x, v[r][i], res[r][NV * VW]);
          res[r][NV * VW + 1] = fma((T)w.y, v[r][i], res[r][NV * VW + 1]);
        }
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const T* row = M + i * kRowStride;
      T acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = T(0);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const V w = reinterpret_cast<const V*>(row)[q];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = vec_dot_acc(w, v[r] + q * VW, acc[r]);
      }
      if (TAIL) {
        const float2 w = *reinterpret_cast<const float2*>(row + NV * VW);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          acc[r] = fma((T)w.x, v[r][NV * VW], acc[r]);
          acc[r] = fma((T)w.y, v[r][NV * VW + 1], acc[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) res[r][i] = acc[r];
    }
  }
}

// The transform of a pass: in the FP32 interior-patch kernel (EO_ALL) from
// the matrices passed by value (constant bank), with the warp-uniform choice
// of matrix (continuous or discontinuous direction of the warp's component)
// as a branch so that every read has a compile-time offset; else from the
// shared tables.  FP32 smoothing at k = 3 measured 19 % faster that way (the
// kernel is bound by the shared-memory pipe); the FP64 kernel, bound by the
// FP64 pipe, measured 5 % slower and keeps the shared tables.
template <int K, typename T, bool FWD, bool VELM, int R, bool EO_ALL>
__device__ __forceinline__ void pass_transform(const T* __restrict__ M, const InteriorMats<K, T>* im, bool eo,
                                               bool along_c, const T (&v)[R][PatchCfg<K>::NPD],
                                               T (&res)[R][PatchCfg<K>::NPD]) {
  if constexpr (EO_ALL && sizeof(T) == 4) {
    if (along_c)
      line_transform<K, T, FWD, VELM, R, true, true>(VELM ? im->SC : im->EC, true, true, v, res);
    else
      line_transform<K, T, FWD, VELM, R, true, true>(VELM ? im->SD : im->FM, true, false, v, res);
  } else {
    line_transform<K, T, FWD, VELM, R, EO_ALL>(M, eo, along_c, v, res);
  }
}

// One pass: every line along direction d of the three component tensors.
// Every tensor is handled as (2k+2)^3 in its padded box: the continuous
// direction of a velocity component has 2k+1 nodes, the extra node holds zero
// (zero rows / columns of SC and EC), so all lines have the same length and
// compile-time loop bounds.  Thread u of component c (warps c W .. c W + W-1)
// owns lines u, u + TPC, ... of that component.  in_shared: all components
// read the same (pressure) box.  Epilogues scale by
// inv_nu / (lam_0 + lam_1 + lam_2) of the output node (the last pass of a
// chain toward eigen-coefficients).  MODE BTBF is the last pass toward the
// eigen-coefficients, the scaling and the first pass back, fused in registers.
template <int K, typename T, int MODE, int EPI, bool EO_ALL>
__device__ __forceinline__ void patch_pass(const T* __restrict__ in, T* __restrict__ out, int d, bool in_shared,
                                           const T* __restrict__ Ft, T* __restrict__ out2,
                                           const PatchTables<T>& tb, const PatchGeo& g,
                                           const InteriorMats<K, T>* im) {
  using C = PatchCfg<K>;
  constexpr int N = C::NPD, LPC = C::LPC, TPC = PatchThreads<K, T>::TPC, R = PatchThreads<K, T>::R;
  constexpr bool VELM = (MODE == VEL_FWD || MODE == VEL_BWD);
  constexpr bool FWD = (MODE == VEL_FWD || MODE == BT || MODE == BTBF);
  const int c = threadIdx.x / TPC, u = threadIdx.x - c * TPC;
  const int e1 = (d == 0) ? 1 : 0, e2 = (d == 2) ? 1 : 2;
  const int sd = box_stride(d, C::BX, N);
  const bool along_c = (d == c);
  const int td = g.t(d);
  const T* M = VELM ? (along_c ? tb.SC : tb.SD[td]) : (along_c ? tb.EC : tb.FM[td]);
  const bool eo = along_c ? (tb.eo_c != 0) : (tb.eo_d[td] != 0);
  const T* src = in + (in_shared ? 0 : c * C::BOX);
  int i1[R], i2[R], base[R];
  bool ok[R];
  T v[R][N], res[R][N];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int l = u + r * TPC;
    ok[r] = l < LPC;
    const int ll = ok[r] ? l : 0;
    i1[r] = ll % N;
    i2[r] = ll / N;
    base[r] = i1[r] * box_stride(e1, C::BX, N) + i2[r] * box_stride(e2, C::BX, N);
#pragma unroll
    for (int i = 0; i < N; ++i) v[r][i] = src[base[r] + i * sd];
  }
  pass_transform<K, T, FWD, VELM, R, EO_ALL>(M, im, eo, along_c, v, res);
  // eigenvalues of the two fixed directions, then of the pass direction
  T lam_fixed[R];
  const T* lam_d = along_c ? tb.LC : tb.LD[td];
  if (EPI != EPI_NONE || MODE == BTBF) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      lam_fixed[r] = ((e1 == c) ? tb.LC[i1[r]] : tb.LD[g.t(e1)][i1[r]]) +
                     ((e2 == c) ? tb.LC[i2[r]] : tb.LD[g.t(e2)][i2[r]]);
  }
  if (MODE == BTBF) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const T ld = lam_d[j];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r][j] = scale_div(tb.inv_nu, lam_fixed[r] + ld) * res[r][j];
    }
    pass_transform<K, T, false, false, R, EO_ALL>(M, im, eo, along_c, v, res);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (!ok[r]) continue;
    T* dst = out + c * C::BOX + base[r];
    if (EPI == EPI_NONE) {
#pragma unroll
      for (int j = 0; j < N; ++j) dst[j * sd] = res[r][j];
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int o = j * sd;
        const T inv = scale_div(tb.inv_nu, lam_fixed[r] + lam_d[j]);
        if (EPI == EPI_SCALE) {
          dst[o] = inv * res[r][j];
        } else if (EPI == EPI_FT_AND_SCALE) {
          dst[o] = res[r][j];                                // Ft = S^T F
          out2[c * C::BOX + base[r] + o] = inv * res[r][j];  // Lam^{-1} Ft / nu
        } else {
          dst[o] = inv * (Ft[c * C::BOX + base[r] + o] - res[r][j]);
        }
      }
    }
  }
  __syncthreads();
}

// The z pass toward the eigen-coefficients, the scaling and the z pass back
// run fused in registers where the two line buffers fit (k <= 3).
template <int K>
constexpr bool kFuseZ = K <= 3;

// global index of the local velocity node (c; i0, i1, i2) or pressure node (c = 3)
template <int K>
__device__ __forceinline__ int64_t patch_node_global(int c, int i0, int i1, int i2, const int* v, int m) {
  constexpr int ND = K + 1;
  const int64_t nvel = (int64_t)(m + 1) * m * m;
  const int ii[3] = {i0, i1, i2};
  int64_t g[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) g[d] = (int64_t)(v[d] - 1) * ND + ii[d] + (d == c ? 1 : 0);
  if (c < 3) {
    const int64_t E0 = (c == 0) ? m + 1 : m, E1 = (c == 1) ? m + 1 : m;
    return c * nvel + g[0] + E0 * (g[1] + E1 * g[2]);
  }
  return 3 * nvel + g[0] + (int64_t)m * (g[1] + (int64_t)m * g[2]);
}

// patch-local DoF j (velocity components then pressure, x fastest, unpadded)
template <int K>
__device__ __forceinline__ void patch_local_decode(int j, int& c, int& i0, int& i1, int& i2) {
  using C = PatchCfg<K>;
  if (j < C::NV) {
    c = j / C::NV1;
    const int li = j - c * C::NV1;
    const int e0 = (c == 0) ? C::NPC : C::NPD, e1 = (c == 1) ? C::NPC : C::NPD;
    i0 = li % e0;
    i1 = (li / e0) % e1;
    i2 = li / (e0 * e1);
  } else {
    c = 3;
    const int q = j - C::NV;
    i0 = q % C::NPD;
    i1 = (q / C::NPD) % C::NPD;
    i2 = q / (C::NPD * C::NPD);
  }
}

template <int K>
__device__ __forceinline__ int64_t patch_global(int j, const int* v, int m) {
  int c, i0, i1, i2;
  patch_local_decode<K>(j, c, i0, i1, i2);
  return patch_node_global<K>(c, i0, i1, i2, v, m);
}

// Index in a padded patch box of the node with coordinate ac along direction
// c and a1, a2 along the two other directions d1 < d2.
template <int K>
__device__ __forceinline__ int box_index(int c, int ac, int a1, int a2) {
  using C = PatchCfg<K>;
  const int x = c == 0 ? ac : a1, y = c == 0 ? a1 : (c == 1 ? ac : a2), z = c == 2 ? ac : a2;
  return x + C::BX * (y + C::NPD * z);
}

// The patch's local residual R_j (b - A x_in) computed inside the patch
// kernel (mode 3, the fused colour step): the operator of Algorithm 1 in the
// Kronecker form of apply.cu, evaluated at the patch DoFs only, from x_in on
// a window of the patch's cells plus one cell of halo in the two
// discontinuous directions of each velocity component (the face terms of
// eq. `bilinear` couple a patch cell to its neighbour there; the continuous
// direction needs only the patch's own 2k+3 nodes, whose two end nodes are
// the patch-boundary normals, in x but not in the patch space).  This keeps
// every coupling across the patch boundary: the result equals the rows R_j
// of the global residual, which all patches of the colour read from the same
// x_in (the kernel writes to a separate x_out).
//   F (3 boxes): velocity rows of the patch (the gather's layout)
//   G (1 box):   pressure rows
//   Wn (4 boxes): window of one component, Pst (1 box): p on the patch
// Per component one thread marches along c on each line (j, l) of the
// patch cross-section, with the line's two 1D penalty rows in registers, as
// the apply kernel does.
template <int K, typename T>
__device__ __forceinline__ void patch_residual(const PatchArgs<T>& A, const int* v, const CellTables<T>& ct, T* F,
                                               T* G, T* Wn, T* Pst) {
  using C = PatchCfg<K>;
  constexpr int ND = K + 1, NC = K + 2, NPD = C::NPD, BX = C::BX, BOX = C::BOX, NT = PatchThreads<K, T>::NT;
  constexpr int WC = 2 * K + 3;  // window nodes along c: the patch's two cells
  constexpr int WD = 4 * ND;     // window nodes along d1, d2: patch cells and one halo cell per side
  constexpr int UL = 8;          // window loads a thread has in flight
  const int m = A.m, n = A.n, tid = threadIdx.x;
  const int64_t nvel = (int64_t)(m + 1) * m * m, mm = (int64_t)m * m;
  // p on the patch cells, and G = b_p
  for (int e = tid; e < NPD * NPD * NPD; e += NT) {
    const int q0 = e % NPD, q1 = (e / NPD) % NPD, q2 = e / (NPD * NPD);
    const int64_t g = 3 * nvel + ((int64_t)(v[0] - 1) * ND + q0) + (int64_t)m * ((v[1] - 1) * ND + q1) +
                      mm * ((v[2] - 1) * ND + q2);
    const int o = q0 + BX * (q1 + NPD * q2);
    Pst[o] = A.xin[g];
    G[o] = A.b[g];
  }
  for (int c = 0; c < 3; ++c) {
    const int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
    const int64_t E0 = (c == 0) ? m + 1 : m, E1 = (c == 1) ? m + 1 : m;
    const int64_t sc = (c == 0) ? 1 : (c == 1 ? E0 : E0 * E1);
    const int64_t s1 = (d1 == 0) ? 1 : E0;
    const int64_t s2 = (d2 == 1) ? E0 : E0 * E1;
    const T* u = A.xin + c * nvel;
    const T* bu = A.b + c * nvel;
    const int vc = c == 0 ? v[0] : (c == 1 ? v[1] : v[2]), vd1 = c == 0 ? v[1] : v[0], vd2 = c == 2 ? v[1] : v[2];
    const int oc = (vc - 1) * ND, o1 = (vd1 - 2) * ND, o2 = (vd2 - 2) * ND;  // window node 0, global
    // stage the window Wn[(i WD + ll) WD + jj] in global memory order (x
    // fastest); corners (halo in both d1 and d2) are never read; nodes outside
    // the domain and the constrained normal nodes (index 0 or m along c) are 0
    for (int e0 = tid; e0 < WC * WD * WD; e0 += NT * UL) {
      T val[UL];
      int dst[UL];
#pragma unroll
      for (int uu = 0; uu < UL; ++uu) {
        const int e = e0 + uu * NT;
        dst[uu] = -1;
        val[uu] = T(0);
        if (e < WC * WD * WD) {
          int i, jj, ll;
          if (c == 0) {
            i = e % WC;
            const int r = e / WC;
            jj = r % WD;
            ll = r / WD;
          } else if (c == 1) {
            jj = e % WD;
            const int r = e / WD;
            i = r % WC;
            ll = r / WC;
          } else {
            jj = e % WD;
            const int r = e / WD;
            ll = r % WD;
            i = r / WD;
          }
          const bool hj = jj < ND || jj >= 3 * ND, hl = ll < ND || ll >= 3 * ND;
          if (!(hj && hl)) {
            dst[uu] = (i * WD + ll) * WD + jj;
            const int gc = oc + i, g1 = o1 + jj, g2 = o2 + ll;
            if (gc > 0 && gc < m && g1 >= 0 && g1 < m && g2 >= 0 && g2 < m) val[uu] = u[gc * sc + g1 * s1 + g2 * s2];
          }
        }
      }
#pragma unroll
      for (int uu = 0; uu < UL; ++uu)
        if (dst[uu] >= 0) Wn[dst[uu]] = val[uu];
    }
    __syncthreads();
    // velocity rows: thread per line (j, l) of the cross-section, marching
    // along c: t = S_d2 L_d1 u + S_d1 L_d2 u and uv = S S u at the 2k+3 nodes,
    // then the cell matrices KC, MC, D^T of the patch's two cells
    for (int e = tid; e < NPD * NPD; e += NT) {
      const int j = e % NPD, l = e / NPD;
      const int jj = ND + j, ll = ND + l;
      const int cj = vd1 - 1 + j / ND, bj = j % ND, cl = vd2 - 1 + l / ND, bl = l % ND;
      const int tj = cj == 0 ? 1 : (cj == n - 1 ? 2 : 0), tl = cl == 0 ? 1 : (cl == n - 1 ? 2 : 0);
      const T sj = ct.S[bj], sl = ct.S[bl], ss = sj * sl;
      T r1s[ND], r1lo[ND], r1hi[ND], r2s[ND], r2lo[ND], r2hi[ND];
#pragma unroll
      for (int q = 0; q < ND; ++q) {
        r1s[q] = sl * ct.LS[tj][bj * ND + q];
        r1lo[q] = sl * ct.LLO[bj * ND + q];
        r1hi[q] = sl * ct.LHI[bj * ND + q];
        r2s[q] = sj * ct.LS[tl][bl * ND + q];
        r2lo[q] = sj * ct.LLO[bl * ND + q];
        r2hi[q] = sj * ct.LHI[bl * ND + q];
      }
      T tv[WC], uv[WC];
#pragma unroll
      for (int i = 0; i < WC; ++i) {
        const T* row = Wn + (i * WD + ll) * WD + jj - bj;
        const T* col = Wn + (i * WD + ll - bl) * WD + jj;
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < ND; ++q) {
          acc += r1s[q] * row[q] + r1lo[q] * row[q - ND] + r1hi[q] * row[q + ND];
          acc += r2s[q] * col[q * WD] + r2lo[q] * col[(q - ND) * WD] + r2hi[q] * col[(q + ND) * WD];
        }
        tv[i] = acc;
        uv[i] = ss * Wn[(i * WD + ll) * WD + jj];
      }
      T y[WC];
#pragma unroll
      for (int i = 0; i < WC; ++i) y[i] = T(0);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        T pv[ND];
#pragma unroll
        for (int q = 0; q < ND; ++q) pv[q] = ss * Pst[box_index<K>(c, h * ND + q, j, l)];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          T z = T(0);
#pragma unroll
          for (int bb = 0; bb < NC; ++bb) z += ct.KC[a * NC + bb] * uv[h * ND + bb] + ct.MC[a * NC + bb] * tv[h * ND + bb];
#pragma unroll
          for (int q = 0; q < ND; ++q) z += ct.D[q * NC + a] * pv[q];
          y[h * ND + a] += z;
        }
      }
      const int64_t gl = ((int64_t)(vd1 - 1) * ND + j) * s1 + ((int64_t)(vd2 - 1) * ND + l) * s2;
#pragma unroll
      for (int i = 1; i < WC - 1; ++i)
        F[c * BOX + box_index<K>(c, i - 1, j, l)] = bu[(int64_t)(oc + i) * sc + gl] - y[i];
    }
    // pressure rows: G -= D_c (M M u_c) on the patch cells
    for (int e = tid; e < NPD * NPD * NPD; e += NT) {
      const int q0 = e % NPD, q1 = (e / NPD) % NPD, q2 = e / (NPD * NPD);
      const int qc = c == 0 ? q0 : (c == 1 ? q1 : q2), qd1 = c == 0 ? q1 : q0, qd2 = c == 2 ? q1 : q2;
      const int h = qc / ND, q = qc % ND;
      const T* col = Wn + ((h * ND) * WD + ND + qd2) * WD + ND + qd1;
      T sdot = T(0);
#pragma unroll
      for (int a = 0; a < NC; ++a) sdot += ct.D[q * NC + a] * col[a * WD * WD];
      G[q0 + BX * (q1 + NPD * q2)] -= ct.S[qd1 % ND] * ct.S[qd2 % ND] * sdot;
    }
    __syncthreads();
  }
}

// Gather, local solve and scatter of patch `blk` of the colour (mode 0) or of
// coarse column `blk` (mode 1); the body of both patch kernels below.  FUSED
// (mode 3): the patch residual is computed in the kernel from x_in and b
// (patch_residual) and the scatter writes x_out = x_in + R_j^T (U, P).
template <int K, typename T, bool EO_ALL, bool FUSED = false>
__device__ __forceinline__ void patch_solve(const PatchArgs<T>& A, const int blk,
                                            const InteriorMats<K, T>* im = nullptr) {
  using C = PatchCfg<K>;
  using PT = PatchThreads<K, T>;
  constexpr int BX = C::BX, BOX = C::BOX, NPD = C::NPD;
  __shared__ PatchTables<T> tb;
  __shared__ T red[3 * PT::NW];
  T* red_a = red;          // single sums
  T* red_b = red + PT::NW;  // the second single sum of the setup, the pair sums of the CG
  extern __shared__ __align__(16) unsigned char patch_smem[];
  T* Ft = reinterpret_cast<T*>(patch_smem);  // 3 boxes: S^T F, kept to the end
  T* Ba = Ft + 3 * BOX;                      // 3 boxes of work space
  T* Bb = Ba + 3 * BOX;                      // 3 boxes of work space
  T* Dd = Bb + 3 * BOX;                      // CG search direction (pressure box)
  T* R = Dd + BOX;                           // CG residual
  T* Pp = R + BOX;                           // pressure solution (holds G until it is set to 0)
  T* SD = Pp + BOX;                          // S applied to the search direction

  const int tid = threadIdx.x;
  constexpr int NL = C::NV + C::NP;  // patch-local DoFs
  constexpr int UG = 8;              // global loads a thread has in flight in gather and scatter
  {
    // tables: 16-byte copies, all issued before the first store
    constexpr int NQ = (int)(sizeof(PatchTables<T>) / 16), UQ = (NQ + PT::NT - 1) / PT::NT;
    const int4* src = reinterpret_cast<const int4*>(A.tab);
    int4 q[UQ];
#pragma unroll
    for (int u = 0; u < UQ; ++u)
      if (tid + u * PT::NT < NQ) q[u] = src[tid + u * PT::NT];
#pragma unroll
    for (int u = 0; u < UQ; ++u)
      if (tid + u * PT::NT < NQ) reinterpret_cast<int4*>(&tb)[tid + u * PT::NT] = q[u];
  }

  int v[3];
  if (A.mode == 0 || FUSED) {
    int p = blk;
    for (int d = 0; d < 3; ++d) {
      const int ext = A.part == 1 ? A.cint[d] : A.cnt[d];
      const int t = (A.part == 1 ? A.tlo[d] : 0) + p % ext;
      p /= ext;
      const int bit = (A.colour >> d) & 1;
      v[d] = bit ? 2 * t + 1 : 2 * t + 2;
    }
  } else {
    v[0] = v[1] = v[2] = 1;
  }
  PatchGeo g;
  for (int d = 0; d < 3; ++d) g.type[d] = A.mode == 2 ? A.btype[d] : (v[d] == 1 ? 1 : 0) | (v[d] == A.n - 1 ? 2 : 0);
  // the boundary launch skips the interior patches (another launch took them)
  if ((A.mode == 0 || FUSED) && A.part == 2 && g.type[0] == 0 && g.type[1] == 0 && g.type[2] == 0) return;

  // SDc = S d per component for the pressure box Dd: (B S) Lam^{-1} (B S)^T d,
  // passes x, y, z then z, y, x; returns the three component boxes to sum
  auto schur_apply = [&]() -> T* {
    patch_pass<K, T, BT, EPI_NONE, EO_ALL>(Dd, Ba, 0, true, nullptr, nullptr, tb, g, im);
    patch_pass<K, T, BT, EPI_NONE, EO_ALL>(Ba, Bb, 1, false, nullptr, nullptr, tb, g, im);
    if constexpr (kFuseZ<K>) {
      patch_pass<K, T, BTBF, EPI_NONE, EO_ALL>(Bb, Ba, 2, false, nullptr, nullptr, tb, g, im);
      patch_pass<K, T, BF, EPI_NONE, EO_ALL>(Ba, Bb, 1, false, nullptr, nullptr, tb, g, im);
      patch_pass<K, T, BF, EPI_NONE, EO_ALL>(Bb, Ba, 0, false, nullptr, nullptr, tb, g, im);
      return Ba;
    } else {
      patch_pass<K, T, BT, EPI_SCALE, EO_ALL>(Bb, Ba, 2, false, nullptr, nullptr, tb, g, im);
      patch_pass<K, T, BF, EPI_NONE, EO_ALL>(Ba, Bb, 2, false, nullptr, nullptr, tb, g, im);
      patch_pass<K, T, BF, EPI_NONE, EO_ALL>(Bb, Ba, 1, false, nullptr, nullptr, tb, g, im);
      patch_pass<K, T, BF, EPI_NONE, EO_ALL>(Ba, Bb, 0, false, nullptr, nullptr, tb, g, im);
      return Bb;
    }
  };

  if (A.mode == 2) {  // column blk of the Schur complement of a patch of types btype
    for (int q = tid; q < C::NP; q += PT::NT) Dd[(q % NPD) + BX * (q / NPD)] = (q == blk) ? T(1) : T(0);
    __syncthreads();
    const T* SDc = schur_apply();
    for (int q = tid; q < C::NP; q += PT::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      A.cols[(int64_t)blk * C::NP + q] = (double)(SDc[o] + SDc[BOX + o] + SDc[2 * BOX + o]);
    }
    return;
  }

  // ---- gather F (velocity boxes in Ba) and G (pressure box in Pp = Ba + 8 BOX);
  // the padded plane (node 2k+1 of the continuous direction) of each velocity
  // box is set to zero.  UG loads per thread are issued before their stores.
  if constexpr (FUSED) {
    // the cell matrices live in the Ft boxes (unused until the residual is
    // done) where they fit, else in static shared memory (k = 1)
    constexpr int NCT = (int)(sizeof(CellTables<T>) / sizeof(T));
    constexpr bool IN_FT = NCT <= 3 * BOX;
    __shared__ T ct_static[IN_FT ? 1 : NCT];
    T* ctp = IN_FT ? Ft : ct_static;
    for (int i = tid; i < NCT; i += PT::NT) ctp[i] = reinterpret_cast<const T*>(A.ctab)[i];
    __syncthreads();
    patch_residual<K, T>(A, v, *reinterpret_cast<const CellTables<T>*>(ctp), Ba, Pp, Bb, R);
  }
  for (int j0 = tid; !FUSED && j0 < NL; j0 += PT::NT * UG) {
    T val[UG];
    int dst[UG];
#pragma unroll
    for (int u = 0; u < UG; ++u) {
      const int j = j0 + u * PT::NT;
      dst[u] = -1;
      val[u] = T(0);
      if (j < NL) {
        int c, i0, i1, i2;
        patch_local_decode<K>(j, c, i0, i1, i2);
        dst[u] = (c < 3 ? c * BOX : 8 * BOX) + i0 + BX * (i1 + NPD * i2);
        if (A.mode == 0)
          val[u] = A.r[patch_node_global<K>(c, i0, i1, i2, v, A.m)];
        else
          val[u] = (j == blk) ? T(1) : T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < UG; ++u)
      if (dst[u] >= 0) Ba[dst[u]] = val[u];
  }
  for (int i = tid; i < 3 * NPD * NPD; i += PT::NT) {
    const int c = i / (NPD * NPD), a = i % NPD, b = (i / NPD) % NPD;
    const int ii[3] = {c == 0 ? C::NPC : a, c == 1 ? C::NPC : (c == 0 ? a : b), c == 2 ? C::NPC : b};
    Ba[c * BOX + ii[0] + BX * (ii[1] + NPD * ii[2])] = T(0);
  }
  __syncthreads();

  // ---- Ft = S^T F; Bb = Lam^{-1} Ft / nu
  patch_pass<K, T, VEL_FWD, EPI_NONE, EO_ALL>(Ba, Bb, 0, false, nullptr, nullptr, tb, g, im);
  patch_pass<K, T, VEL_FWD, EPI_NONE, EO_ALL>(Bb, Ba, 1, false, nullptr, nullptr, tb, g, im);
  patch_pass<K, T, VEL_FWD, EPI_FT_AND_SCALE, EO_ALL>(Ba, Ft, 2, false, nullptr, Bb, tb, g, im);
  // ---- R = sum_c (B_c S_c) Bb_c - G (not needed when P comes from the GEMM)
  T s1 = T(0), s2 = T(0), mean = T(0), rr = T(0), rr0 = T(0);
  if (A.gemm_phase != 2) {
    patch_pass<K, T, BF, EPI_NONE, EO_ALL>(Bb, Ba, 0, false, nullptr, nullptr, tb, g, im);
    patch_pass<K, T, BF, EPI_NONE, EO_ALL>(Ba, Bb, 1, false, nullptr, nullptr, tb, g, im);
    patch_pass<K, T, BF, EPI_NONE, EO_ALL>(Bb, Ba, 2, false, nullptr, nullptr, tb, g, im);
    for (int q = tid; q < C::NP; q += PT::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      const T r = (Ba[o] + Ba[BOX + o] + Ba[2 * BOX + o]) - Pp[o];
      R[o] = r;
      s1 += r;
    }
    mean = block_sum<T, PT::NW>(s1, red_a) / T(C::NP);
    s2 = T(0);
    for (int q = tid; q < C::NP; q += PT::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      const T r = R[o] - mean;
      R[o] = r;
      Dd[o] = r;
      Pp[o] = T(0);
      s2 += r * r;
    }
    rr = block_sum<T, PT::NW>(s2, red_b);
    rr0 = rr;
  }
  if (A.gemm_phase == 1) {  // R leaves for the colour's GEMM
    for (int q = tid; q < C::NP; q += PT::NT) A.rout[(int64_t)blk * C::NP + q] = R[(q % NPD) + BX * (q / NPD)];
    return;
  }
  if (A.gemm_phase == 2) {  // P = M R from the colour's GEMM
    for (int q = tid; q < C::NP; q += PT::NT) Pp[(q % NPD) + BX * (q / NPD)] = A.pin[(int64_t)blk * C::NP + q];
    __syncthreads();
  }

  // ---- the local Schur system S P = R on mean-free pressures: Direct (a
  // precomputed (S + a 1 1^T)^{-1} of this patch type, which maps a mean-free
  // R to the mean-free solution) or conjugate gradients
  const T* Mdir = ((A.mode == 0 || FUSED) && A.dir && A.gemm_phase == 0)
                      ? A.dir[g.type[0] + 4 * g.type[1] + 16 * g.type[2]]
                      : nullptr;
  if (Mdir) {
    // 16-byte loads where the vectors of a column keep every thread busy
    // (19 % faster at k = 3 in FP32), else one output per load: thread t
    // owns outputs VW s .. VW s + VW-1 for s = t, t + NT, ...
    using V = typename Vec16<T>::type;
    constexpr int VW = (C::NP / Vec16<T>::width >= PT::NT) ? Vec16<T>::width : 1;
    constexpr int NPV = C::NP / VW;                  // (2k+2)^3 is a multiple of 8
    constexpr int NO = (NPV + PT::NT - 1) / PT::NT;    // vectors per thread
    T acc[NO][VW];
#pragma unroll
    for (int u = 0; u < NO; ++u)
#pragma unroll
      for (int e = 0; e < VW; ++e) acc[u][e] = T(0);
    for (int j = 0; j < C::NP; ++j) {
      const T rj = R[(j % NPD) + BX * (j / NPD)];
      const T* colp = Mdir + (int64_t)j * C::NP;  // column j, across the threads
#pragma unroll
      for (int u = 0; u < NO; ++u) {
        if (tid + u * PT::NT >= NPV) continue;
        if constexpr (VW == Vec16<T>::width)
          vec_fma(acc[u], reinterpret_cast<const V*>(colp)[tid + u * PT::NT], rj);
        else
          acc[u][0] = fma(colp[tid + u * PT::NT], rj, acc[u][0]);
      }
    }
#pragma unroll
    for (int u = 0; u < NO; ++u)
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int q = (tid + u * PT::NT) * VW + e;
        if (tid + u * PT::NT < NPV) Pp[(q % NPD) + BX * (q / NPD)] = acc[u][e];
      }
    __syncthreads();
  }
  for (int it = 0; !Mdir && A.gemm_phase == 0 && it < A.cg_iters; ++it) {
    if (A.cg_tol_mode && rr <= A.cg_tol * A.cg_tol * rr0) break;
    if (!(rr > T(0))) break;
    T* SDc = schur_apply();
    T part = T(0);
    for (int q = tid; q < C::NP; q += PT::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      const T s = SDc[o] + SDc[BOX + o] + SDc[2 * BOX + o];
      SD[o] = s;
      part += Dd[o] * s;
    }
    const T dSd = block_sum<T, PT::NW>(part, red_a);
    if (!(dSd > T(0))) break;
    const T alpha = rr / dSd;
    s1 = T(0);
    s2 = T(0);
    for (int q = tid; q < C::NP; q += PT::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      Pp[o] += alpha * Dd[o];
      const T r = R[o] - alpha * SD[o];
      R[o] = r;
      s1 += r;
      s2 += r * r;
    }
    block_sum2<T, PT::NW>(s1, s2, red_b);
    mean = s1 / T(C::NP);
    T rr_new = s2 - s1 * mean;  // sum (r - mean)^2
    if (rr_new < T(0)) rr_new = T(0);
    const T beta = rr_new / rr;
    for (int q = tid; q < C::NP; q += PT::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      const T r = R[o] - mean;
      R[o] = r;
      Dd[o] = r + beta * Dd[o];
    }
    rr = rr_new;
    __syncthreads();
  }

  // ---- U_c = S_c Lam_c^{-1} (Ft_c - (B_c S_c)^T P) / nu
  patch_pass<K, T, BT, EPI_NONE, EO_ALL>(Pp, Ba, 0, true, nullptr, nullptr, tb, g, im);
  patch_pass<K, T, BT, EPI_NONE, EO_ALL>(Ba, Bb, 1, false, nullptr, nullptr, tb, g, im);
  patch_pass<K, T, BT, EPI_SUB_SCALE, EO_ALL>(Bb, Ba, 2, false, Ft, nullptr, tb, g, im);
  patch_pass<K, T, VEL_BWD, EPI_NONE, EO_ALL>(Ba, Bb, 0, false, nullptr, nullptr, tb, g, im);
  patch_pass<K, T, VEL_BWD, EPI_NONE, EO_ALL>(Bb, Ba, 1, false, nullptr, nullptr, tb, g, im);
  patch_pass<K, T, VEL_BWD, EPI_NONE, EO_ALL>(Ba, Bb, 2, false, nullptr, nullptr, tb, g, im);

  // ---- scatter: x += (U, P); UG loads of x per thread in flight
  for (int j0 = tid; j0 < NL; j0 += PT::NT * UG) {
    T val[UG], old[UG];
    int64_t gi[UG];
#pragma unroll
    for (int u = 0; u < UG; ++u) {
      const int j = j0 + u * PT::NT;
      gi[u] = -1;
      val[u] = T(0);
      if (j < NL) {
        int c, i0, i1, i2;
        patch_local_decode<K>(j, c, i0, i1, i2);
        const int o = i0 + BX * (i1 + NPD * i2);
        val[u] = (c < 3) ? Bb[c * BOX + o] : Pp[o];
        gi[u] = (A.mode == 0 || FUSED) ? patch_node_global<K>(c, i0, i1, i2, v, A.m) : (int64_t)blk * NL + j;
      }
    }
    if (A.mode == 0 || FUSED) {
#pragma unroll
      for (int u = 0; u < UG; ++u)
        if (gi[u] >= 0) old[u] = FUSED ? A.xin[gi[u]] : A.x[gi[u]];
#pragma unroll
      for (int u = 0; u < UG; ++u)
        if (gi[u] >= 0) A.x[gi[u]] = old[u] + val[u];
    } else {
#pragma unroll
      for (int u = 0; u < UG; ++u)
        if (gi[u] >= 0) A.cols[gi[u]] = (double)val[u];
    }
  }
}

template <int K, typename T, bool FUSED = false>
__global__ void __launch_bounds__(PatchThreads<K, T>::NT, (PatchOcc<K, T>::value)) patch_kernel(PatchArgs<T> A) {
  patch_solve<K, T, false, FUSED>(A, blockIdx.x);
}

// Interior patches only: every 1D eigenbasis is symmetric, so the dense
// transform code is not compiled in and the kernel's loop stays small in the
// instruction cache; the transform matrices come with the launch (IM).
template <int K, typename T, bool FUSED = false>
__global__ void __launch_bounds__(PatchThreads<K, T>::NT, (PatchOcc<K, T>::value))
    patch_kernel_interior(PatchArgs<T> A, InteriorMats<K, T> IM) {
  patch_solve<K, T, true, FUSED>(A, blockIdx.x, &IM);
}

// One colour of several problems of the same degree in one launch: CTA b
// solves patch b - first[j] of problem j (first[] ascending); the per-problem
// fields replace those of the common arguments.
template <int K, typename T>
__global__ void __launch_bounds__(PatchThreads<K, T>::NT, (PatchOcc<K, T>::value))
    patch_kernel_multi(PatchArgs<T> A, PatchJobs<T> J) {
  int lo = 0, hi = J.count - 1;  // last job with first[job] <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (J.first[mid] <= (int)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  PatchArgs<T> a = A;
  a.r = J.r[lo];
  a.x = J.x[lo];
  a.tab = J.tab[lo];
  a.n = J.n[lo];
  a.m = J.m[lo];
  for (int d = 0; d < 3; ++d) a.cnt[d] = J.cnt[lo][d];
  patch_solve<K, T, false>(a, (int)blockIdx.x - J.first[lo]);
}

template <int K>
size_t patch_smem_bytes(size_t esize) {
  using C = PatchCfg<K>;
  return esize * (9 * C::BOX + 4 * C::BOX);
}

// Launch the patch kernel (part 1: the interior-patch kernel) over nblocks
// CTAs, or the multi-problem kernel over the jobs of J.  Defined in
// patch_launch.cuh and instantiated once per degree by patch_k<K>.cu.
template <int K, typename T>
cudaError_t launch_patch_k(PatchArgs<T> a, int nblocks, cudaStream_t s);
template <int K, typename T>
cudaError_t launch_patch_multi_k(const PatchArgs<T>& a, const PatchJobs<T>& J, int nblocks, cudaStream_t s);

}  // namespace stk
