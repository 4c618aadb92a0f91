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
// Fast diagonalization (eq. `inverse2d`, eq. `fast_inverse` in 3D): per
// velocity component c,  A_c^{-1} = (1/nu) S_c Lam_c^{-1} S_c^T  with
// S_c = S_x (x) S_y (x) S_z (continuous-direction eigenvectors along c,
// discontinuous ones along the other two).  Because B_c = D (x) W (x) W
// (eq. `b`) is a Kronecker product too, so is  B_c S_c = (D S) (x) (W S) (x) (W S),
// and the Schur operator is  S = (1/nu) sum_c (B_c S_c) Lam_c^{-1} (B_c S_c)^T.
// One CG step is therefore six passes of batched 1D line transforms (three
// from pressure space to the scaled eigen-coefficients, three back) over all
// three components, instead of B^T, A^{-1} (six passes) and B separately.
//   start:  Ft_c = S_c^T F_c,  R = sum_c (B_c S_c) Lam_c^{-1} Ft_c / nu - G
//   end:    U_c = S_c Lam_c^{-1} (Ft_c - (B_c S_c)^T P) / nu
// Every patch tensor lives in shared memory in a (2k+3) x (2k+2) x (2k+2)
// box (odd x stride: strided line accesses hit distinct banks).
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
  static constexpr int NV1 = NPC * NPD * NPD;  // one velocity component (unpadded)
  static constexpr int NV = 3 * NV1;
  static constexpr int NP = NPD * NPD * NPD;
  static constexpr int BX = NPD + 1;           // padded x extent of every patch tensor
  static constexpr int BOX = BX * NPD * NPD;   // one padded tensor
  static constexpr int NT = ((3 * NPD * NPD + 31) / 32) * 32;  // one thread per line of a pass
  static constexpr int NW = NT / 32;
};

// Resident CTAs per SM the register budget must allow: as many as the shared
// memory of one patch (13 padded tensors + tables) permits.
template <int K, typename T>
struct PatchOcc {
  static constexpr int value = sizeof(T) == 4 ? ((K == 1) ? 16 : (K == 2) ? 8 : (K == 3) ? 5 : (K == 4) ? 3 : 2)
                                              : ((K == 1) ? 8 : (K == 2) ? 4 : (K == 3) ? 3 : 1);
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

// two sums at once
template <typename T, int NW>
__device__ __forceinline__ void block_sum2(T& a, T& b, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
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
__device__ __forceinline__ float vec_dot(const float4& w, const float* v) {
  return w.x * v[0] + w.y * v[1] + w.z * v[2] + w.w * v[3];
}
__device__ __forceinline__ double vec_dot(const double2& w, const double* v) { return w.x * v[0] + w.y * v[1]; }

// pass kinds: velocity eigen-transform (S^T: VEL_FWD, S: VEL_BWD), pressure to
// eigen-coefficients ((B S)^T: BT), eigen-coefficients to pressure (B S: BF)
enum { VEL_FWD = 0, VEL_BWD = 1, BT = 2, BF = 3 };
// epilogues of a pass
enum { EPI_NONE = 0, EPI_SCALE = 1, EPI_FT_AND_SCALE = 2, EPI_SUB_SCALE = 3 };

struct PatchGeo {
  int type[3];
  __device__ __forceinline__ int t(int d) const { return d == 0 ? type[0] : (d == 1 ? type[1] : type[2]); }
};

// Extent of component c along direction e during a pass of kind MODE, given
// the directions already transformed in the current chain (bit mask).
template <int K, int MODE>
__device__ __forceinline__ int ext_of(int c, int e, int done) {
  using C = PatchCfg<K>;
  const int vel = (e == c) ? C::NPC : C::NPD;
  if (MODE == VEL_FWD || MODE == VEL_BWD) return vel;
  const bool tr = (done >> e) & 1;
  if (MODE == BT) return tr ? vel : C::NPD;
  return tr ? C::NPD : vel;  // BF
}

// One pass: every line along direction d of the three component tensors.
// in_shared: all components read the same (pressure) box.  Epilogues scale by
// inv_nu / (lam_0 + lam_1 + lam_2) of the output node (the last pass of a
// chain toward eigen-coefficients).
template <int K, typename T, int MODE>
__device__ void patch_pass_fma(const T* __restrict__ in, T* __restrict__ out, int d, int done, bool in_shared,
                               int epi, const T* __restrict__ Ft, T* __restrict__ out2, const PatchTables<T>& tb,
                               const PatchGeo& g) {
  using C = PatchCfg<K>;
  constexpr int NMAX = C::NPD;
  const int e1 = (d == 0) ? 1 : 0, e2 = (d == 2) ? 1 : 2;
  int lines[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) lines[c] = ext_of<K, MODE>(c, e1, done) * ext_of<K, MODE>(c, e2, done);
  const int total = lines[0] + lines[1] + lines[2];
  const int sd = box_stride(d, C::BX, C::NPD);
  for (int L = threadIdx.x; L < total; L += C::NT) {
    int c = 0, l = L;
    if (l >= lines[0]) {
      l -= lines[0];
      c = 1;
      if (l >= lines[1]) {
        l -= lines[1];
        c = 2;
      }
    }
    // the extent along e1 is NPC or NPD: divide by compile-time constants
    const int x1 = ext_of<K, MODE>(c, e1, done);
    int i1, i2;
    if (x1 == C::NPC) {
      i1 = l % C::NPC;
      i2 = l / C::NPC;
    } else {
      i1 = l % C::NPD;
      i2 = l / C::NPD;
    }
    const int base = i1 * box_stride(e1, C::BX, C::NPD) + i2 * box_stride(e2, C::BX, C::NPD);
    const T* src = in + (in_shared ? 0 : c * C::BOX) + base;
    T* dst = out + c * C::BOX + base;
    const bool along_c = (d == c);
    int n_in, n_out;
    const T* M;  // rows of kRowStride entries, zero padded
    if (MODE == VEL_FWD || MODE == VEL_BWD) {
      n_in = n_out = along_c ? C::NPC : C::NPD;
      M = along_c ? tb.SC : tb.SD[g.t(d)];
    } else if (MODE == BT) {
      n_in = C::NPD;
      n_out = along_c ? C::NPC : C::NPD;
      M = along_c ? tb.EC : tb.FM[g.t(d)];
    } else {
      n_in = along_c ? C::NPC : C::NPD;
      n_out = C::NPD;
      M = along_c ? tb.EC : tb.FM[g.t(d)];
    }
    using V = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::width;
    constexpr int NP4 = ((NMAX + VW - 1) / VW) * VW;  // padded row length read per row
    T v[NP4];
#pragma unroll
    for (int i = 0; i < NP4; ++i) v[i] = (i < n_in) ? src[i * sd] : T(0);
    // eigenvalues of the two fixed directions (scaling epilogues only)
    T lam_fixed = T(0);
    if (epi != EPI_NONE) {
      const int ii[2] = {i1, i2};
      const int ee[2] = {e1, e2};
#pragma unroll
      for (int q = 0; q < 2; ++q) lam_fixed += (ee[q] == c) ? tb.LC[ii[q]] : tb.LD[g.t(ee[q])][ii[q]];
    }
    T res[NP4];
    if (MODE == VEL_FWD || MODE == BT) {
      // out_j = sum_i M[i][j] v_i: one vector load feeds VW outputs
#pragma unroll
      for (int j = 0; j < NP4; ++j) res[j] = T(0);
#pragma unroll
      for (int i = 0; i < NMAX; ++i) {
        if (i >= n_in) break;
        const V* row = reinterpret_cast<const V*>(M + i * kRowStride);
#pragma unroll
        for (int q = 0; q < NP4 / VW; ++q) {
          const V w = row[q];
          vec_fma(res + q * VW, w, v[i]);
        }
      }
    } else {
      // out_i = sum_j M[i][j] v_j
#pragma unroll
      for (int i = 0; i < NMAX; ++i) {
        res[i] = T(0);
        if (i >= n_out) continue;
        const V* row = reinterpret_cast<const V*>(M + i * kRowStride);
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < NP4 / VW; ++q) acc += vec_dot(row[q], v + q * VW);
        res[i] = acc;
      }
    }
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      if (j >= n_out) break;
      const T acc = res[j];
      const int o = j * sd;
      if (epi == EPI_NONE) {
        dst[o] = acc;
      } else {
        const T lam = lam_fixed + (along_c ? tb.LC[j] : tb.LD[g.t(d)][j]);
        const T inv = tb.inv_nu / lam;
        if (epi == EPI_SCALE) {
          dst[o] = inv * acc;
        } else if (epi == EPI_FT_AND_SCALE) {
          dst[o] = acc;                                   // Ft = S^T F
          out2[c * C::BOX + base + o] = inv * acc;        // Lam^{-1} Ft / nu
        } else {
          dst[o] = inv * (Ft[c * C::BOX + base + o] - acc);
        }
      }
    }
  }
  __syncthreads();
}

template <int K, typename T, int MODE>
__device__ __forceinline__ void patch_pass(const T* in, T* out, int d, int done, bool in_shared, int epi, const T* Ft,
                                           T* out2, const PatchTables<T>& tb, const PatchGeo& g) {
  patch_pass_fma<K, T, MODE>(in, out, d, done, in_shared, epi, Ft, out2, tb, g);
}

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

template <int K, typename T>
__global__ void __launch_bounds__(PatchCfg<K>::NT, (PatchOcc<K, T>::value)) patch_kernel(PatchArgs<T> A) {
  using C = PatchCfg<K>;
  constexpr int BX = C::BX, BOX = C::BOX, NPD = C::NPD;
  __shared__ PatchTables<T> tb;
  __shared__ T red[2 * C::NW];
  extern __shared__ __align__(16) unsigned char patch_smem[];
  T* Ft = reinterpret_cast<T*>(patch_smem);  // 3 boxes: S^T F, kept to the end
  T* Ba = Ft + 3 * BOX;                      // 3 boxes of work space
  T* Bb = Ba + 3 * BOX;                      // 3 boxes of work space
  T* Dd = Bb + 3 * BOX;                      // CG search direction (pressure box)
  T* R = Dd + BOX;                           // CG residual
  T* Pp = R + BOX;                           // pressure solution (holds G until it is set to 0)
  T* SD = Pp + BOX;                          // S applied to the search direction

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
  PatchGeo g;
  for (int d = 0; d < 3; ++d) g.type[d] = (v[d] == 1 ? 1 : 0) | (v[d] == A.n - 1 ? 2 : 0);

  // ---- gather F (velocity boxes in Ba) and G (pressure box in Pp)
  for (int j = tid; j < C::NV + C::NP; j += C::NT) {
    int c, i0, i1, i2;
    patch_local_decode<K>(j, c, i0, i1, i2);
    T val;
    if (A.mode == 0)
      val = A.r[patch_node_global<K>(c, i0, i1, i2, v, A.m)];
    else
      val = (j == (int)blockIdx.x) ? T(1) : T(0);
    const int o = i0 + BX * (i1 + NPD * i2);
    if (c < 3)
      Ba[c * BOX + o] = val;
    else
      Pp[o] = val;
  }
  __syncthreads();

  // ---- Ft = S^T F; Bb = Lam^{-1} Ft / nu
  patch_pass<K, T, VEL_FWD>(Ba, Bb, 0, 0, false, EPI_NONE, nullptr, nullptr, tb, g);
  patch_pass<K, T, VEL_FWD>(Bb, Ba, 1, 0, false, EPI_NONE, nullptr, nullptr, tb, g);
  patch_pass<K, T, VEL_FWD>(Ba, Ft, 2, 0, false, EPI_FT_AND_SCALE, nullptr, Bb, tb, g);
  // ---- R = sum_c (B_c S_c) Bb_c - G
  patch_pass<K, T, BF>(Bb, Ba, 0, 0, false, EPI_NONE, nullptr, nullptr, tb, g);
  patch_pass<K, T, BF>(Ba, Bb, 1, 1, false, EPI_NONE, nullptr, nullptr, tb, g);
  patch_pass<K, T, BF>(Bb, Ba, 2, 3, false, EPI_NONE, nullptr, nullptr, tb, g);
  T s1 = T(0), s2 = T(0);
  for (int q = tid; q < C::NP; q += C::NT) {
    const int o = (q % NPD) + BX * (q / NPD);
    const T r = (Ba[o] + Ba[BOX + o] + Ba[2 * BOX + o]) - Pp[o];
    R[o] = r;
    s1 += r;
  }
  T mean = block_sum<T, C::NW>(s1, red) / T(C::NP);
  s2 = T(0);
  for (int q = tid; q < C::NP; q += C::NT) {
    const int o = (q % NPD) + BX * (q / NPD);
    const T r = R[o] - mean;
    R[o] = r;
    Dd[o] = r;
    Pp[o] = T(0);
    s2 += r * r;
  }
  T rr = block_sum<T, C::NW>(s2, red);
  const T rr0 = rr;

  // ---- conjugate gradients on the mean-free pressures
  for (int it = 0; it < A.cg_iters; ++it) {
    if (A.cg_tol_mode && rr <= A.cg_tol * A.cg_tol * rr0) break;
    if (!(rr > T(0))) break;
    patch_pass<K, T, BT>(Dd, Ba, 0, 0, true, EPI_NONE, nullptr, nullptr, tb, g);
    patch_pass<K, T, BT>(Ba, Bb, 1, 1, false, EPI_NONE, nullptr, nullptr, tb, g);
    patch_pass<K, T, BT>(Bb, Ba, 2, 3, false, EPI_SCALE, nullptr, nullptr, tb, g);
    patch_pass<K, T, BF>(Ba, Bb, 0, 0, false, EPI_NONE, nullptr, nullptr, tb, g);
    patch_pass<K, T, BF>(Bb, Ba, 1, 1, false, EPI_NONE, nullptr, nullptr, tb, g);
    patch_pass<K, T, BF>(Ba, Bb, 2, 3, false, EPI_NONE, nullptr, nullptr, tb, g);
    T part = T(0);
    for (int q = tid; q < C::NP; q += C::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      const T s = Bb[o] + Bb[BOX + o] + Bb[2 * BOX + o];
      SD[o] = s;
      part += Dd[o] * s;
    }
    const T dSd = block_sum<T, C::NW>(part, red);
    if (!(dSd > T(0))) break;
    const T alpha = rr / dSd;
    s1 = T(0);
    s2 = T(0);
    for (int q = tid; q < C::NP; q += C::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      Pp[o] += alpha * Dd[o];
      const T r = R[o] - alpha * SD[o];
      R[o] = r;
      s1 += r;
      s2 += r * r;
    }
    block_sum2<T, C::NW>(s1, s2, red);
    mean = s1 / T(C::NP);
    T rr_new = s2 - s1 * mean;  // sum (r - mean)^2
    if (rr_new < T(0)) rr_new = T(0);
    const T beta = rr_new / rr;
    for (int q = tid; q < C::NP; q += C::NT) {
      const int o = (q % NPD) + BX * (q / NPD);
      const T r = R[o] - mean;
      R[o] = r;
      Dd[o] = r + beta * Dd[o];
    }
    rr = rr_new;
    __syncthreads();
  }

  // ---- U_c = S_c Lam_c^{-1} (Ft_c - (B_c S_c)^T P) / nu
  patch_pass<K, T, BT>(Pp, Ba, 0, 0, true, EPI_NONE, nullptr, nullptr, tb, g);
  patch_pass<K, T, BT>(Ba, Bb, 1, 1, false, EPI_NONE, nullptr, nullptr, tb, g);
  patch_pass<K, T, BT>(Bb, Ba, 2, 3, false, EPI_SUB_SCALE, Ft, nullptr, tb, g);
  patch_pass<K, T, VEL_BWD>(Ba, Bb, 0, 0, false, EPI_NONE, nullptr, nullptr, tb, g);
  patch_pass<K, T, VEL_BWD>(Bb, Ba, 1, 0, false, EPI_NONE, nullptr, nullptr, tb, g);
  patch_pass<K, T, VEL_BWD>(Ba, Bb, 2, 0, false, EPI_NONE, nullptr, nullptr, tb, g);

  // ---- scatter
  for (int j = tid; j < C::NV + C::NP; j += C::NT) {
    int c, i0, i1, i2;
    patch_local_decode<K>(j, c, i0, i1, i2);
    const int o = i0 + BX * (i1 + NPD * i2);
    const T val = (c < 3) ? Bb[c * BOX + o] : Pp[o];
    if (A.mode == 0)
      A.x[patch_node_global<K>(c, i0, i1, i2, v, A.m)] += val;
    else
      A.cols[(int64_t)blockIdx.x * (C::NV + C::NP) + j] = (double)val;
  }
}

template <int K>
size_t patch_smem_bytes(size_t esize) {
  using C = PatchCfg<K>;
  return esize * (9 * C::BOX + 4 * C::BOX);
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

cudaError_t launch_patch_colour_cg(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x,
                                   int cg_tol_mode, int cg_iters, double cg_tol) {
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
    a.cg_tol_mode = cg_tol_mode;
    a.cg_iters = cg_iters;
    a.cg_tol = cg_tol;
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
  a.cg_tol_mode = cg_tol_mode;
  a.cg_iters = cg_iters;
  a.cg_tol = (float)cg_tol;
  return dispatch_patch<float>(P->k, a, nb, P->stream);
}

cudaError_t launch_patch_colour(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x) {
  return launch_patch_colour_cg(P, level, dtype, colour, r, x, P->opt.local_cg_mode == STK_CG_TOL,
                                P->opt.local_cg_iters, P->opt.local_cg_tol);
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
