// Matrix-free Stokes operator (Algorithm 1, Sec. 2.2-2.3) on a uniform
// Cartesian mesh, in Kronecker form.
//
// With the diagonal Gauss mass M (entries S[a] = h w_a) of the discontinuous
// directions, the continuous-direction stiffness KC and mass MC, the 1D
// interior-penalty operator L (blocks LS / LLO / LHI) and the divergence
// factor D, component c of the velocity rows is
//     y_c = KC_c (M_d1 M_d2 u_c) + MC_c (M_d2 L_d1 u_c + M_d1 L_d2 u_c) + D_c^T (M_d1 M_d2 p)
// (d1 < d2 the two other directions; all viscous tables carry nu), and the
// pressure rows are  y_p = sum_c D_c (M_d1 M_d2 u_c).  This is eq. `bilinear`
// plus eq. `weak_form` integrated exactly: face terms of eq. `bilinear` only
// see tangential components, whose jumps live in the discontinuous directions.
//
// Velocity kernel: a CTA works on a tile of (d1, d2) node lines and marches
// along the continuous direction c through a run of cells (a persistent CTA
// takes an equal share of all columns' cells, possibly several runs).  Per
// cell it
// stages the k+1 new node layers of u_c (plus one cell of halo in d1 and d2)
// in shared memory, forms t = M_d2 L_d1 u + M_d1 L_d2 u per node, and then
// contracts along c in registers with the cell matrices KC, MC and D^T, in
// even-odd form: KC and MC are centro-symmetric and D antisymmetric under the
// reflection of the cell, so the contraction works on sums and differences of
// mirrored nodes with half the products (ContractTables).  The
// contribution of a cell to its upper shared node is carried to the next step,
// so no face or node is computed twice inside a run; a run re-does only
// the cell below it.  Pressure kernel: one thread per pressure node.
#include <algorithm>

#include "internal.h"

namespace stk {

template <typename T>
struct ApplyArgs {
  const T* x;
  const T* b;  // residual form: y = b - A x; NULL: y = A x
  T* y;
  T alpha;     // -1 in the residual form, 1 otherwise (pressure kernel)
  CellTables<T> tv;      // by value: constant-bank operands for compile-time indices
  ContractTables<T> ce;  // even-odd contraction along c, by value
  int n, m;
  int ntile;
  int chunk;  // cells per run of the persistent march along c
};

template <int K>
struct ApplyCfg {
  static constexpr int ND = K + 1, NC = K + 2;
  static constexpr int BJ = (K == 1) ? 8 : (K == 2) ? 5 : (K == 3) ? 4 : (K == 4) ? 3 : 2;  // cells per tile side
  static constexpr int TJ = BJ * ND;                                          // nodes per tile side
  static constexpr int H = ND;                                                // halo width (one cell)
  static constexpr int J = TJ + 2 * H;                                        // staged extent
  static constexpr int NT = TJ * TJ;                                          // threads per CTA
};

// Whether the velocity kernel marches persistently (FP64 up to k = 4; the
// k = 5 kernel spills and measured 2 % slower that way) or one run per CTA.
template <int K, typename T>
__host__ __device__ constexpr bool velocity_persistent() {
  return sizeof(T) == 8 && K <= 4;
}

// Row pitch of the staged layers: odd for the persistent FP64 kernels, so
// that the two node rows a warp reads along d1 fall in different banks
// (measured 4 % faster at k = 3, where the staged extent is 24; the FP32
// kernel measured 3 % slower with the odd pitch).
template <int K, typename T>
struct StagePitch {
  static constexpr int value = velocity_persistent<K, T>() ? (ApplyCfg<K>::J | 1) : ApplyCfg<K>::J;
};

// Stage NA node layers a0 .. a0+NA-1 of cell cc along c into U[a][ll][jj],
// one cell of halo in d1 and d2 (corners skipped: never read).  Global memory
// is walked in its own order (x fastest) so that loads coalesce.
template <int K, typename T, int NA>
__device__ __forceinline__ void stage_layers(T* __restrict__ U, const T* __restrict__ u, int a0, int c, int cc,
                                             int j0, int l0, int m, int64_t sc, int64_t s1, int64_t s2) {
  using Cfg = ApplyCfg<K>;
  constexpr int ND = Cfg::ND, TJ = Cfg::TJ, H = Cfg::H, J = Cfg::J, NT = Cfg::NT;
  constexpr int total = NA * J * J;
  for (int e = threadIdx.x; e < total; e += NT) {
    int a, jj, ll;
    if (c == 0) {
      a = e % NA;
      const int r = e / NA;
      jj = r % J;
      ll = r / J;
    } else if (c == 1) {
      jj = e % J;
      const int r = e / J;
      a = r % NA;
      ll = r / NA;
    } else {
      jj = e % J;
      const int r = e / J;
      ll = r % J;
      a = r / J;
    }
    a += a0;
    const bool hj = (jj < H) || (jj >= H + TJ), hl = (ll < H) || (ll >= H + TJ);
    if (hj && hl) continue;
    const int gj = j0 - H + jj, gl = l0 - H + ll, ic = cc * ND + a;
    T v = T(0);
    if (gj >= 0 && gj < m && gl >= 0 && gl < m && ic > 0 && ic < m) v = u[ic * sc + gj * s1 + gl * s2];
    U[(a * J + ll) * StagePitch<K, T>::value + jj] = v;
  }
}

// Element e of the staged layers 1..K+1 of a cell: (a, jj, ll) in global
// memory order (x fastest) so that loads coalesce.
template <int K>
__device__ __forceinline__ void stage_decode(int e, int c, int& a, int& jj, int& ll) {
  using Cfg = ApplyCfg<K>;
  constexpr int ND = Cfg::ND, J = Cfg::J;
  if (c == 0) {
    a = e % ND;
    const int r = e / ND;
    jj = r % J;
    ll = r / J;
  } else if (c == 1) {
    jj = e % J;
    const int r = e / J;
    a = r % ND;
    ll = r / ND;
  } else {
    jj = e % J;
    const int r = e / J;
    ll = r % J;
    a = r / J;
  }
  a += 1;
}

// Which elements of layers 1..K+1 this thread stages, worked out once per
// CTA: the element's global offset for cell 0 (-1: never loaded: a corner or
// outside the domain in d1 / d2), its shared-memory index (-1: not stored)
// and whether it is the cell's top node (ic = m on the last cell: load 0).
template <int NREG>
struct StagePlan {
  int goff[NREG];
  int sidx[NREG];
  unsigned top;
};

template <int K, typename T, int NREG>
__device__ __forceinline__ void stage_plan(StagePlan<NREG>& pl, int c, int j0, int l0, int m, int64_t s1,
                                           int64_t s2, int64_t sc) {
  using Cfg = ApplyCfg<K>;
  constexpr int ND = Cfg::ND, TJ = Cfg::TJ, H = Cfg::H, J = Cfg::J, NT = Cfg::NT;
  constexpr int total = ND * J * J;
  pl.top = 0u;
#pragma unroll
  for (int i = 0; i < NREG; ++i) {
    const int e = threadIdx.x + i * NT;
    pl.goff[i] = -1;
    pl.sidx[i] = -1;
    if (e < total) {
      int a, jj, ll;
      stage_decode<K>(e, c, a, jj, ll);
      const bool hj = (jj < H) || (jj >= H + TJ), hl = (ll < H) || (ll >= H + TJ);
      if (!(hj && hl)) {
        pl.sidx[i] = (a * J + ll) * StagePitch<K, T>::value + jj;
        const int gj = j0 - H + jj, gl = l0 - H + ll;
        if (gj >= 0 && gj < m && gl >= 0 && gl < m) pl.goff[i] = (int)(a * sc + gj * s1 + gl * s2);
        if (a == ND) pl.top |= 1u << i;
      }
    }
  }
}

// Load layers 1..K+1 of cell cc into registers (corners and out-of-domain: 0).
template <int K, typename T, int NREG>
__device__ __forceinline__ void stage_fetch(T* regs, const T* __restrict__ u, const StagePlan<NREG>& pl, int cc,
                                            bool last_cell, int64_t sc) {
  constexpr int ND = ApplyCfg<K>::ND;
  const T* base = u + (int64_t)cc * ND * sc;
#pragma unroll
  for (int i = 0; i < NREG; ++i) {
    const bool ok = pl.goff[i] >= 0 && !(last_cell && ((pl.top >> i) & 1u));
    regs[i] = ok ? base[pl.goff[i]] : T(0);
  }
}

template <int K, typename T, int NREG>
__device__ __forceinline__ void stage_put(T* __restrict__ U, const T* regs, const StagePlan<NREG>& pl) {
#pragma unroll
  for (int i = 0; i < NREG; ++i)
    if (pl.sidx[i] >= 0) U[pl.sidx[i]] = regs[i];
}

// One run of the velocity march: cells cc0 .. cc1-1 of column col
// (component c = col / tiles, tile col % tiles), after a carry-only step for
// the cell below cc0 when cc0 > 0.  U is the staging buffer, srow / sct the
// FP64 row and contraction tables.
template <int K, typename T, bool RES>
__device__ __forceinline__ void march_run(const ApplyArgs<T>& A, const CellTables<T>& tab, T* __restrict__ U,
                                          const T* __restrict__ srow, const T* __restrict__ sct, int col, int cc0,
                                          int cc1) {
  using Cfg = ApplyCfg<K>;
  constexpr int ND = Cfg::ND, NC = Cfg::NC, TJ = Cfg::TJ, H = Cfg::H, J = Cfg::J, NT = Cfg::NT;
  constexpr int JP = StagePitch<K, T>::value;
  constexpr bool ROWREG = sizeof(T) == 4;
  constexpr int RW = 3 * ND;
  constexpr int CP = NC / 2, CQ = ND / 2;
  constexpr int CNE = CP + (NC % 2), CQE = CQ + (ND % 2);
  constexpr int SCW = CNE * CNE + CP * CP + CNE * CQ + CP * CQE;
  const int tid = threadIdx.x, tj = tid % TJ, tl = tid / TJ;
  const int m = A.m, n = A.n;
  const int tiles = A.ntile * A.ntile;

  const int c = col / tiles, tile = col - c * tiles;
  const int d1 = (c == 0) ? 1 : 0;
  const int d2 = (c == 2) ? 1 : 2;
  const int j0 = (tile % A.ntile) * TJ, l0 = (tile / A.ntile) * TJ;
  const int jn = j0 + tj, ln = l0 + tl;
  const bool active = (jn < m) && (ln < m);

  // strides of u_c along c, d1, d2 (x-fastest grid, extent m+1 along c) and of p
  const int64_t E0 = (c == 0) ? m + 1 : m, E1 = (c == 1) ? m + 1 : m;
  const int64_t sc = (c == 0) ? 1 : (c == 1 ? E0 : E0 * E1);
  const int64_t s1 = (d1 == 0) ? 1 : E0;
  const int64_t s2 = (d2 == 1) ? E0 : E0 * E1;
  const int64_t mm = (int64_t)m * m;
  const int64_t psc = (c == 0) ? 1 : (c == 1 ? m : mm);
  const int64_t ps1 = (d1 == 0) ? 1 : m;
  const int64_t ps2 = (d2 == 1) ? m : mm;
  const int64_t nvel = (int64_t)(m + 1) * m * m;
  const T* u = A.x + c * nvel;
  const T* p = A.x + 3 * nvel;
  T* yc = A.y + c * nvel;
  const T* bc = RES ? A.b + c * nvel : nullptr;

  const int cj = jn / ND, bj = jn - cj * ND, cl = ln / ND, bl = ln - cl * ND;
  const int typej = (cj == 0) ? 1 : ((cj == n - 1) ? 2 : 0);
  const int typel = (cl == 0) ? 1 : ((cl == n - 1) ? 2 : 0);
  const int64_t line_off = (int64_t)jn * s1 + (int64_t)ln * s2;
  const int64_t pline_off = (int64_t)jn * ps1 + (int64_t)ln * ps2;

  T tcar = T(0), ucar = T(0), zcar = T(0);
  const T sj = tab.S[bj], sl = tab.S[bl], ss = sj * sl;
  const T* row1 = ROWREG ? nullptr : srow + ((typej * ND + bl) * ND + bj) * RW;
  const T* row2 = ROWREG ? nullptr : srow + ((typel * ND + bj) * ND + bl) * RW;
  const T* ctab = ROWREG ? nullptr : sct + (bj * ND + bl) * SCW;
  T r1s[ND], r1lo[ND], r1hi[ND], r2s[ND], r2lo[ND], r2hi[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    r1s[q] = ROWREG ? tab.LS[typej][bj * ND + q] : T(0);
    r1lo[q] = ROWREG ? tab.LLO[bj * ND + q] : T(0);
    r1hi[q] = ROWREG ? tab.LHI[bj * ND + q] : T(0);
    r2s[q] = ROWREG ? tab.LS[typel][bl * ND + q] : T(0);
    r2lo[q] = ROWREG ? tab.LLO[bl * ND + q] : T(0);
    r2hi[q] = ROWREG ? tab.LHI[bl * ND + q] : T(0);
  }

  // Software pipeline (FP32): the layers, pressure values and b entries of the
  // next cell are fetched into registers while the current cell is computed.
  // FP64 is bound by the FP64 pipe and stages synchronously (fewer registers).
  constexpr bool PIPE = sizeof(T) == 4 && K <= 3;
  constexpr int NREG = PIPE ? (ND * J * J + NT - 1) / NT : 1;
  T nxt[NREG];
  StagePlan<NREG> plan;
  if constexpr (PIPE) stage_plan<K, T, NREG>(plan, c, j0, l0, m, s1, s2, sc);
  T pv_next[ND], b_next[ND];
  const int cstart = (cc0 > 0 ? cc0 - 1 : 0);
  // the first step of a run computes its bottom node; later steps carry it
  stage_layers<K, T, NC>(U, u, 0, c, cstart, j0, l0, m, sc, s1, s2);
  if (active) {
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      pv_next[q] = p[(int64_t)(cstart * ND + q) * psc + pline_off];
      b_next[q] = RES ? bc[(int64_t)(cstart * ND + q) * sc + line_off] : T(0);
    }
  }
  __syncthreads();
  for (int cc = cstart; cc < cc1; ++cc) {
    const bool warm = cc < cc0;  // carry-only step for the cell below the run
    const int a0 = (cc == cstart) ? 0 : 1;
    T pv[ND], bv[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      pv[q] = ROWREG ? ss * pv_next[q] : pv_next[q];
      bv[q] = b_next[q];
    }
    const bool has_next = cc + 1 < cc1;
    if (has_next) {
      if constexpr (PIPE) stage_fetch<K, T, NREG>(nxt, u, plan, cc + 1, cc + 1 == n - 1, sc);
      if (active) {
#pragma unroll
        for (int q = 0; q < ND; ++q) {
          pv_next[q] = p[(int64_t)((cc + 1) * ND + q) * psc + pline_off];
          b_next[q] = RES ? bc[(int64_t)((cc + 1) * ND + q) * sc + line_off] : T(0);
        }
      }
    }
    if (active) {
      T tv[NC], uv[NC], z[NC];
      tv[0] = tcar;
      uv[0] = ucar;
#pragma unroll
      for (int a = 0; a < NC; ++a) {
        if (a < a0) continue;
        const T* row = &U[(a * J + tl + H) * JP];
        const int bj0 = tj - bj + H;
        const int bl0 = tl - bl + H;
        if constexpr (ROWREG) {
          T acc1 = T(0), acc2 = T(0);
#pragma unroll
          for (int q = 0; q < ND; ++q) {
            acc1 += r1s[q] * row[bj0 + q];
            acc1 += r1lo[q] * row[bj0 - ND + q];
            acc1 += r1hi[q] * row[bj0 + ND + q];
          }
#pragma unroll
          for (int q = 0; q < ND; ++q) {
            acc2 += r2s[q] * U[(a * J + bl0 + q) * JP + tj + H];
            acc2 += r2lo[q] * U[(a * J + bl0 - ND + q) * JP + tj + H];
            acc2 += r2hi[q] * U[(a * J + bl0 + ND + q) * JP + tj + H];
          }
          tv[a] = sl * acc1 + sj * acc2;
        } else {
          T acc = T(0);
#pragma unroll
          for (int q = 0; q < ND; ++q) {
            acc += row1[q] * row[bj0 + q];
            acc += row1[ND + q] * row[bj0 - ND + q];
            acc += row1[2 * ND + q] * row[bj0 + ND + q];
          }
#pragma unroll
          for (int q = 0; q < ND; ++q) {
            acc += row2[q] * U[(a * J + bl0 + q) * JP + tj + H];
            acc += row2[ND + q] * U[(a * J + bl0 - ND + q) * JP + tj + H];
            acc += row2[2 * ND + q] * U[(a * J + bl0 + ND + q) * JP + tj + H];
          }
          tv[a] = acc;
        }
        uv[a] = ROWREG ? ss * U[(a * J + tl + H) * JP + tj + H] : U[(a * J + tl + H) * JP + tj + H];
      }
      // contraction along c, even-odd form (ContractTables)
      constexpr int P = NC / 2, Q = ND / 2;
      constexpr bool CC = NC % 2 == 1, CD = ND % 2 == 1;
      constexpr int NE = P + (CC ? 1 : 0), QE = Q + (CD ? 1 : 0);
      T ue[NE], te[NE], uo[P], to[P], pe[QE], po[Q];
#pragma unroll
      for (int a = 0; a < P; ++a) {
        ue[a] = uv[a] + uv[NC - 1 - a];
        uo[a] = uv[a] - uv[NC - 1 - a];
        te[a] = tv[a] + tv[NC - 1 - a];
        to[a] = tv[a] - tv[NC - 1 - a];
      }
      if constexpr (CC) {
        ue[P] = uv[P];
        te[P] = tv[P];
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        pe[q] = pv[q] + pv[ND - 1 - q];
        po[q] = pv[q] - pv[ND - 1 - q];
      }
      if constexpr (CD) pe[Q] = pv[Q];
#pragma unroll
      for (int i = 0; i < NE; ++i) {
        T ze = T(0), zo = T(0);
#pragma unroll
        for (int a = 0; a < NE; ++a)
          ze += (ROWREG ? A.ce.EK[i * kMaxC + a] : ctab[i * NE + a]) * ue[a] + A.ce.EM[i * kMaxC + a] * te[a];
#pragma unroll
        for (int q = 0; q < Q; ++q)
          ze += (ROWREG ? A.ce.ED[i * kMaxD + q] : ctab[NE * NE + P * P + i * Q + q]) * po[q];
        if (i < P) {
#pragma unroll
          for (int a = 0; a < P; ++a)
            zo += (ROWREG ? A.ce.OK[i * kMaxC + a] : ctab[NE * NE + i * P + a]) * uo[a] + A.ce.OM[i * kMaxC + a] * to[a];
#pragma unroll
          for (int q = 0; q < QE; ++q)
            zo += (ROWREG ? A.ce.OD[i * kMaxD + q] : ctab[NE * NE + P * P + NE * Q + i * QE + q]) * pe[q];
          z[i] = ze + zo;
          z[NC - 1 - i] = ze - zo;
        } else {
          z[i] = ze;
        }
      }
      if (!warm) {
#pragma unroll
        for (int i = 0; i < ND; ++i) {
          const int ic = cc * ND + i;
          const int64_t g = (int64_t)ic * sc + line_off;
          T val = (i == 0) ? z[0] + zcar : z[i];
          if constexpr (RES) val = bv[i] - val;
          yc[g] = (ic == 0) ? T(0) : val;
        }
        if (cc == n - 1) yc[(int64_t)m * sc + line_off] = T(0);
      }
      tcar = tv[NC - 1];
      ucar = uv[NC - 1];
      zcar = z[NC - 1];
    }
    __syncthreads();
    if (has_next) {
      if constexpr (PIPE)
        stage_put<K, T, NREG>(U, nxt, plan);
      else
        stage_layers<K, T, ND>(U, u, 1, c, cc + 1, j0, l0, m, sc, s1, s2);
      __syncthreads();
    }
  }
}

// Resident CTAs per SM: 2 for k <= 4, 3 for the 2-cell tiles of k = 5.  One
// CTA per SM (the register count the compiler picks unbounded) left the FP64
// pipe half idle at k = 4 and 5; the register cap costs a few spills there and
// measured 1.2-1.3x faster at 64^3.
template <int K, typename T, bool RES>
__global__ void __launch_bounds__(ApplyCfg<K>::NT, (K <= 4 ? 2 : 3)) apply_velocity_kernel(ApplyArgs<T> A) {
  using Cfg = ApplyCfg<K>;
  constexpr int ND = Cfg::ND, NC = Cfg::NC, NT = Cfg::NT;
  __shared__ CellTables<T> tab;
  extern __shared__ __align__(16) unsigned char apply_smem[];
  T* U = reinterpret_cast<T*>(apply_smem);  // [NC][J][J] staged layers, jj fastest

  const int tid = threadIdx.x;
  const int n = A.n;
  for (int i = tid; i < (int)(sizeof(CellTables<T>) / sizeof(T)); i += NT)
    reinterpret_cast<T*>(&tab)[i] = reinterpret_cast<const T*>(&A.tv)[i];
  __syncthreads();
  // FP64: the 1D penalty rows with the mass of the other discontinuous
  // direction folded in, so that t = M_d2 L_d1 u + M_d1 L_d2 u is one sum of
  // products (two fewer FP64 operations per node), read from a shared table
  // of every (boundary type, mass node, row) (registers are the FP64
  // kernel's occupancy limit).  FP32 keeps this thread's two plain rows in
  // registers for the whole march and scales the two sums (the FP32 kernel
  // is latency-bound; the folded form cost it register spills).
  constexpr bool ROWREG = sizeof(T) == 4;
  constexpr int RW = 3 * ND;  // one scaled row: LS, LLO, LHI
  __shared__ T srow[ROWREG ? 1 : 3 * ND * ND * RW];
  if constexpr (!ROWREG) {
    for (int i = tid; i < 3 * ND * ND * RW; i += NT) {
      const int qq = i % RW, b = (i / RW) % ND, sidx = (i / (RW * ND)) % ND, t = i / (RW * ND * ND);
      const T v = qq < ND ? tab.LS[t][b * ND + qq] : (qq < 2 * ND ? tab.LLO[b * ND + qq - ND] : tab.LHI[b * ND + qq - 2 * ND]);
      srow[i] = tab.S[sidx] * v;
    }
    __syncthreads();
  }
  // FP64: the blocks of the contraction that act on u and p (EK, OK, ED, OD)
  // with this thread's cross-section mass S[bj] S[bl] folded in, one table
  // per (bj, bl), so that neither u nor p is scaled per node
  constexpr int CP = NC / 2, CQ = ND / 2;
  constexpr int CNE = CP + (NC % 2), CQE = CQ + (ND % 2);
  constexpr int SCW = CNE * CNE + CP * CP + CNE * CQ + CP * CQE;  // one (bj, bl) table
  __shared__ T sct[ROWREG ? 1 : ND * ND * SCW];
  if constexpr (!ROWREG) {
    for (int i = tid; i < ND * ND * SCW; i += NT) {
      const int w = i % SCW, sb = i / SCW, b1 = sb / ND, b2 = sb % ND;
      T v;
      if (w < CNE * CNE)
        v = A.ce.EK[(w / CNE) * kMaxC + w % CNE];
      else if (w < CNE * CNE + CP * CP)
        v = A.ce.OK[((w - CNE * CNE) / CP) * kMaxC + (w - CNE * CNE) % CP];
      else if (w < CNE * CNE + CP * CP + CNE * CQ) {
        const int o = w - CNE * CNE - CP * CP;
        v = CQ > 0 ? A.ce.ED[(o / (CQ > 0 ? CQ : 1)) * kMaxD + o % (CQ > 0 ? CQ : 1)] : T(0);
      } else {
        const int o = w - CNE * CNE - CP * CP - CNE * CQ;
        v = A.ce.OD[(o / CQE) * kMaxD + o % CQE];
      }
      sct[i] = tab.S[b1] * tab.S[b2] * v;
    }
    __syncthreads();
  }

  // Every column (component c, tile of (d1, d2) lines, n cells along c) is
  // cut into runs of `chunk` cells (the last one shorter), numbered column by
  // column.  FP32 (latency-bound, register-capped) and the spilling FP64
  // kernel of k = 5: one run per CTA, the grid covers every run.  FP64 up to
  // k = 4 (bound by the FP64 pipe): a balanced persistent march over one wave
  // of resident CTAs.  Round r of G = gridDim.x CTAs:
  // CTA g marches run g + r G, as long as a whole round remains, so the CTAs
  // of a round work on neighbouring tiles at the same heights and find the
  // halos they stage in L2.  The cells of the remaining runs (fewer than G)
  // are then split evenly: each CTA takes an equal contiguous range of them
  // in column order, which may start or end inside a run and span several,
  // so that all CTAs finish together and no partial last wave idles the SMs.
  constexpr bool PERSIST = velocity_persistent<K, T>();
  const int tiles = A.ntile * A.ntile, ncol = 3 * tiles, chunk = A.chunk;
  const int nch = (n + chunk - 1) / chunk;  // runs per column
  int rounds = 1, f = 0, fend = 0, r = 0;
  if constexpr (PERSIST) {
    const int G = gridDim.x;
    rounds = (ncol * nch) / G;
    const int u_rest = rounds * G;  // first run of the split remainder
    const int64_t f_rest = (int64_t)(u_rest / nch) * n + (int64_t)(u_rest % nch) * chunk;
    const int64_t rest = (int64_t)ncol * n - f_rest;
    f = (int)(f_rest + rest * blockIdx.x / G);
    fend = (int)(f_rest + rest * (blockIdx.x + 1) / G);
  }
  for (;;) {
    int col, cc0, cc1;
    if (r < rounds) {
      const int u = blockIdx.x + r * gridDim.x;
      ++r;
      col = u / nch;
      cc0 = (u - col * nch) * chunk;
      cc1 = min(n, cc0 + chunk);
    } else if (PERSIST && f < fend) {
      col = f / n;
      cc0 = f - col * n;
      cc1 = min(n, cc0 + (fend - f));
      f += cc1 - cc0;
    } else {
      break;
    }
    march_run<K, T, RES>(A, tab, U, srow, sct, col, cc0, cc1);
    if constexpr (!PERSIST) break;
  }
}

template <int K, typename T>
__global__ void __launch_bounds__(256) apply_pressure_kernel(ApplyArgs<T> A) {
  constexpr int ND = K + 1, NC = K + 2;
  __shared__ CellTables<T> tab;
  for (int i = threadIdx.x; i < (int)(sizeof(CellTables<T>) / sizeof(T)); i += blockDim.x)
    reinterpret_cast<T*>(&tab)[i] = reinterpret_cast<const T*>(&A.tv)[i];
  __syncthreads();
  const int m = A.m;
  const int64_t mm = (int64_t)m * m, np = mm * m;
  const int64_t nvel = (int64_t)(m + 1) * mm;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < np; idx += (int64_t)gridDim.x * blockDim.x) {
    const int px = (int)(idx % m), py = (int)((idx / m) % m), pz = (int)(idx / mm);
    const int pc[3] = {px, py, pz};
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
      int64_t E[3] = {m, m, m};
      E[c] = m + 1;
      const int64_t st[3] = {1, E[0], E[0] * E[1]};
      const int cell = pc[c] / ND, q = pc[c] - cell * ND;
      const T* u = A.x + c * nvel + (int64_t)pc[d1] * st[d1] + (int64_t)pc[d2] * st[d2];
      T s = T(0);
#pragma unroll
      for (int a = 0; a < NC; ++a) {
        const int ic = cell * ND + a;
        const T v = (ic > 0 && ic < m) ? u[(int64_t)ic * st[c]] : T(0);
        s += tab.D[q * NC + a] * v;
      }
      acc += tab.S[pc[d1] % ND] * tab.S[pc[d2] % ND] * s;
    }
    const int64_t g = 3 * nvel + idx;
    A.y[g] = A.alpha * acc + (A.b ? A.b[g] : T(0));
  }
}

// Resident CTAs of the velocity kernel on the whole GPU (one wave) and the SM count.
template <int K, typename T>
static cudaError_t velocity_wave(bool res, int* wave, int* nsm) {
  using Cfg = ApplyCfg<K>;
  const size_t smem = sizeof(T) * Cfg::NC * Cfg::J * StagePitch<K, T>::value;
  static std::atomic<unsigned long long> smem_set{0}, smem_set_res{0};
  static std::atomic<int> occ_plain{0}, occ_res{0};
  auto* kern = res ? apply_velocity_kernel<K, T, true> : apply_velocity_kernel<K, T, false>;
  cudaError_t e = allow_dynamic_smem(kern, smem, res ? smem_set_res : smem_set);
  if (e != cudaSuccess) return e;
  std::atomic<int>& occ = res ? occ_res : occ_plain;
  int per_sm = occ.load();
  if (per_sm == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::NT, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    occ.store(per_sm);
  }
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *nsm = std::max(sms, 1);
  *wave = per_sm * *nsm;
  return e;
}

// cells of all (component, tile) columns of a level
template <int K>
static int64_t velocity_cells(const Level& L) {
  const int ntile = (L.m + ApplyCfg<K>::TJ - 1) / ApplyCfg<K>::TJ;
  return 3LL * ntile * ntile * L.n;
}

template <int K, typename T>
static cudaError_t launch_apply_k(const Level& L, const CellTables<T>& tab, const ContractTables<T>& ce, const T* x,
                                  const T* b, T* y, T alpha, int stages, cudaStream_t s) {
  // the two forms the library uses: y = A x and y = b - A x
  if (b ? alpha != T(-1) : alpha != T(1)) return cudaErrorInvalidValue;
  using Cfg = ApplyCfg<K>;
  ApplyArgs<T> a;
  a.x = x;
  a.b = b;
  a.y = y;
  a.alpha = alpha;
  a.tv = tab;
  a.ce = ce;
  a.n = L.n;
  a.m = L.m;
  a.ntile = (L.m + Cfg::TJ - 1) / Cfg::TJ;
  a.chunk = L.n;
  if (stages & 1) {
    int wave = 0, nsm = 1;
    const cudaError_t e = velocity_wave<K, T>(b != nullptr, &wave, &nsm);
    if (e != cudaSuccess) return e;
    // cells per run: the tuned value if set; else the persistent march takes
    // whole columns on one wave of resident CTAs (at least 4 cells each), and
    // one run per CTA cuts the columns so that there are about 8 CTAs per SM
    // with runs of at least 4 cells
    const int64_t total = velocity_cells<K>(L);
    const int tiles = a.ntile * a.ntile;
    const int tuned = L.apply_chunk[sizeof(T) == 8 ? STK_F64 : STK_F32];
    int nch = (8 * nsm + 3 * tiles - 1) / (3 * tiles);
    nch = std::max(1, std::min(nch, L.n / 4 > 0 ? L.n / 4 : 1));
    constexpr bool persist = velocity_persistent<K, T>();
    a.chunk = tuned > 0 ? std::min(tuned, L.n) : (persist ? L.n : (L.n + nch - 1) / nch);
    const int64_t runs = 3LL * tiles * ((L.n + a.chunk - 1) / a.chunk);
    const int64_t grid =
        persist ? std::max<int64_t>(1, std::min<int64_t>(wave, total / 4)) : runs;
    const size_t smem = sizeof(T) * Cfg::NC * Cfg::J * StagePitch<K, T>::value;
    if (b)
      apply_velocity_kernel<K, T, true><<<(unsigned)grid, Cfg::NT, smem, s>>>(a);
    else
      apply_velocity_kernel<K, T, false><<<(unsigned)grid, Cfg::NT, smem, s>>>(a);
  }
  if (stages & 2) {
    const int64_t np = (int64_t)L.m * L.m * L.m;
    int blocks = (int)std::min<int64_t>((np + 255) / 256, 152 * 16);
    apply_pressure_kernel<K, T><<<blocks, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch_apply(int k, const Level& L, const CellTables<T>& tab, const ContractTables<T>& ce,
                                  const T* x, const T* b, T* y, T alpha, int stages, cudaStream_t s) {
  switch (k) {
    case 1: return launch_apply_k<1, T>(L, tab, ce, x, b, y, alpha, stages, s);
    case 2: return launch_apply_k<2, T>(L, tab, ce, x, b, y, alpha, stages, s);
    case 3: return launch_apply_k<3, T>(L, tab, ce, x, b, y, alpha, stages, s);
    case 4: return launch_apply_k<4, T>(L, tab, ce, x, b, y, alpha, stages, s);
    case 5: return launch_apply_k<5, T>(L, tab, ce, x, b, y, alpha, stages, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply_on(const stk_problem* P, int level, int dtype, const void* x, const void* b, void* y,
                            double alpha, int stages, cudaStream_t stream) {
  if (P->dim == 2) {
    if (b ? alpha != -1.0 : alpha != 1.0) return cudaErrorInvalidValue;
    return launch_apply_planar(P, level, dtype, x, b, y, stages, stream);
  }
  const Level& L = P->levels[level];
  if (dtype == STK_F64)
    return dispatch_apply<double>(P->k, L, L.htab64, L.hce64, (const double*)x, (const double*)b, (double*)y, alpha,
                                  stages, stream);
  return dispatch_apply<float>(P->k, L, L.htab32, L.hce32, (const float*)x, (const float*)b, (float*)y, (float)alpha,
                               stages, stream);
}

cudaError_t launch_apply(const stk_problem* P, int level, int dtype, const void* x, const void* b, void* y,
                         double alpha, int stages) {
  return launch_apply_on(P, level, dtype, x, b, y, alpha, stages, P->stream);
}

}  // namespace stk
