// Level transfers of the V-cycle (Sec. 3): prolongation I^up is the canonical
// embedding of the nested RT_k x DGQ_k spaces, restriction I^down its
// transpose (the residual restriction).
//
// In the nodal bases the embedding of one coarse cell into its 2x2x2 children
// is a Kronecker product of 1D child matrices
//     PC[ch][a][b] = l^C_b((ch + zC_a) / 2)   continuous direction (Gauss-Lobatto)
//     PD[ch][a][b] = l^D_b((ch + zD_a) / 2)   discontinuous direction (Gauss)
// for child ch in {0, 1}.  One CTA handles one coarse cell and contracts one
// direction at a time through shared memory (sum factorization).  Along a
// component's continuous direction every CTA writes the lower k+1 nodes of
// each child, so each fine node is written once; for the restriction the
// coarse nodes on a coarse face receive exactly two atomic contributions onto
// a zeroed vector, which is order independent.
#include <algorithm>

#include "internal.h"

namespace stk {

template <int K, typename T>
struct XferSmem {
  static constexpr int ND = K + 1, NC = K + 2;
  T X[NC * ND * ND];           // coarse cell values [bc][b1][b2]
  T T1[2 * NC * ND * ND];      // [ch2][bc][b1][a2]
  T T2[4 * NC * ND * ND];      // [ch1][ch2][bc][a1][a2]
  T PC[2 * NC * NC];
  T PD[2 * ND * ND];
};

// Geometry of field f (0..2 velocity component, 3 pressure) on a level with m nodes per side.
struct FieldGeom {
  int64_t off, st[3];
  int ext[3];
  int cdir;  // continuous direction, -1 for pressure
};

__device__ __forceinline__ FieldGeom field_geom(int f, int m) {
  FieldGeom g;
  const int64_t nvel = (int64_t)(m + 1) * m * m;
  g.cdir = f < 3 ? f : -1;
  for (int d = 0; d < 3; ++d) g.ext[d] = (d == g.cdir) ? m + 1 : m;
  g.st[0] = 1;
  g.st[1] = g.ext[0];
  g.st[2] = (int64_t)g.ext[0] * g.ext[1];
  g.off = (f < 3) ? f * nvel : 3 * nvel;
  return g;
}

template <int K, typename T>
__global__ void __launch_bounds__(128) prolongate_add_kernel(const T* __restrict__ xc, T* __restrict__ xf,
                                                              const T* __restrict__ ptab, int nc_cells) {
  constexpr int ND = K + 1, NC = K + 2;
  __shared__ XferSmem<K, T> s;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 2 * NC * NC; i += nt) s.PC[i] = ptab[i];
  for (int i = tid; i < 2 * ND * ND; i += nt) s.PD[i] = ptab[2 * NC * NC + i];
  const int cell = blockIdx.x;
  const int pcell[3] = {cell % nc_cells, (cell / nc_cells) % nc_cells, cell / (nc_cells * nc_cells)};
  const int mc = nc_cells * ND, mf = 2 * mc;
  for (int f = 0; f < 4; ++f) {
    const FieldGeom gc = field_geom(f, mc), gf = field_geom(f, mf);
    // directions in storage order: along x (0), y (1), z (2); n[d] nodes per cell
    int n[3];
    for (int d = 0; d < 3; ++d) n[d] = (d == gc.cdir) ? NC : ND;
    __syncthreads();
    for (int i = tid; i < n[0] * n[1] * n[2]; i += nt) {
      const int b0 = i % n[0], b1 = (i / n[0]) % n[1], b2 = i / (n[0] * n[1]);
      const int g[3] = {pcell[0] * ND + b0, pcell[1] * ND + b1, pcell[2] * ND + b2};
      const bool bnd = gc.cdir >= 0 && (g[gc.cdir] == 0 || g[gc.cdir] == mc);
      s.X[i] = bnd ? T(0) : xc[gc.off + g[0] * gc.st[0] + g[1] * gc.st[1] + g[2] * gc.st[2]];
    }
    __syncthreads();
    // contract direction 2: T1[ch2][b0][b1][a2] (a2 < ND: only lower nodes of each child)
    const T* P2 = (gc.cdir == 2) ? s.PC : s.PD;
    const int n2 = n[2];
    for (int i = tid; i < 2 * n[0] * n[1] * ND; i += nt) {
      const int b0 = i % n[0], b1 = (i / n[0]) % n[1], a2 = (i / (n[0] * n[1])) % ND, ch = i / (n[0] * n[1] * ND);
      T acc = T(0);
      for (int b2 = 0; b2 < n2; ++b2) acc += P2[(ch * n2 + a2) * n2 + b2] * s.X[(b2 * n[1] + b1) * n[0] + b0];
      s.T1[i] = acc;  // layout [ch2][a2][b1][b0]
    }
    __syncthreads();
    // contract direction 1: T2[ch1][ch2][a2][a1][b0]
    const T* P1 = (gc.cdir == 1) ? s.PC : s.PD;
    const int n1 = n[1];
    for (int i = tid; i < 4 * ND * ND * n[0]; i += nt) {
      const int b0 = i % n[0], a1 = (i / n[0]) % ND, a2 = (i / (n[0] * ND)) % ND, ch2 = (i / (n[0] * ND * ND)) % 2,
                ch1 = i / (n[0] * ND * ND * 2);
      T acc = T(0);
      for (int b1 = 0; b1 < n1; ++b1)
        acc += P1[(ch1 * n1 + a1) * n1 + b1] * s.T1[((ch2 * ND + a2) * n[1] + b1) * n[0] + b0];
      s.T2[i] = acc;
    }
    __syncthreads();
    // contract direction 0 and add into the fine vector
    const T* P0 = (gc.cdir == 0) ? s.PC : s.PD;
    const int n0 = n[0];
    for (int i = tid; i < 8 * ND * ND * ND; i += nt) {
      const int a0 = i % ND, a1 = (i / ND) % ND, a2 = (i / (ND * ND)) % ND, ch = i / (ND * ND * ND);
      const int ch0 = ch & 1, ch2 = (ch >> 1) & 1, ch1 = ch >> 2;
      T acc = T(0);
      for (int b0 = 0; b0 < n0; ++b0)
        acc += P0[(ch0 * n0 + a0) * n0 + b0] * s.T2[((((ch1 * 2 + ch2) * ND + a2) * ND + a1) * n[0]) + b0];
      const int g[3] = {(2 * pcell[0] + ch0) * ND + a0, (2 * pcell[1] + ch1) * ND + a1, (2 * pcell[2] + ch2) * ND + a2};
      if (gf.cdir >= 0 && g[gf.cdir] == 0) continue;  // constrained boundary normal node
      xf[gf.off + g[0] * gf.st[0] + g[1] * gf.st[1] + g[2] * gf.st[2]] += acc;
    }
  }
}

template <int K, typename T>
__global__ void __launch_bounds__(128) restrict_kernel(const T* __restrict__ rf, T* __restrict__ rc,
                                                        const T* __restrict__ ptab, int nc_cells) {
  constexpr int ND = K + 1, NC = K + 2;
  __shared__ XferSmem<K, T> s;
  __shared__ T Y[8 * ND * ND * ND];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 2 * NC * NC; i += nt) s.PC[i] = ptab[i];
  for (int i = tid; i < 2 * ND * ND; i += nt) s.PD[i] = ptab[2 * NC * NC + i];
  const int cell = blockIdx.x;
  const int pcell[3] = {cell % nc_cells, (cell / nc_cells) % nc_cells, cell / (nc_cells * nc_cells)};
  const int mc = nc_cells * ND, mf = 2 * mc;
  for (int f = 0; f < 4; ++f) {
    const FieldGeom gc = field_geom(f, mc), gf = field_geom(f, mf);
    int n[3];
    for (int d = 0; d < 3; ++d) n[d] = (d == gc.cdir) ? NC : ND;
    __syncthreads();
    // fine values of the 8 children, lower k+1 nodes per direction: Y[ch1][ch2][a2][a1][ch0][a0]
    for (int i = tid; i < 8 * ND * ND * ND; i += nt) {
      const int a0 = i % ND, ch0 = (i / ND) % 2, a1 = (i / (2 * ND)) % ND, a2 = (i / (2 * ND * ND)) % ND,
                ch2 = (i / (2 * ND * ND * ND)) % 2, ch1 = i / (4 * ND * ND * ND);
      const int g[3] = {(2 * pcell[0] + ch0) * ND + a0, (2 * pcell[1] + ch1) * ND + a1, (2 * pcell[2] + ch2) * ND + a2};
      const bool bnd = gf.cdir >= 0 && g[gf.cdir] == 0;
      Y[i] = bnd ? T(0) : rf[gf.off + g[0] * gf.st[0] + g[1] * gf.st[1] + g[2] * gf.st[2]];
    }
    __syncthreads();
    // direction 0: T2[ch1][ch2][a2][a1][b0] = sum_{ch0,a0} P0[ch0][a0][b0] Y
    const T* P0 = (gc.cdir == 0) ? s.PC : s.PD;
    const int n0 = n[0];
    for (int i = tid; i < 4 * ND * ND * n0; i += nt) {
      const int b0 = i % n0, rest = i / n0;  // rest = ((ch1*2+ch2)*ND + a2)*ND + a1
      T acc = T(0);
      for (int ch0 = 0; ch0 < 2; ++ch0)
        for (int a0 = 0; a0 < ND; ++a0) acc += P0[(ch0 * n0 + a0) * n0 + b0] * Y[(rest * 2 + ch0) * ND + a0];
      s.T2[i] = acc;
    }
    __syncthreads();
    // direction 1: T1[ch2][a2][b1][b0] = sum_{ch1,a1} P1[ch1][a1][b1] T2[ch1][ch2][a2][a1][b0]
    const T* P1 = (gc.cdir == 1) ? s.PC : s.PD;
    const int n1 = n[1];
    for (int i = tid; i < 2 * ND * n1 * n0; i += nt) {
      const int b0 = i % n0, b1 = (i / n0) % n1, a2 = (i / (n0 * n1)) % ND, ch2 = i / (n0 * n1 * ND);
      T acc = T(0);
      for (int ch1 = 0; ch1 < 2; ++ch1)
        for (int a1 = 0; a1 < ND; ++a1)
          acc += P1[(ch1 * n1 + a1) * n1 + b1] * s.T2[(((ch1 * 2 + ch2) * ND + a2) * ND + a1) * n0 + b0];
      s.T1[i] = acc;
    }
    __syncthreads();
    // direction 2 and accumulate into the coarse vector
    const T* P2 = (gc.cdir == 2) ? s.PC : s.PD;
    const int n2 = n[2];
    for (int i = tid; i < n0 * n1 * n2; i += nt) {
      const int b0 = i % n0, b1 = (i / n0) % n1, b2 = i / (n0 * n1);
      T acc = T(0);
      for (int ch2 = 0; ch2 < 2; ++ch2)
        for (int a2 = 0; a2 < ND; ++a2) acc += P2[(ch2 * n2 + a2) * n2 + b2] * s.T1[((ch2 * ND + a2) * n1 + b1) * n0 + b0];
      const int g[3] = {pcell[0] * ND + b0, pcell[1] * ND + b1, pcell[2] * ND + b2};
      if (gc.cdir >= 0 && (g[gc.cdir] == 0 || g[gc.cdir] == mc)) continue;
      atomicAdd(&rc[gc.off + g[0] * gc.st[0] + g[1] * gc.st[1] + g[2] * gc.st[2]], acc);
    }
  }
}

template <typename T>
static cudaError_t dispatch_xfer(bool prolong, int k, const T* in, T* out, const T* ptab, int nc_cells,
                                 cudaStream_t s) {
  const int blocks = nc_cells * nc_cells * nc_cells;
#define STK_XFER_CASE(KK)                                                                   \
  case KK:                                                                                  \
    if (prolong)                                                                            \
      prolongate_add_kernel<KK, T><<<blocks, 128, 0, s>>>(in, out, ptab, nc_cells);         \
    else                                                                                    \
      restrict_kernel<KK, T><<<blocks, 128, 0, s>>>(in, out, ptab, nc_cells);               \
    break;
  switch (k) {
    STK_XFER_CASE(1)
    STK_XFER_CASE(2)
    STK_XFER_CASE(3)
    STK_XFER_CASE(4)
    STK_XFER_CASE(5)
    default:
      return cudaErrorInvalidValue;
  }
#undef STK_XFER_CASE
  return cudaGetLastError();
}

cudaError_t launch_prolongate_add(const stk_problem* P, int fine_level, int dtype, const void* xc, void* xf) {
  if (P->dim == 2) return launch_prolongate_add_planar(P, fine_level, dtype, xc, xf);
  const Level& C = P->levels[fine_level - 1];
  if (dtype == STK_F64)
    return dispatch_xfer<double>(true, P->k, (const double*)xc, (double*)xf, P->xfer64, C.n, P->stream);
  return dispatch_xfer<float>(true, P->k, (const float*)xc, (float*)xf, P->xfer32, C.n, P->stream);
}

cudaError_t launch_restrict(const stk_problem* P, int fine_level, int dtype, const void* rf, void* rc) {
  if (P->dim == 2) return launch_restrict_planar(P, fine_level, dtype, rf, rc);
  const Level& C = P->levels[fine_level - 1];
  const size_t bytes = (size_t)C.ntotal * (dtype == STK_F64 ? 8 : 4);
  cudaError_t e = cudaMemsetAsync(rc, 0, bytes, P->stream);
  if (e != cudaSuccess) return e;
  if (dtype == STK_F64)
    return dispatch_xfer<double>(false, P->k, (const double*)rf, (double*)rc, P->xfer64, C.n, P->stream);
  return dispatch_xfer<float>(false, P->k, (const float*)rf, (float*)rc, P->xfer32, C.n, P->stream);
}

}  // namespace stk
