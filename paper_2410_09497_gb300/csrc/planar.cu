// The method on the unit square (the two-dimensional results of Table 1,
// Sec. 3.3): RT_k x DGQ_k on n x n cells (n = 2^L), k = 1..8, with the same
// operator, vertex-patch smoother, transfers and solver as in three
// dimensions, specialised to two.
//
// Layout [u_x | u_y | p], x fastest: u_x on (m+1) x m nodes (continuous in
// x), u_y on m x (m+1) (continuous in y), p on m x m, m = n (k+1).  The
// operator in Kronecker form (Sec. 2.3), with KC, MC, D, LS / LLO / LHI and S
// the 1D cell tables of the 3D path (tables.cpp):
//     y_x = KC_x (M_y u_x) + MC_x (L_y u_x) + D_x^T (M_y p)
//     y_y = KC_y (M_x u_y) + MC_y (L_x u_y) + D_y^T (M_x p)
//     y_p = D_x (M_y u_x) + D_y (M_x u_y).
// The 2D problems are small (the largest case of Table 1 has 64 M DoF), so
// the kernels take the degree at run time and favour plain code: one thread
// per output entry for the operator and the transfers.
//
// Local solver: the paper's Direct solver (Sec. 3.3), the pseudo-inverse of
// each patch type's matrix with the pressure mean fixed by a border row
// (built once on the host in FP64 by Gauss-Jordan elimination with partial
// pivoting).  In two dimensions the velocity block of a patch does not
// depend on h (stiffness ~ 1/h times mass ~ h, penalty ~ 1/h) and the
// divergence blocks scale with h, so A_h = S A_1 S with S = diag(I, h I):
// one inverse per type at h = 1 serves every level, A_h^+ = S^-1 A_1^+ S^-1,
// applied by scaling the pressure entries of the gathered residual and of
// the correction by 1/h.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"
#include "manufactured.cuh"

namespace stk {

namespace {

// offsets of the flat 1D tables (order of stk_cell_tables)
struct Flat {
  int nc, nd, KC, MC, D, LS, LLO, LHI, S, size;
  __host__ __device__ explicit Flat(int k) {
    nc = k + 2;
    nd = k + 1;
    KC = 0;
    MC = KC + nc * nc;
    D = MC + nc * nc;
    LS = D + nd * nc;
    LLO = LS + 3 * nd * nd;
    LHI = LLO + nd * nd;
    S = LHI + nd * nd;
    size = S + nd;
  }
};

int flat_size(int k) { return Flat(k).size; }

}  // namespace

// ------------------------------------------------------------------ operator
// y = A x (RES: y = b - A x) on one level; stages as in 3D (bit 0 velocity
// rows, bit 1 pressure rows).  Constrained rows are written 0.
template <typename T, bool RES>
__global__ void __launch_bounds__(256) apply_planar_kernel(const T* __restrict__ tab, const T* __restrict__ x,
                                                           const T* __restrict__ b, T* __restrict__ y, int n, int k,
                                                           int stages) {
  extern __shared__ __align__(16) unsigned char planar_smem[];
  T* t = reinterpret_cast<T*>(planar_smem);
  const Flat F(k);
  for (int i = threadIdx.x; i < F.size; i += blockDim.x) t[i] = tab[i];
  __syncthreads();
  const int nc = F.nc, nd = F.nd, m = n * nd;
  const T *KC = t + F.KC, *MC = t + F.MC, *D = t + F.D, *LS = t + F.LS, *LLO = t + F.LLO, *LHI = t + F.LHI,
          *S = t + F.S;
  const int64_t nvel = (int64_t)(m + 1) * m, N = 2 * nvel + (int64_t)m * m;
  const T* p = x + 2 * nvel;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    if (e < 2 * nvel) {
      if (!(stages & 1)) continue;
      const int c = (int)(e / nvel);
      const int64_t loc = e - c * nvel;
      const int E0 = c == 0 ? m + 1 : m;
      const int i0 = (int)(loc % E0), i1 = (int)(loc / E0);
      const int ic = c == 0 ? i0 : i1, id = c == 0 ? i1 : i0;
      if (ic == 0 || ic == m) {
        y[e] = T(0);
        continue;
      }
      const T* u = x + c * nvel;
      // u_c at continuous node jc, discontinuous node jd (constrained and outside: 0)
      auto U = [&](int jc, int jd) -> T {
        if (jc <= 0 || jc >= m || jd < 0 || jd >= m) return T(0);
        return c == 0 ? u[jc + (int64_t)(m + 1) * jd] : u[jd + (int64_t)m * jc];
      };
      const int ed = id / nd, bd = id % nd, td = ed == 0 ? 1 : (ed == n - 1 ? 2 : 0);
      const T sd = S[bd];
      int cells[2], locs[2], ncell;
      if (ic % nd == 0) {  // a node on a cell boundary belongs to two cells
        cells[0] = ic / nd - 1;
        locs[0] = nd;
        cells[1] = ic / nd;
        locs[1] = 0;
        ncell = 2;
      } else {
        cells[0] = ic / nd;
        locs[0] = ic % nd;
        ncell = 1;
      }
      for (int h = 0; h < ncell; ++h) {
        const int cc = cells[h], a = locs[h];
        for (int bb = 0; bb < nc; ++bb) {
          const int jc = cc * nd + bb;
          T lv = T(0);
          for (int q = 0; q < nd; ++q) {
            lv += LS[td * nd * nd + bd * nd + q] * U(jc, ed * nd + q);
            lv += LLO[bd * nd + q] * U(jc, (ed - 1) * nd + q);
            lv += LHI[bd * nd + q] * U(jc, (ed + 1) * nd + q);
          }
          acc += KC[a * nc + bb] * sd * U(jc, id) + MC[a * nc + bb] * lv;
        }
        for (int q = 0; q < nd; ++q) {
          const int pc = cc * nd + q;
          const T pv = c == 0 ? p[pc + (int64_t)m * id] : p[id + (int64_t)m * pc];
          acc += D[q * nc + a] * sd * pv;
        }
      }
    } else {
      if (!(stages & 2)) continue;
      const int64_t loc = e - 2 * nvel;
      const int px = (int)(loc % m), py = (int)(loc / m);
      for (int c = 0; c < 2; ++c) {
        const T* u = x + c * nvel;
        const int pc = c == 0 ? px : py, pd = c == 0 ? py : px;
        const int cell = pc / nd, q = pc % nd;
        T sdot = T(0);
        for (int a = 0; a < nc; ++a) {
          const int jc = cell * nd + a;
          if (jc <= 0 || jc >= m) continue;
          sdot += D[q * nc + a] * (c == 0 ? u[jc + (int64_t)(m + 1) * pd] : u[pd + (int64_t)m * jc]);
        }
        acc += S[pd % nd] * sdot;
      }
    }
    y[e] = RES ? b[e] - acc : acc;
  }
}

cudaError_t launch_apply_planar(const stk_problem* P, int level, int dtype, const void* x, const void* b, void* y,
                                int stages, cudaStream_t s) {
  const Level& L = P->levels[level];
  const int64_t N = L.ntotal;
  const int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 16);
  if (dtype == STK_F64) {
    const size_t smem = sizeof(double) * flat_size(P->k);
    if (b)
      apply_planar_kernel<double, true><<<blocks, 256, smem, s>>>(L.flat64, (const double*)x, (const double*)b,
                                                                   (double*)y, L.n, P->k, stages);
    else
      apply_planar_kernel<double, false><<<blocks, 256, smem, s>>>(L.flat64, (const double*)x, nullptr, (double*)y,
                                                                    L.n, P->k, stages);
  } else {
    const size_t smem = sizeof(float) * flat_size(P->k);
    if (b)
      apply_planar_kernel<float, true><<<blocks, 256, smem, s>>>(L.flat32, (const float*)x, (const float*)b,
                                                                  (float*)y, L.n, P->k, stages);
    else
      apply_planar_kernel<float, false><<<blocks, 256, smem, s>>>(L.flat32, (const float*)x, nullptr, (float*)y,
                                                                   L.n, P->k, stages);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------- transfers
// The 1D child matrices PC[ch][a][b], PD[ch][a][b] of transfer.cu; along a
// field's continuous direction every child owns its lower k+1 nodes, so each
// fine node has one parent cell.
template <typename T>
__global__ void __launch_bounds__(256) prolongate_planar_kernel(const T* __restrict__ ptab, const T* __restrict__ xc,
                                                                T* __restrict__ xf, int ncc, int k) {
  const int nc = k + 2, nd = k + 1;
  const T* PC = ptab;
  const T* PD = ptab + 2 * nc * nc;
  const int mc = ncc * nd, mf = 2 * mc;
  const int64_t nvf = (int64_t)(mf + 1) * mf, nvc = (int64_t)(mc + 1) * mc, Nf = 2 * nvf + (int64_t)mf * mf;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < Nf; e += (int64_t)gridDim.x * blockDim.x) {
    const int f = e < nvf ? 0 : (e < 2 * nvf ? 1 : 2);
    const int64_t loc = e - (f < 2 ? f * nvf : 2 * nvf);
    const int E0f = f == 0 ? mf + 1 : mf, E0c = f == 0 ? mc + 1 : mc;
    const int i[2] = {(int)(loc % E0f), (int)(loc / E0f)};
    if (f < 2 && (i[f] == 0 || i[f] == mf)) continue;  // constrained
    int pc[2], ch[2], a[2], nb[2];
    const T* Pm[2];
    for (int d = 0; d < 2; ++d) {
      const int fc = i[d] / nd;
      a[d] = i[d] % nd;
      pc[d] = fc / 2;
      ch[d] = fc % 2;
      nb[d] = (d == f) ? nc : nd;
      Pm[d] = (d == f) ? PC : PD;
    }
    const T* src = xc + (f < 2 ? f * nvc : 2 * nvc);
    T acc = T(0);
    for (int b1 = 0; b1 < nb[1]; ++b1) {
      const int j1 = pc[1] * nd + b1;
      const T w1 = Pm[1][(ch[1] * nb[1] + a[1]) * nb[1] + b1];
      for (int b0 = 0; b0 < nb[0]; ++b0) {
        const int j0 = pc[0] * nd + b0;
        if (f < 2) {
          const int jcont = f == 0 ? j0 : j1;
          if (jcont == 0 || jcont == mc) continue;
        }
        acc += Pm[0][(ch[0] * nb[0] + a[0]) * nb[0] + b0] * w1 * src[j0 + (int64_t)E0c * j1];
      }
    }
    xf[e] += acc;
  }
}

// rc = P^T rf: every coarse entry gathers from the fine nodes of the coarse
// cells that hold it (two cells for a continuous node on a cell boundary).
template <typename T>
__global__ void __launch_bounds__(256) restrict_planar_kernel(const T* __restrict__ ptab, const T* __restrict__ rf,
                                                              T* __restrict__ rc, int ncc, int k) {
  const int nc = k + 2, nd = k + 1;
  const T* PC = ptab;
  const T* PD = ptab + 2 * nc * nc;
  const int mc = ncc * nd, mf = 2 * mc;
  const int64_t nvf = (int64_t)(mf + 1) * mf, nvc = (int64_t)(mc + 1) * mc, Nc = 2 * nvc + (int64_t)mc * mc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < Nc; e += (int64_t)gridDim.x * blockDim.x) {
    const int f = e < nvc ? 0 : (e < 2 * nvc ? 1 : 2);
    const int64_t loc = e - (f < 2 ? f * nvc : 2 * nvc);
    const int E0c = f == 0 ? mc + 1 : mc, E0f = f == 0 ? mf + 1 : mf;
    const int j[2] = {(int)(loc % E0c), (int)(loc / E0c)};
    if (f < 2 && (j[f] == 0 || j[f] == mc)) {
      rc[e] = T(0);
      continue;
    }
    // (coarse cell, local node) pairs per direction
    int cells[2][2], locs[2][2], ncell[2], nb[2];
    const T* Pm[2];
    for (int d = 0; d < 2; ++d) {
      nb[d] = (d == f) ? nc : nd;
      Pm[d] = (d == f) ? PC : PD;
      ncell[d] = 0;
      if (d == f && j[d] % nd == 0) {
        const int cc = j[d] / nd;
        if (cc - 1 >= 0) {
          cells[d][ncell[d]] = cc - 1;
          locs[d][ncell[d]++] = nd;
        }
        if (cc <= ncc - 1) {
          cells[d][ncell[d]] = cc;
          locs[d][ncell[d]++] = 0;
        }
      } else {
        cells[d][0] = j[d] / nd;
        locs[d][0] = j[d] % nd;
        ncell[d] = 1;
      }
    }
    const T* src = rf + (f < 2 ? f * nvf : 2 * nvf);
    T acc = T(0);
    for (int h1 = 0; h1 < ncell[1]; ++h1)
      for (int h0 = 0; h0 < ncell[0]; ++h0)
        for (int ch1 = 0; ch1 < 2; ++ch1)
          for (int a1 = 0; a1 < nd; ++a1) {
            const int i1 = (2 * cells[1][h1] + ch1) * nd + a1;
            const T w1 = Pm[1][(ch1 * nb[1] + a1) * nb[1] + locs[1][h1]];
            for (int ch0 = 0; ch0 < 2; ++ch0)
              for (int a0 = 0; a0 < nd; ++a0) {
                const int i0 = (2 * cells[0][h0] + ch0) * nd + a0;
                if (f < 2 && (f == 0 ? i0 : i1) == 0) continue;  // constrained fine node
                acc += Pm[0][(ch0 * nb[0] + a0) * nb[0] + locs[0][h0]] * w1 * src[i0 + (int64_t)E0f * i1];
              }
          }
    rc[e] = acc;
  }
}

cudaError_t launch_prolongate_add_planar(const stk_problem* P, int fine_level, int dtype, const void* xc, void* xf) {
  const Level& F = P->levels[fine_level];
  const int ncc = P->levels[fine_level - 1].n;
  const int blocks = (int)std::min<int64_t>((F.ntotal + 255) / 256, 152 * 16);
  if (dtype == STK_F64)
    prolongate_planar_kernel<double><<<blocks, 256, 0, P->stream>>>(P->xfer64, (const double*)xc, (double*)xf, ncc,
                                                                     P->k);
  else
    prolongate_planar_kernel<float><<<blocks, 256, 0, P->stream>>>(P->xfer32, (const float*)xc, (float*)xf, ncc,
                                                                    P->k);
  return cudaGetLastError();
}

cudaError_t launch_restrict_planar(const stk_problem* P, int fine_level, int dtype, const void* rf, void* rc) {
  const Level& C = P->levels[fine_level - 1];
  const int blocks = (int)std::min<int64_t>((C.ntotal + 255) / 256, 152 * 16);
  if (dtype == STK_F64)
    restrict_planar_kernel<double><<<blocks, 256, 0, P->stream>>>(P->xfer64, (const double*)rf, (double*)rc, C.n,
                                                                   P->k);
  else
    restrict_planar_kernel<float><<<blocks, 256, 0, P->stream>>>(P->xfer32, (const float*)rf, (float*)rc, C.n,
                                                                  P->k);
  return cudaGetLastError();
}

// ------------------------------------------------------------- patch solves
// Patch-local numbering: u_x (2k+1 continuous x 2k+2), u_y (2k+2 x 2k+1
// continuous), p (2k+2 x 2k+2), x fastest in each.
__device__ __forceinline__ int64_t planar_patch_global(int j, int v0, int v1, int k, int m) {
  const int nd = k + 1, npc = 2 * k + 1, npd = 2 * k + 2, nv = npc * npd;
  const int64_t nvel = (int64_t)(m + 1) * m;
  if (j < nv) {
    const int ix = j % npc, iy = j / npc;
    return ((int64_t)(v0 - 1) * nd + 1 + ix) + (int64_t)(m + 1) * ((v1 - 1) * nd + iy);
  }
  if (j < 2 * nv) {
    const int jj = j - nv, ix = jj % npd, iy = jj / npd;
    return nvel + ((int64_t)(v0 - 1) * nd + ix) + (int64_t)m * ((v1 - 1) * nd + 1 + iy);
  }
  const int jj = j - 2 * nv, ix = jj % npd, iy = jj / npd;
  return 2 * nvel + ((int64_t)(v0 - 1) * nd + ix) + (int64_t)m * ((v1 - 1) * nd + iy);
}

// One CTA per patch of a colour (mode 0) or the single patch of the 2 x 2
// coarse mesh (mode 1): gather r, multiply by the patch type's inverse
// (columns read coalesced across the threads), scatter x += the correction.
template <typename T>
__global__ void __launch_bounds__(256) patch_planar_kernel(const T* const* __restrict__ inv, const T* __restrict__ r,
                                                           T* __restrict__ x, int n, int k, int colour, int cnt0,
                                                           T inv_h, int mode) {
  extern __shared__ __align__(16) unsigned char planar_smem[];
  T* rl = reinterpret_cast<T*>(planar_smem);
  const int npc = 2 * k + 1, npd = 2 * k + 2, nv = npc * npd, nloc = 2 * nv + npd * npd, m = n * (k + 1);
  int v0 = 1, v1 = 1;
  if (mode == 0) {
    const int t0 = blockIdx.x % cnt0, t1 = blockIdx.x / cnt0;
    v0 = (colour & 1) ? 2 * t0 + 1 : 2 * t0 + 2;
    v1 = (colour & 2) ? 2 * t1 + 1 : 2 * t1 + 2;
  }
  const int ty0 = (v0 == 1 ? 1 : 0) | (v0 == n - 1 ? 2 : 0), ty1 = (v1 == 1 ? 1 : 0) | (v1 == n - 1 ? 2 : 0);
  const T* M = inv[ty0 + 4 * ty1];
  for (int j = threadIdx.x; j < nloc; j += blockDim.x)
    rl[j] = r[planar_patch_global(j, v0, v1, k, m)] * (j >= 2 * nv ? inv_h : T(1));
  __syncthreads();
  for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
    T acc = T(0);
    for (int j = 0; j < nloc; ++j) acc += M[(int64_t)j * nloc + i] * rl[j];
    if (i >= 2 * nv) acc *= inv_h;
    const int64_t g = planar_patch_global(i, v0, v1, k, m);
    x[g] += acc;
  }
}

static int planar_block(int k) { return std::min(256, ((2 * (2 * k + 1) * (2 * k + 2) + (2 * k + 2) * (2 * k + 2)) + 31) / 32 * 32); }

cudaError_t launch_patch_colour_planar(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x) {
  const Level& L = P->levels[level];
  const int cnt0 = (colour & 1) ? L.n / 2 : (L.n - 1) / 2, cnt1 = (colour & 2) ? L.n / 2 : (L.n - 1) / 2;
  const int nb = cnt0 * cnt1;
  if (nb == 0) return cudaSuccess;
  const int nloc = P->pinv2->nloc, bs = planar_block(P->k);
  if (dtype == STK_F64)
    patch_planar_kernel<double><<<nb, bs, sizeof(double) * nloc, P->stream>>>(
        P->pinv2->tab64, (const double*)r, (double*)x, L.n, P->k, colour, cnt0, 1.0 / L.h, 0);
  else
    patch_planar_kernel<float><<<nb, bs, sizeof(float) * nloc, P->stream>>>(
        P->pinv2->tab32, (const float*)r, (float*)x, L.n, P->k, colour, cnt0, (float)(1.0 / L.h), 0);
  return cudaGetLastError();
}

// x = A_0^+ b on the 2 x 2 mesh: its one vertex patch holds every free DoF
cudaError_t launch_coarse_solve_planar(const stk_problem* P, int dtype, const void* b, void* x) {
  const Level& L = P->levels[0];
  cudaError_t e = cudaMemsetAsync(x, 0, (size_t)L.ntotal * (dtype == STK_F64 ? 8 : 4), P->stream);
  if (e != cudaSuccess) return e;
  const int nloc = P->pinv2->nloc, bs = planar_block(P->k);
  if (dtype == STK_F64)
    patch_planar_kernel<double><<<1, bs, sizeof(double) * nloc, P->stream>>>(P->pinv2->tab64, (const double*)b,
                                                                              (double*)x, L.n, P->k, 0, 1, 1.0 / L.h, 1);
  else
    patch_planar_kernel<float><<<1, bs, sizeof(float) * nloc, P->stream>>>(P->pinv2->tab32, (const float*)b, (float*)x,
                                                                            L.n, P->k, 0, 1, (float)(1.0 / L.h), 1);
  return cudaGetLastError();
}

// ------------------------------------------------------- pressure mean (2D)
__global__ void __launch_bounds__(256) planar_mean_partial(const double* __restrict__ p, int m, int nd,
                                                           const double* __restrict__ S, double* __restrict__ partial) {
  __shared__ double red[2][8];
  const int64_t np = (int64_t)m * m;
  double a = 0.0, b = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.x * blockDim.x) {
    const double w = S[(int)(e % m) % nd] * S[(int)(e / m) % nd];
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
    for (int q = 0; q < 8; ++q) s += red[threadIdx.x][q];
    partial[blockIdx.x * 2 + threadIdx.x] = s;
  }
}

__global__ void planar_mean_shift(double* __restrict__ p, int64_t np, const double* __restrict__ partial, int nblocks) {
  double a = 0.0, b = 0.0;
  for (int q = 0; q < nblocks; ++q) {
    a += partial[2 * q];
    b += partial[2 * q + 1];
  }
  const double mean = a / b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.x * blockDim.x)
    p[e] -= mean;
}

cudaError_t launch_pressure_mean_planar(stk_problem* P, double* x, double* partial, int nblocks) {
  const Level& L = P->levels.back();
  double* p = x + 2 * L.nvel;
  planar_mean_partial<<<nblocks, 256, 0, P->stream>>>(p, L.m, P->k + 1, P->pmean_w, partial);
  planar_mean_shift<<<(int)std::min<int64_t>((L.npress + 255) / 256, 1216), 256, 0, P->stream>>>(p, L.npress, partial,
                                                                                                nblocks);
  return cudaGetLastError();
}

// ---------------------------------------------------- manufactured solution
// psi = sum_t psi_amp[t] G_a(x) G_b(y) (the first component's terms of the 3D
// coefficient arrays), u = (d_y psi, -d_x psi), p = sum_t p_amp[t] cos(a pi x)
// cos(b pi y); f = -nu Laplace(u) + grad p.  The paper's 2D reference solution
// (Sec. 3.3) has this form with one term.
struct PlanarRhs {
  int psi_freq[3][2];
  double psi_amp[3];
  int p_freq[3][2];
  double p_amp[3];
  double nu, h;
  int n, k, nq;
  double xq[kMaxPlanarDegree + 3], wq[kMaxPlanarDegree + 3];
  double VC[kMaxPlanarDegree + 2][kMaxPlanarDegree + 3];
  double VD[kMaxPlanarDegree + 1][kMaxPlanarDegree + 3];
};

// f_c at (x, y): velocity component c of -nu Laplace(u) + grad p
__device__ double planar_force(const PlanarRhs& R, int c, double x, double y) {
  double f = 0.0;
  for (int t = 0; t < 3; ++t) {
    double gx[4], gy[4];
    G_all(R.psi_freq[t][0], x, gx);
    G_all(R.psi_freq[t][1], y, gy);
    // u_x = G(x) G'(y): Laplace = G'' G' + G G'''; u_y = -G'(x) G(y): Laplace = -(G''' G + G' G'')
    if (c == 0)
      f += -R.nu * R.psi_amp[t] * (gx[2] * gy[1] + gx[0] * gy[3]);
    else
      f += R.nu * R.psi_amp[t] * (gx[3] * gy[0] + gx[1] * gy[2]);
    const double wa = R.p_freq[t][0] * M_PI, wb = R.p_freq[t][1] * M_PI;
    if (c == 0)
      f += -R.p_amp[t] * wa * sin(wa * x) * cos(wb * y);
    else
      f += -R.p_amp[t] * wb * cos(wa * x) * sin(wb * y);
  }
  return f;
}

// b_i = (f, phi_i) by the (k+3)-point Gauss rule of each cell: one thread per
// velocity entry, summing over the one or two cells that carry it
__global__ void __launch_bounds__(256) rhs_planar_kernel(const PlanarRhs R, double* __restrict__ b) {
  const int nd = R.k + 1, m = R.n * nd, nq = R.nq;
  const int64_t nvel = (int64_t)(m + 1) * m, N = 2 * nvel + (int64_t)m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    if (e >= 2 * nvel) {
      b[e] = 0.0;
      continue;
    }
    const int c = (int)(e / nvel);
    const int64_t loc = e - c * nvel;
    const int E0 = c == 0 ? m + 1 : m;
    const int i0 = (int)(loc % E0), i1 = (int)(loc / E0);
    const int ic = c == 0 ? i0 : i1, id = c == 0 ? i1 : i0;
    if (ic == 0 || ic == m) {
      b[e] = 0.0;
      continue;
    }
    const int ed = id / nd, bd = id % nd;
    int cells[2], locs[2], ncell;
    if (ic % nd == 0) {
      cells[0] = ic / nd - 1;
      locs[0] = nd;
      cells[1] = ic / nd;
      locs[1] = 0;
      ncell = 2;
    } else {
      cells[0] = ic / nd;
      locs[0] = ic % nd;
      ncell = 1;
    }
    double acc = 0.0;
    for (int h = 0; h < ncell; ++h)
      for (int qc = 0; qc < nq; ++qc) {
        const double sc = (cells[h] + R.xq[qc]) * R.h;
        const double wc = R.wq[qc] * R.VC[locs[h]][qc];
        for (int qd = 0; qd < nq; ++qd) {
          const double sdp = (ed + R.xq[qd]) * R.h;
          const double w = wc * R.wq[qd] * R.VD[bd][qd];
          acc += w * (c == 0 ? planar_force(R, 0, sc, sdp) : planar_force(R, 1, sdp, sc));
        }
      }
    b[e] = acc * R.h * R.h;
  }
}

static PlanarRhs planar_rhs_params(const stk_problem* P, const int* psi_freq, const double* psi_amp,
                                   const int* p_freq, const double* p_amp) {
  const Level& L = P->levels.back();
  PlanarRhs R{};
  for (int t = 0; t < 3; ++t) {
    R.psi_freq[t][0] = psi_freq[t * 3 + 0];  // component 0, term t, directions x, y
    R.psi_freq[t][1] = psi_freq[t * 3 + 1];
    R.psi_amp[t] = psi_amp[t];
    R.p_freq[t][0] = p_freq[t * 3 + 0];
    R.p_freq[t][1] = p_freq[t * 3 + 1];
    R.p_amp[t] = p_amp[t];
  }
  R.nu = P->nu;
  R.h = L.h;
  R.n = L.n;
  R.k = P->k;
  R.nq = P->k + 3;
  std::vector<double> xq, wq, V, Dv;
  gauss_legendre(R.nq, xq, wq);
  for (int q = 0; q < R.nq; ++q) {
    R.xq[q] = xq[q];
    R.wq[q] = wq[q];
  }
  lagrange(L.t1d.zC, xq, V, Dv);
  for (int a = 0; a < P->k + 2; ++a)
    for (int q = 0; q < R.nq; ++q) R.VC[a][q] = V[a * R.nq + q];
  lagrange(L.t1d.zD, xq, V, Dv);
  for (int a = 0; a < P->k + 1; ++a)
    for (int q = 0; q < R.nq; ++q) R.VD[a][q] = V[a * R.nq + q];
  return R;
}

cudaError_t launch_rhs_planar(const stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq,
                              const double* p_amp, double* b) {
  const PlanarRhs R = planar_rhs_params(P, psi_freq, psi_amp, p_freq, p_amp);
  const int64_t N = P->levels.back().ntotal;
  rhs_planar_kernel<<<(int)std::min<int64_t>((N + 255) / 256, 152 * 16), 256, 0, P->stream>>>(R, b);
  return cudaGetLastError();
}

// L2 errors of a discrete solution x against the manufactured u and -p (the
// discrete pressure approximates -p, Sec. 2 reading): one thread per cell at
// the (k+3)^2 Gauss points; partial[2 b] / [2 b + 1]: block sums of the
// squared velocity / pressure errors.
__global__ void __launch_bounds__(256) errors_planar_kernel(const PlanarRhs R, const double* __restrict__ x,
                                                            double* __restrict__ partial) {
  __shared__ double red[2][8];
  const int nd = R.k + 1, nc = R.k + 2, m = R.n * nd, nq = R.nq;
  const int64_t nvel = (int64_t)(m + 1) * m;
  double eu = 0.0, ep = 0.0;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < R.n * R.n; cell += gridDim.x * blockDim.x) {
    const int cx = cell % R.n, cy = cell / R.n;
    for (int qy = 0; qy < nq; ++qy)
      for (int qx = 0; qx < nq; ++qx) {
        const double X = (cx + R.xq[qx]) * R.h, Y = (cy + R.xq[qy]) * R.h, w = R.wq[qx] * R.wq[qy] * R.h * R.h;
        double uxh = 0.0, uyh = 0.0, ph = 0.0;
        for (int b = 0; b < nd; ++b)
          for (int a = 0; a < nc; ++a) {
            const int ja = cx * nd + a, jb = cy * nd + b;  // u_x: continuous x, discontinuous y
            const int ka = cy * nd + a, kb = cx * nd + b;  // u_y: continuous y, discontinuous x
            const double vx = (ja == 0 || ja == m) ? 0.0 : x[ja + (int64_t)(m + 1) * jb];
            const double vy = (ka == 0 || ka == m) ? 0.0 : x[nvel + kb + (int64_t)m * ka];
            uxh += vx * R.VC[a][qx] * R.VD[b][qy];
            uyh += vy * R.VC[a][qy] * R.VD[b][qx];
          }
        for (int b = 0; b < nd; ++b)
          for (int a = 0; a < nd; ++a)
            ph += x[2 * nvel + (cx * nd + a) + (int64_t)m * (cy * nd + b)] * R.VD[a][qx] * R.VD[b][qy];
        double ux = 0.0, uy = 0.0, p = 0.0;
        for (int t = 0; t < 3; ++t) {
          double gx[4], gy[4];
          G_all(R.psi_freq[t][0], X, gx);
          G_all(R.psi_freq[t][1], Y, gy);
          ux += R.psi_amp[t] * gx[0] * gy[1];
          uy -= R.psi_amp[t] * gx[1] * gy[0];
          p += R.p_amp[t] * cos(R.p_freq[t][0] * M_PI * X) * cos(R.p_freq[t][1] * M_PI * Y);
        }
        eu += w * ((uxh - ux) * (uxh - ux) + (uyh - uy) * (uyh - uy));
        ep += w * (ph + p) * (ph + p);
      }
  }
  for (int o = 16; o > 0; o >>= 1) {
    eu += __shfl_xor_sync(0xffffffffu, eu, o);
    ep += __shfl_xor_sync(0xffffffffu, ep, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = eu;
    red[1][threadIdx.x >> 5] = ep;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += red[threadIdx.x][q];
    partial[2 * blockIdx.x + threadIdx.x] = s;
  }
}

cudaError_t launch_errors_planar(const stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq,
                                 const double* p_amp, const double* x, double* partial, int nblocks) {
  const PlanarRhs R = planar_rhs_params(P, psi_freq, psi_amp, p_freq, p_amp);
  errors_planar_kernel<<<nblocks, 256, 0, P->stream>>>(R, x, partial);
  return cudaGetLastError();
}

// --------------------------------------------------------------- host setup
PlanarInverses::~PlanarInverses() {
  for (int t = 0; t < 16; ++t) {
    if (m64[t]) cudaFree(m64[t]);
    if (m32[t]) cudaFree(m32[t]);
  }
  if (tab64) cudaFree(tab64);
  if (tab32) cudaFree(tab32);
}

namespace {

// The matrix of the vertex patch of boundary types (t0, t1) at h = 1 in the
// patch-local numbering, bordered by the pressure ones-vector; Gauss-Jordan
// with partial pivoting; returns the leading nloc x nloc block of the
// inverse, column-major (the pseudo-inverse with the pressure mean fixed).
bool planar_patch_inverse(const Tables1D& t, int t0, int t1, std::vector<double>& out) {
  const int k = t.k, nc = k + 2, nd = k + 1, npc = 2 * k + 1, npd = 2 * k + 2;
  const int nv = npc * npd, np = npd * npd, nloc = 2 * nv + np, nb = nloc + 1;
  // 1D patch matrices: continuous (interior nodes 1..2k+1 of the two cells)
  std::vector<double> KCp(npc * npc, 0.0), MCp(npc * npc, 0.0), Dp(npd * npc, 0.0);
  for (int cell = 0; cell < 2; ++cell)
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < nc; ++b) {
        const int i = cell * nd + a - 1, j = cell * nd + b - 1;
        if (i < 0 || i >= npc || j < 0 || j >= npc) continue;
        KCp[i * npc + j] += t.KC[a * nc + b];
        MCp[i * npc + j] += t.MC[a * nc + b];
      }
  for (int cell = 0; cell < 2; ++cell)
    for (int q = 0; q < nd; ++q)
      for (int a = 0; a < nc; ++a) {
        const int j = cell * nd + a - 1;
        if (j < 0 || j >= npc) continue;
        Dp[(cell * nd + q) * npc + j] += t.D[q * nc + a];
      }
  // discontinuous direction of boundary type ty: [[LS, LHI], [LLO, LS]] and diag(S, S)
  auto Lp = [&](int ty, std::vector<double>& L, std::vector<double>& M) {
    L.assign(npd * npd, 0.0);
    M.assign(npd * npd, 0.0);
    const int s0 = (ty & 1) ? 1 : 0, s1 = (ty & 2) ? 2 : 0;
    for (int a = 0; a < nd; ++a) {
      M[a * npd + a] = t.S[a];
      M[(nd + a) * npd + nd + a] = t.S[a];
      for (int b = 0; b < nd; ++b) {
        L[a * npd + b] = t.LS[s0][a * nd + b];
        L[(nd + a) * npd + nd + b] = t.LS[s1][a * nd + b];
        L[a * npd + nd + b] = t.LHI[a * nd + b];
        L[(nd + a) * npd + b] = t.LLO[a * nd + b];
      }
    }
  };
  std::vector<double> Lx, Mx, Ly, My;
  Lp(t0, Lx, Mx);
  Lp(t1, Ly, My);
  std::vector<double> K((size_t)nb * nb, 0.0);  // row-major
  auto at = [&](int i, int j) -> double& { return K[(size_t)i * nb + j]; };
  // u_x rows (ix + npc iy), continuous in x: KC_x M_y + MC_x L_y; pressure columns D_x^T M_y
  for (int iy = 0; iy < npd; ++iy)
    for (int ix = 0; ix < npc; ++ix) {
      const int r = ix + npc * iy;
      for (int jy = 0; jy < npd; ++jy)
        for (int jx = 0; jx < npc; ++jx)
          at(r, jx + npc * jy) = KCp[ix * npc + jx] * My[iy * npd + jy] + MCp[ix * npc + jx] * Ly[iy * npd + jy];
      for (int py = 0; py < npd; ++py)
        for (int px = 0; px < npd; ++px) {
          const double v = Dp[px * npc + ix] * My[py * npd + iy];
          at(r, 2 * nv + px + npd * py) = v;
          at(2 * nv + px + npd * py, r) = v;
        }
    }
  // u_y rows (ix + npd iy), continuous in y: M_x KC_y + L_x MC_y; pressure columns M_x D_y^T
  for (int iy = 0; iy < npc; ++iy)
    for (int ix = 0; ix < npd; ++ix) {
      const int r = nv + ix + npd * iy;
      for (int jy = 0; jy < npc; ++jy)
        for (int jx = 0; jx < npd; ++jx)
          at(r, nv + jx + npd * jy) = Mx[ix * npd + jx] * KCp[iy * npc + jy] + Lx[ix * npd + jx] * MCp[iy * npc + jy];
      for (int py = 0; py < npd; ++py)
        for (int px = 0; px < npd; ++px) {
          const double v = Mx[px * npd + ix] * Dp[py * npc + iy];
          at(r, 2 * nv + px + npd * py) = v;
          at(2 * nv + px + npd * py, r) = v;
        }
    }
  for (int q = 0; q < np; ++q) {
    at(2 * nv + q, nloc) = 1.0;
    at(nloc, 2 * nv + q) = 1.0;
  }
  // Gauss-Jordan with partial pivoting on [K | I]
  std::vector<double> Inv((size_t)nb * nb, 0.0);
  for (int i = 0; i < nb; ++i) Inv[(size_t)i * nb + i] = 1.0;
  for (int col = 0; col < nb; ++col) {
    int piv = col;
    for (int i = col + 1; i < nb; ++i)
      if (std::fabs(at(i, col)) > std::fabs(at(piv, col))) piv = i;
    if (!(std::fabs(at(piv, col)) > 0.0)) return false;
    if (piv != col)
      for (int j = 0; j < nb; ++j) {
        std::swap(at(piv, j), at(col, j));
        std::swap(Inv[(size_t)piv * nb + j], Inv[(size_t)col * nb + j]);
      }
    const double d = 1.0 / at(col, col);
    for (int j = 0; j < nb; ++j) {
      at(col, j) *= d;
      Inv[(size_t)col * nb + j] *= d;
    }
    for (int i = 0; i < nb; ++i) {
      if (i == col) continue;
      const double f = at(i, col);
      if (f == 0.0) continue;
      double* ri = &K[(size_t)i * nb];
      const double* rc = &K[(size_t)col * nb];
      double* ii = &Inv[(size_t)i * nb];
      const double* ic = &Inv[(size_t)col * nb];
      for (int j = 0; j < nb; ++j) {
        ri[j] -= f * rc[j];
        ii[j] -= f * ic[j];
      }
    }
  }
  out.assign((size_t)nloc * nloc, 0.0);
  for (int j = 0; j < nloc; ++j)
    for (int i = 0; i < nloc; ++i) out[(size_t)j * nloc + i] = Inv[(size_t)i * nb + j];
  return true;
}

std::mutex g_pinv_mutex;
std::map<std::tuple<int, int, double, double>, std::weak_ptr<PlanarInverses>> g_pinv_cache;

}  // namespace

// Per level: the flat 1D tables; per problem: the patch inverses of the
// boundary types that occur on any level (from the process-wide cache).
cudaError_t setup_planar(stk_problem* P) {
  for (Level& L : P->levels) {
    std::vector<double> flat;
    for (const std::vector<double>* v : {&L.t1d.KC, &L.t1d.MC, &L.t1d.D, &L.t1d.LS[0], &L.t1d.LS[1], &L.t1d.LS[2],
                                         &L.t1d.LLO, &L.t1d.LHI, &L.t1d.S})
      flat.insert(flat.end(), v->begin(), v->end());
    std::vector<float> f32(flat.begin(), flat.end());
    cudaError_t e = dev_alloc(&L.flat64, sizeof(double) * flat.size());
    if (e == cudaSuccess) e = dev_alloc(&L.flat32, sizeof(float) * flat.size());
    if (e == cudaSuccess) e = cudaMemcpy(L.flat64, flat.data(), sizeof(double) * flat.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.flat32, f32.data(), sizeof(float) * flat.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(dev, P->k, P->nu, P->opt.penalty_factor);
  std::lock_guard<std::mutex> lock(g_pinv_mutex);
  std::shared_ptr<PlanarInverses> inv = g_pinv_cache[key].lock();
  if (!inv) {
    inv = std::make_shared<PlanarInverses>();
    const Tables1D t = build_tables(P->k, 1.0, P->nu, P->opt.penalty_factor);
    const int npc = 2 * P->k + 1, npd = 2 * P->k + 2;
    inv->nloc = 2 * npc * npd + npd * npd;
    const size_t nn = (size_t)inv->nloc * inv->nloc;
    std::vector<double> M;
    // the boundary types of meshes of 2 (type 3 only) and of 4 or more cells
    // (types 0, 1, 2) per direction
    for (int t1 = 0; t1 < 4 && e == cudaSuccess; ++t1)
      for (int t0 = 0; t0 < 4 && e == cudaSuccess; ++t0) {
        if ((t0 == 3) != (t1 == 3)) continue;
        if (!planar_patch_inverse(t, t0, t1, M)) return cudaErrorInvalidValue;
        std::vector<float> M32(M.begin(), M.end());
        const int slot = t0 + 4 * t1;
        e = dev_alloc(&inv->m64[slot], sizeof(double) * nn);
        if (e == cudaSuccess) e = dev_alloc(&inv->m32[slot], sizeof(float) * nn);
        if (e == cudaSuccess) e = cudaMemcpy(inv->m64[slot], M.data(), sizeof(double) * nn, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(inv->m32[slot], M32.data(), sizeof(float) * nn, cudaMemcpyHostToDevice);
      }
    if (e == cudaSuccess) e = dev_alloc(&inv->tab64, sizeof(double*) * 16);
    if (e == cudaSuccess) e = dev_alloc(&inv->tab32, sizeof(float*) * 16);
    if (e == cudaSuccess) e = cudaMemcpy(inv->tab64, inv->m64, sizeof(double*) * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(inv->tab32, inv->m32, sizeof(float*) * 16, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    g_pinv_cache[key] = inv;
  }
  P->pinv2 = inv;
  return cudaSuccess;
}

}  // namespace stk
