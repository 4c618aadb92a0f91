// Right-hand side of a manufactured Stokes problem (Sec. 3.3): b_i = (f, phi_i)
// with f = -nu Laplace(u) + grad p (eq. `model`), u = curl(psi), integrated
// with the (k+3)-point Gauss rule of every cell; pressure rows are zero.
//
// The stream functions are seeded sums  psi_c = sum_t amp[c][t] G_a(x) G_b(y) G_c(z),
// G_a(s) = s^2 (1-s)^2 sin(a pi s), and p = sum_t pamp[t] cos(a pi x) cos(b pi y) cos(c pi z)
// (the paper's own psi uses constants it does not state).  All derivatives
// are exact: G^(n) follows from the Leibniz rule.  One CTA per cell tabulates
// the 1D factors at its quadrature points (one sincos per factor), evaluates
// f at the quadrature points and contracts it with the 1D bases one direction
// at a time; nodes on a cell face normal to a component's continuous
// direction receive two atomic contributions onto a zeroed vector.
#include <cmath>

#include "internal.h"
#include "manufactured.cuh"

namespace stk {

struct RhsParams {
  int psi_freq[3][3][3];  // [component][term][direction]
  double psi_amp[3][3];
  int p_freq[3][3];  // [term][direction]
  double p_amp[3];
  double nu, h;
  int n, m;
  double xq[kMaxDegree + 3], wq[kMaxDegree + 3];
  double VC[kMaxC][kMaxDegree + 3];  // continuous basis at the quadrature points
  double VD[kMaxD][kMaxDegree + 3];  // discontinuous basis at the quadrature points
};

template <int K>
__global__ void __launch_bounds__(256) rhs_kernel(const RhsParams P, double* __restrict__ b) {
  constexpr int NQ = K + 3, ND = K + 1, NC = K + 2;
  constexpr int NQ3 = NQ * NQ * NQ;
  __shared__ double F[3][NQ3];
  __shared__ double T1[NQ * NQ * NC];
  __shared__ double T2[NQ * NC * NC];
  // the 1D factors of the cell, tabulated once: G[c][t][d][q][n] = G^(n) of
  // term t of psi_c in direction d at quadrature point q; Pt: sin, cos of the
  // pressure terms
  __shared__ double G[3][3][3][NQ][4];
  __shared__ double Pt[3][3][NQ][2];
  const int cell = blockIdx.x;
  const int cidx[3] = {cell % P.n, (cell / P.n) % P.n, cell / (P.n * P.n)};
  for (int i = threadIdx.x; i < 27 * NQ; i += blockDim.x) {
    const int q = i % NQ, d = (i / NQ) % 3, t = (i / (3 * NQ)) % 3, c = i / (9 * NQ);
    G_all(P.psi_freq[c][t][d], (cidx[d] + P.xq[q]) * P.h, G[c][t][d][q]);
  }
  for (int i = threadIdx.x; i < 9 * NQ; i += blockDim.x) {
    const int q = i % NQ, d = (i / NQ) % 3, t = i / (3 * NQ);
    sincos(P.p_freq[t][d] * M_PI * (cidx[d] + P.xq[q]) * P.h, &Pt[t][d][q][0], &Pt[t][d][q][1]);
  }
  __syncthreads();
  // ---- forcing at the quadrature points, times the quadrature weight
  for (int q = threadIdx.x; q < NQ3; q += blockDim.x) {
    const int qi[3] = {q % NQ, (q / NQ) % NQ, q / (NQ * NQ)};
    const double W = P.wq[qi[0]] * P.wq[qi[1]] * P.wq[qi[2]] * P.h * P.h * P.h;
    // d_e Laplace(psi_c) for all c, e
    double dl[3][3];
    for (int c = 0; c < 3; ++c)
      for (int e = 0; e < 3; ++e) dl[c][e] = 0.0;
    for (int c = 0; c < 3; ++c)
      for (int t = 0; t < 3; ++t) {
        const double* g[3] = {G[c][t][0][qi[0]], G[c][t][1][qi[1]], G[c][t][2][qi[2]]};
        const double A = P.psi_amp[c][t];
        for (int e = 0; e < 3; ++e) {
          double s = 0.0;
          for (int l = 0; l < 3; ++l) {
            int o[3] = {0, 0, 0};
            o[e] += 1;
            o[l] += 2;
            s += g[0][o[0]] * g[1][o[1]] * g[2][o[2]];
          }
          dl[c][e] += A * s;
        }
      }
    // Laplace(u) = curl(Laplace(psi))
    const double lap[3] = {dl[2][1] - dl[1][2], dl[0][2] - dl[2][0], dl[1][0] - dl[0][1]};
    double gp[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < 3; ++t) {
      double cs[3], sn[3];
      for (int d = 0; d < 3; ++d) {
        sn[d] = Pt[t][d][qi[d]][0];
        cs[d] = Pt[t][d][qi[d]][1];
      }
      const double A = P.p_amp[t];
      gp[0] += -A * P.p_freq[t][0] * M_PI * sn[0] * cs[1] * cs[2];
      gp[1] += -A * P.p_freq[t][1] * M_PI * cs[0] * sn[1] * cs[2];
      gp[2] += -A * P.p_freq[t][2] * M_PI * cs[0] * cs[1] * sn[2];
    }
    for (int c = 0; c < 3; ++c) F[c][q] = W * (-P.nu * lap[c] + gp[c]);
  }
  __syncthreads();
  // ---- contract with the basis of each component (continuous direction: NC functions)
  for (int c = 0; c < 3; ++c) {
    int nb[3];
    for (int d = 0; d < 3; ++d) nb[d] = (d == c) ? NC : ND;
    // direction 2: T1[a2][q1][q0]
    for (int i = threadIdx.x; i < nb[2] * NQ * NQ; i += blockDim.x) {
      const int q01 = i % (NQ * NQ), a2 = i / (NQ * NQ);
      double s = 0.0;
      for (int q2 = 0; q2 < NQ; ++q2) s += (c == 2 ? P.VC[a2][q2] : P.VD[a2][q2]) * F[c][q2 * NQ * NQ + q01];
      T1[i] = s;
    }
    __syncthreads();
    // direction 1: T2[a2][a1][q0]
    for (int i = threadIdx.x; i < nb[2] * nb[1] * NQ; i += blockDim.x) {
      const int q0 = i % NQ, a1 = (i / NQ) % nb[1], a2 = i / (NQ * nb[1]);
      double s = 0.0;
      for (int q1 = 0; q1 < NQ; ++q1) s += (c == 1 ? P.VC[a1][q1] : P.VD[a1][q1]) * T1[(a2 * NQ + q1) * NQ + q0];
      T2[i] = s;
    }
    __syncthreads();
    const int64_t nvel = (int64_t)(P.m + 1) * P.m * P.m;
    int64_t E[3] = {P.m, P.m, P.m};
    E[c] = P.m + 1;
    for (int i = threadIdx.x; i < nb[0] * nb[1] * nb[2]; i += blockDim.x) {
      const int a0 = i % nb[0], a1 = (i / nb[0]) % nb[1], a2 = i / (nb[0] * nb[1]);
      double s = 0.0;
      for (int q0 = 0; q0 < NQ; ++q0) s += (c == 0 ? P.VC[a0][q0] : P.VD[a0][q0]) * T2[(a2 * nb[1] + a1) * NQ + q0];
      const int g[3] = {cidx[0] * ND + a0, cidx[1] * ND + a1, cidx[2] * ND + a2};
      if (g[c] == 0 || g[c] == P.m) continue;  // constrained normal DoF
      const int64_t idx = c * nvel + g[0] + E[0] * (g[1] + E[1] * (int64_t)g[2]);
      const int ac = (c == 0) ? a0 : (c == 1) ? a1 : a2;
      if (ac == 0 || ac == NC - 1)
        atomicAdd(&b[idx], s);
      else
        b[idx] = s;
    }
    __syncthreads();
  }
}

cudaError_t launch_rhs(const stk_problem* Pr, const int* psi_freq, const double* psi_amp, const int* p_freq,
                       const double* p_amp, double* b) {
  const Level& L = Pr->levels.back();
  const int k = Pr->k;
  RhsParams P{};
  for (int c = 0; c < 3; ++c)
    for (int t = 0; t < 3; ++t) {
      for (int d = 0; d < 3; ++d) P.psi_freq[c][t][d] = psi_freq[(c * 3 + t) * 3 + d];
      P.psi_amp[c][t] = psi_amp[c * 3 + t];
    }
  for (int t = 0; t < 3; ++t) {
    for (int d = 0; d < 3; ++d) P.p_freq[t][d] = p_freq[t * 3 + d];
    P.p_amp[t] = p_amp[t];
  }
  P.nu = Pr->nu;
  P.h = L.h;
  P.n = L.n;
  P.m = L.m;
  std::vector<double> xq, wq, V, Dv;
  gauss_legendre(k + 3, xq, wq);
  for (int q = 0; q < k + 3; ++q) {
    P.xq[q] = xq[q];
    P.wq[q] = wq[q];
  }
  lagrange(L.t1d.zC, xq, V, Dv);
  for (int a = 0; a < k + 2; ++a)
    for (int q = 0; q < k + 3; ++q) P.VC[a][q] = V[a * (k + 3) + q];
  lagrange(L.t1d.zD, xq, V, Dv);
  for (int a = 0; a < k + 1; ++a)
    for (int q = 0; q < k + 3; ++q) P.VD[a][q] = V[a * (k + 3) + q];
  cudaError_t e = cudaMemsetAsync(b, 0, sizeof(double) * (size_t)L.ntotal, Pr->stream);
  if (e != cudaSuccess) return e;
  const int blocks = L.n * L.n * L.n;
  switch (k) {
    case 1: rhs_kernel<1><<<blocks, 256, 0, Pr->stream>>>(P, b); break;
    case 2: rhs_kernel<2><<<blocks, 256, 0, Pr->stream>>>(P, b); break;
    case 3: rhs_kernel<3><<<blocks, 256, 0, Pr->stream>>>(P, b); break;
    case 4: rhs_kernel<4><<<blocks, 256, 0, Pr->stream>>>(P, b); break;
    case 5: rhs_kernel<5><<<blocks, 256, 0, Pr->stream>>>(P, b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace stk
