// Host-side tables of the vertex-patch local solver (setup only), Sec. 3.2.
//
// On a 2x2x2-cell vertex patch the velocity block of component c is
//     A_c = nu (Lc (x) M (x) M + Mc (x) L (x) M + Mc (x) M (x) L)     (eq. `block_A`)
// with the continuous-direction stiffness / mass Lc, Mc restricted to the
// 2k+1 patch-interior nodes and, in each discontinuous direction, the 1D
// interior-penalty operator L and the diagonal Gauss mass M restricted to the
// 2k+2 nodes of the two cells (principal submatrices of the global 1D
// matrices).  The fast diagonalization method (eq. `inverse2d`,
// eq. `fast_inverse`) needs the generalized eigenpairs L S = M S Lambda with
// S^T M S = I, computed here by a Cholesky reduction and the cyclic Jacobi
// eigenvalue method (Jacobi 1846; Golub & Van Loan, Matrix Computations,
// Sec. 8.5).  L depends on whether the patch touches the boundary in that
// direction: type 0 interior, 1 lower boundary, 2 upper boundary, 3 both.
#include <cmath>

#include "internal.h"

namespace stk {

// Symmetric eigen-decomposition A = Q diag(w) Q^T by cyclic Jacobi rotations.
static void jacobi_eigen(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& Q) {
  Q.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += A[i * n + j] * A[i * n + j];
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[p * n + p], aqq = A[q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // Q <- Q J
          const double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - s * qkq;
          Q[k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

// Generalized symmetric-definite eigenproblem K S = M S diag(lam), S^T M S = I.
void generalized_eigen(int n, const std::vector<double>& K, const std::vector<double>& M, std::vector<double>& S,
                       std::vector<double>& lam) {
  // Cholesky M = L L^T (lower)
  std::vector<double> L(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = M[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    L[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = M[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / L[j * n + j];
    }
  }
  // Linv = L^{-1}
  std::vector<double> Li(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    Li[j * n + j] = 1.0 / L[j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s -= L[i * n + k] * Li[k * n + j];
      Li[i * n + j] = s / L[i * n + i];
    }
  }
  // C = Linv K Linv^T
  std::vector<double> T(n * n, 0.0), C(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += Li[i * n + k] * K[k * n + j];
      T[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += T[i * n + k] * Li[j * n + k];
      C[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) C[i * n + j] = C[j * n + i] = 0.5 * (C[i * n + j] + C[j * n + i]);
  std::vector<double> Q;
  jacobi_eigen(n, C, lam, Q);
  // S = Linv^T Q
  S.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += Li[k * n + i] * Q[k * n + j];
      S[i * n + j] = s;
    }
}

// Reorders the generalized eigenpairs (columns of S, row-major n x n) of a
// reflection-symmetric 1D operator so that eigenvectors with v(n-1-i) = v(i)
// come first and those with v(n-1-i) = -v(i) after.  Returns false (and
// leaves S, lam unchanged) unless every column has a parity to rounding
// accuracy and the counts are ceil(n/2) even, floor(n/2) odd.
static bool sort_by_parity(int n, std::vector<double>& S, std::vector<double>& lam) {
  std::vector<int> even, odd;
  for (int j = 0; j < n; ++j) {
    double ps = 0.0, pa = 0.0;
    for (int i = 0; i < n; ++i) {
      const double a = S[i * n + j], b = S[(n - 1 - i) * n + j];
      ps += (a + b) * (a + b);
      pa += (a - b) * (a - b);
    }
    if (pa <= 1e-20 * ps)
      even.push_back(j);
    else if (ps <= 1e-20 * pa)
      odd.push_back(j);
    else
      return false;
  }
  if ((int)even.size() != (n + 1) / 2) return false;
  std::vector<int> order(even);
  order.insert(order.end(), odd.begin(), odd.end());
  std::vector<double> S2(n * n), l2(n);
  for (int jn = 0; jn < n; ++jn) {
    for (int i = 0; i < n; ++i) S2[i * n + jn] = S[i * n + order[jn]];
    l2[jn] = lam[order[jn]];
  }
  S.swap(S2);
  lam.swap(l2);
  return true;
}

PatchTables1D build_patch_tables(const Tables1D& t) {
  const int k = t.k, nc = k + 2, nd = k + 1;
  const int npc = 2 * k + 1, npd = 2 * k + 2;
  PatchTables1D P;
  P.k = k;
  P.nu = t.nu;
  // continuous direction: assemble the two cells, keep the interior nodes 1..2k+1 (nu removed)
  std::vector<double> K2((2 * k + 3) * (2 * k + 3), 0.0), M2((2 * k + 3) * (2 * k + 3), 0.0);
  for (int cell = 0; cell < 2; ++cell)
    for (int i = 0; i < nc; ++i)
      for (int j = 0; j < nc; ++j) {
        const int gi = cell * nd + i, gj = cell * nd + j;
        K2[gi * (2 * k + 3) + gj] += t.KC[i * nc + j] / t.nu;
        M2[gi * (2 * k + 3) + gj] += t.MC[i * nc + j];
      }
  std::vector<double> Kc(npc * npc), Mc(npc * npc);
  for (int i = 0; i < npc; ++i)
    for (int j = 0; j < npc; ++j) {
      Kc[i * npc + j] = K2[(i + 1) * (2 * k + 3) + (j + 1)];
      Mc[i * npc + j] = M2[(i + 1) * (2 * k + 3) + (j + 1)];
    }
  generalized_eigen(npc, Kc, Mc, P.SC, P.LC);
  P.eo_c = sort_by_parity(npc, P.SC, P.LC);
  // discontinuous directions, four boundary types
  for (int type = 0; type < 4; ++type) {
    const int t0 = (type & 1) ? 1 : 0;  // lower cell is the first cell of the mesh
    const int t1 = (type & 2) ? 2 : 0;  // upper cell is the last cell of the mesh
    std::vector<double> Kd(npd * npd, 0.0), Md(npd * npd, 0.0);
    for (int b = 0; b < nd; ++b)
      for (int c = 0; c < nd; ++c) {
        Kd[b * npd + c] = t.LS[t0][b * nd + c] / t.nu;
        Kd[(nd + b) * npd + nd + c] = t.LS[t1][b * nd + c] / t.nu;
        Kd[b * npd + nd + c] = t.LHI[b * nd + c] / t.nu;
        Kd[(nd + b) * npd + c] = t.LLO[b * nd + c] / t.nu;
      }
    for (int j = 0; j < npd; ++j) Md[j * npd + j] = t.S[j % nd];
    generalized_eigen(npd, Kd, Md, P.SD[type], P.LD[type]);
    // types 0 and 3 are symmetric under the reflection of the patch
    P.eo_d[type] = (type == 0 || type == 3) && sort_by_parity(npd, P.SD[type], P.LD[type]);
  }
  // local divergence factor: pressure nodes of the two cells x patch-interior velocity nodes
  P.DL.assign(npd * npc, 0.0);
  for (int q = 0; q < npd; ++q)
    for (int a = 0; a < npc; ++a) {
      const int i2 = a + 1;  // node index within the two cells, 0..2k+2
      double v = 0.0;
      if (q < nd && i2 <= k + 1) v += t.D[q * nc + i2];
      if (q >= nd && i2 >= nd) v += t.D[(q - nd) * nc + (i2 - nd)];
      P.DL[q * npc + a] = v;
    }
  P.W.assign(npd, 0.0);
  for (int j = 0; j < npd; ++j) P.W[j] = t.S[j % nd];
  return P;
}

template <typename T>
void fill_patch_tables(const PatchTables1D& p, PatchTables<T>* out) {
  *out = PatchTables<T>{};
  const int k = p.k, npc = 2 * k + 1, npd = 2 * k + 2;
  constexpr int RS = kRowStride;
  for (int i = 0; i < npc; ++i)
    for (int j = 0; j < npc; ++j) out->SC[i * RS + j] = (T)p.SC[i * npc + j];
  for (int i = 0; i < npc; ++i) out->LC[i] = (T)p.LC[i];
  out->LC[npc] = T(1);  // padded node (its coefficients are zero)
  for (int t = 0; t < 4; ++t) {
    for (int i = 0; i < npd; ++i)
      for (int j = 0; j < npd; ++j) out->SD[t][i * RS + j] = (T)p.SD[t][i * npd + j];
    for (int i = 0; i < npd; ++i) out->LD[t][i] = (T)p.LD[t][i];
  }
  for (int i = 0; i < npd * npc; ++i) out->DL[i] = (T)p.DL[i];
  for (int i = 0; i < npd; ++i) out->W[i] = (T)p.W[i];
  // B_c (S_c (x) S_d1 (x) S_d2) = (DL SC) (x) (W SD) (x) (W SD): the Schur operator in the eigenbasis
  for (int q = 0; q < npd; ++q)
    for (int j = 0; j < npc; ++j) {
      double s = 0.0;
      for (int a = 0; a < npc; ++a) s += p.DL[q * npc + a] * p.SC[a * npc + j];
      out->EC[q * RS + j] = (T)s;
    }
  for (int t = 0; t < 4; ++t)
    for (int q = 0; q < npd; ++q)
      for (int j = 0; j < npd; ++j) out->FM[t][q * RS + j] = (T)(p.W[q] * p.SD[t][q * npd + j]);
  out->inv_nu = (T)(1.0 / p.nu);
  out->eo_c = p.eo_c ? 1 : 0;
  for (int t = 0; t < 4; ++t) out->eo_d[t] = p.eo_d[t] ? 1 : 0;
}

template void fill_patch_tables<double>(const PatchTables1D&, PatchTables<double>*);
template void fill_patch_tables<float>(const PatchTables1D&, PatchTables<float>*);

std::vector<double> build_transfer_tables(int k) {
  // PC[ch][a][b] = l^C_b((ch + zC_a)/2), PD[ch][a][b] = l^D_b((ch + zD_a)/2)
  const int nc = k + 2, nd = k + 1;
  std::vector<double> zC, wC, zD, wD;
  gauss_lobatto(nc, zC, wC);
  gauss_legendre(nd, zD, wD);
  std::vector<double> out;
  for (int ch = 0; ch < 2; ++ch) {
    std::vector<double> t(nc), V, Dv;
    for (int a = 0; a < nc; ++a) t[a] = 0.5 * (ch + zC[a]);
    lagrange(zC, t, V, Dv);  // V[b*nc + a] = l_b(t_a)
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < nc; ++b) out.push_back(V[b * nc + a]);
  }
  for (int ch = 0; ch < 2; ++ch) {
    std::vector<double> t(nd), V, Dv;
    for (int a = 0; a < nd; ++a) t[a] = 0.5 * (ch + zD[a]);
    lagrange(zD, t, V, Dv);
    for (int a = 0; a < nd; ++a)
      for (int b = 0; b < nd; ++b) out.push_back(V[b * nd + a]);
  }
  return out;
}

}  // namespace stk
