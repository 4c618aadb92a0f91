// Host-side 1D tables (setup only): quadrature rules, Lagrange bases and the
// 1D cell matrices whose Kronecker sums form the Stokes operator on a
// Cartesian mesh (Sec. 2.3, the Kronecker form noted after Fig. 1) and the
// patch matrices of the local solver (Sec. 3.2, eq. `block_A` and eq. `b`).
#include <cmath>
#include <stdexcept>

#include "internal.h"

namespace stk {

// Legendre polynomial P_n and its derivative at x by the three-term recurrence.
static void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = (std::fabs(x) < 1.0) ? n * (x * p1 - p0) / (x * x - 1.0) : 0.5 * n * (n + 1) * std::pow(x, n + 1);
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on P_n from the Chebyshev-like initial guesses.
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double r = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, r, p, dp);
      double dr = p / dp;
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    double p, dp;
    legendre(n, r, p, dp);
    // map [-1, 1] -> [0, 1]; nodes ascending
    x[n - 1 - i] = 0.5 * (r + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - r * r) * dp * dp);  // 2/((1-r^2)P'^2) halved
  }
}

void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w) {
  // End points plus the roots of P'_N, N = n - 1, by Newton with P''_N from
  // the Legendre equation; weights 2 / (N (N+1) P_N^2), halved for [0, 1].
  const int N = n - 1;
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  std::vector<double> r(n);
  r[0] = -1.0;
  r[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double t = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(N, t, p, dp);
      double d2p = (2.0 * t * dp - N * (N + 1.0) * p) / (1.0 - t * t);
      double dt = dp / d2p;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    r[i] = t;
  }
  for (int i = 0; i <= N; ++i) {
    double p, dp;
    legendre(N, r[i], p, dp);
    x[i] = 0.5 * (r[i] + 1.0);
    w[i] = 1.0 / (N * (N + 1.0) * p * p);
  }
}

void lagrange(const std::vector<double>& z, const std::vector<double>& t, std::vector<double>& V,
              std::vector<double>& Dv) {
  const int p = (int)z.size(), nq = (int)t.size();
  V.assign(p * nq, 0.0);
  Dv.assign(p * nq, 0.0);
  for (int i = 0; i < p; ++i) {
    double denom = 1.0;
    for (int j = 0; j < p; ++j)
      if (j != i) denom *= z[i] - z[j];
    for (int q = 0; q < nq; ++q) {
      double num = 1.0;
      for (int j = 0; j < p; ++j)
        if (j != i) num *= t[q] - z[j];
      V[i * nq + q] = num / denom;
      double d = 0.0;
      for (int l = 0; l < p; ++l) {
        if (l == i) continue;
        double prod = 1.0;
        for (int j = 0; j < p; ++j)
          if (j != i && j != l) prod *= t[q] - z[j];
        d += prod;
      }
      Dv[i * nq + q] = d / denom;
    }
  }
}

Tables1D build_tables(int k, double h, double nu, double penalty_factor) {
  Tables1D T;
  T.k = k;
  T.h = h;
  T.nu = nu;
  T.gamma = penalty_factor * (k + 1) * (k + 2) / h;
  const int nc = k + 2, nd = k + 1;
  std::vector<double> wC;
  gauss_lobatto(nc, T.zC, wC);
  gauss_legendre(nd, T.zD, T.wD);
  // exact integration: (k+3)-point Gauss rule covers degree 2k+5
  std::vector<double> xq, wq;
  gauss_legendre(k + 3, xq, wq);
  const int nq = k + 3;
  std::vector<double> VC, DC, VD, DD;
  lagrange(T.zC, xq, VC, DC);
  lagrange(T.zD, xq, VD, DD);
  T.KC.assign(nc * nc, 0.0);
  T.MC.assign(nc * nc, 0.0);
  T.D.assign(nd * nc, 0.0);
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) {
      double s1 = 0, s2 = 0;
      for (int q = 0; q < nq; ++q) {
        s1 += wq[q] * DC[i * nq + q] * DC[j * nq + q];
        s2 += wq[q] * VC[i * nq + q] * VC[j * nq + q];
      }
      T.KC[i * nc + j] = nu * s1 / h;
      T.MC[i * nc + j] = s2 * h;  // plain mass: it multiplies the nu-scaled 1D penalty operator
    }
  for (int a = 0; a < nd; ++a)
    for (int i = 0; i < nc; ++i) {
      double s = 0;
      for (int q = 0; q < nq; ++q) s += wq[q] * VD[a * nq + q] * DC[i * nq + q];
      T.D[a * nc + i] = s;  // int psi_a d/dx phi_i dx = int psi_a phi_i'(xi) dxi
    }
  // 1D interior-penalty operator of a discontinuous direction: broken
  // stiffness plus, per face point, gamma [[u]][[v]] - {{u'}}[[v]] - [[u]]{{v'}}
  // with [[w]] = w^- - w^+, n = +1 from the lower to the upper cell; on the
  // boundary 2 gamma u v - d_n u v - u d_n v (eq. `bilinear` restricted to a line).
  std::vector<double> e0, e1, d0, d1, Vt, Dt;
  lagrange(T.zD, std::vector<double>{0.0, 1.0}, Vt, Dt);
  e0.resize(nd);
  e1.resize(nd);
  d0.resize(nd);
  d1.resize(nd);
  for (int b = 0; b < nd; ++b) {
    e0[b] = Vt[b * 2 + 0];
    e1[b] = Vt[b * 2 + 1];
    d0[b] = Dt[b * 2 + 0] / h;  // physical derivative at the cell's lower end
    d1[b] = Dt[b * 2 + 1] / h;  // ... at its upper end
  }
  const double g = T.gamma;
  std::vector<double> K(nd * nd), lowface(nd * nd), highface(nd * nd), lowbnd(nd * nd), highbnd(nd * nd);
  for (int b = 0; b < nd; ++b)
    for (int c = 0; c < nd; ++c) {
      double s = 0;
      for (int q = 0; q < nq; ++q) s += wq[q] * DD[b * nq + q] * DD[c * nq + q];
      K[b * nd + c] = s / h;
      // cell is the upper (+) side of its lower face: [[u]] = -u, {{u'}} = u'/2
      lowface[b * nd + c] = g * e0[c] * e0[b] + 0.5 * d0[c] * e0[b] + 0.5 * e0[c] * d0[b];
      // cell is the lower (-) side of its upper face: [[u]] = u, {{u'}} = u'/2
      highface[b * nd + c] = g * e1[c] * e1[b] - 0.5 * d1[c] * e1[b] - 0.5 * e1[c] * d1[b];
      // boundary x = 0, outward normal -1: d_n u = -u'
      lowbnd[b * nd + c] = 2.0 * g * e0[c] * e0[b] + d0[c] * e0[b] + e0[c] * d0[b];
      // boundary x = 1, outward normal +1
      highbnd[b * nd + c] = 2.0 * g * e1[c] * e1[b] - d1[c] * e1[b] - e1[c] * d1[b];
    }
  for (int t = 0; t < 3; ++t) T.LS[t].assign(nd * nd, 0.0);
  T.LLO.assign(nd * nd, 0.0);
  T.LHI.assign(nd * nd, 0.0);
  for (int b = 0; b < nd; ++b)
    for (int c = 0; c < nd; ++c) {
      const int i = b * nd + c;
      T.LS[0][i] = nu * (K[i] + lowface[i] + highface[i]);
      T.LS[1][i] = nu * (K[i] + lowbnd[i] + highface[i]);
      T.LS[2][i] = nu * (K[i] + lowface[i] + highbnd[i]);
      // row b of this cell (+ side), column c of the lower cell (- side)
      T.LLO[i] = nu * (-g * e1[c] * e0[b] + 0.5 * d1[c] * e0[b] - 0.5 * e1[c] * d0[b]);
      // row b of this cell (- side), column c of the upper cell (+ side)
      T.LHI[i] = nu * (-g * e0[c] * e1[b] - 0.5 * d0[c] * e1[b] + 0.5 * e0[c] * d1[b]);
    }
  T.S.assign(nd, 0.0);
  for (int a = 0; a < nd; ++a) T.S[a] = T.wD[a] * h;
  return T;
}

template <typename T>
void fill_cell_tables(const Tables1D& t, CellTables<T>* out) {
  const int nc = t.k + 2, nd = t.k + 1;
  *out = CellTables<T>{};
  for (int i = 0; i < nc * nc; ++i) {
    out->KC[i] = (T)t.KC[i];
    out->MC[i] = (T)t.MC[i];
  }
  for (int i = 0; i < nd * nc; ++i) out->D[i] = (T)t.D[i];
  for (int s = 0; s < 3; ++s)
    for (int i = 0; i < nd * nd; ++i) out->LS[s][i] = (T)t.LS[s][i];
  for (int i = 0; i < nd * nd; ++i) {
    out->LLO[i] = (T)t.LLO[i];
    out->LHI[i] = (T)t.LHI[i];
  }
  for (int a = 0; a < nd; ++a) out->S[a] = (T)t.S[a];
}

template void fill_cell_tables<double>(const Tables1D&, CellTables<double>*);
template void fill_cell_tables<float>(const Tables1D&, CellTables<float>*);

// Even-odd contraction tables (see ContractTables): built from the dense
// blocks in double precision; the reflection symmetries of KC, MC and D hold
// to rounding, so this is the same linear map.
template <typename T>
void fill_contract_tables(const Tables1D& t, ContractTables<T>* out) {
  const int nc = t.k + 2, nd = t.k + 1;
  const int P = nc / 2, Q = nd / 2;
  const bool cenc = nc % 2 == 1, cend = nd % 2 == 1;
  *out = ContractTables<T>{};
  auto KC = [&](int i, int a) { return t.KC[i * nc + a]; };
  auto MC = [&](int i, int a) { return t.MC[i * nc + a]; };
  auto D = [&](int q, int a) { return t.D[q * nc + a]; };
  for (int i = 0; i < P + (cenc ? 1 : 0); ++i) {
    const bool centre = i == P;
    for (int a = 0; a < P + (cenc ? 1 : 0); ++a) {
      double ek, em;
      if (a == P) {  // centre input
        ek = KC(i, P);
        em = MC(i, P);
      } else if (centre) {
        ek = KC(P, a);
        em = MC(P, a);
      } else {
        ek = 0.5 * (KC(i, a) + KC(i, nc - 1 - a));
        em = 0.5 * (MC(i, a) + MC(i, nc - 1 - a));
      }
      out->EK[i * kMaxC + a] = (T)ek;
      out->EM[i * kMaxC + a] = (T)em;
    }
    for (int q = 0; q < Q; ++q)
      out->ED[i * kMaxD + q] = (T)(centre ? D(q, P) : 0.5 * (D(q, i) - D(nd - 1 - q, i)));
    if (centre) continue;
    for (int a = 0; a < P; ++a) {
      out->OK[i * kMaxC + a] = (T)(0.5 * (KC(i, a) - KC(i, nc - 1 - a)));
      out->OM[i * kMaxC + a] = (T)(0.5 * (MC(i, a) - MC(i, nc - 1 - a)));
    }
    for (int q = 0; q < Q + (cend ? 1 : 0); ++q)
      out->OD[i * kMaxD + q] = (T)(q == Q ? D(Q, i) : 0.5 * (D(q, i) + D(nd - 1 - q, i)));
  }
}

template void fill_contract_tables<double>(const Tables1D&, ContractTables<double>*);
template void fill_contract_tables<float>(const Tables1D&, ContractTables<float>*);

}  // namespace stk
