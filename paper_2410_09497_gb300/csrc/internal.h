// Internal declarations of libstokesmg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "stokesmg.h"

namespace stk {

constexpr int kMaxDegree = 5;
constexpr int kMaxC = kMaxDegree + 2;  // nodes of a cell in the continuous direction
constexpr int kMaxD = kMaxDegree + 1;  // nodes of a cell in a discontinuous direction

// 1D cell matrices of one level (Sec. 2.3 and Sec. 3.2), row-major, in the
// precision of the kernel that reads them.  Layout is fixed so a kernel can
// copy the whole struct into shared memory.
//   KC[i][j]  nu * int phi_i' phi_j'        continuous (Gauss-Lobatto) basis, (k+2)^2
//   MC[i][j]  nu * int phi_i  phi_j         continuous basis, (k+2)^2
//   D[q][a]   int psi_q phi_a'              pressure (Gauss) x continuous derivative, (k+1)(k+2)
//   LS[t][b][c] nu * 1D interior-penalty block of a cell with itself:
//             t = 0 interior cell, 1 first cell (face x = 0), 2 last cell (x = 1)
//   LLO[b][c] nu * coupling of a cell row to its lower neighbour's column
//   LHI[b][c] nu * coupling of a cell row to its upper neighbour's column
//   S[a]      h * Gauss weight a: the diagonal discontinuous mass matrix
template <typename T>
struct CellTables {
  T KC[kMaxC * kMaxC];
  T MC[kMaxC * kMaxC];
  T D[kMaxD * kMaxC];
  T LS[3][kMaxD * kMaxD];
  T LLO[kMaxD * kMaxD];
  T LHI[kMaxD * kMaxD];
  T S[kMaxD];
};

// Host-side double precision 1D data of one (k, h, nu, penalty) combination.
struct Tables1D {
  int k = 0;
  double h = 0, nu = 0, gamma = 0;
  std::vector<double> zC, zD, wD;  // nodes / Gauss weights on [0, 1]
  std::vector<double> KC, MC, D;   // as CellTables, double
  std::vector<double> LS[3], LLO, LHI;
  std::vector<double> S;
};

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w);
// values V[i*np+q] = l_i(t_q) and derivatives Dv[i*np+q] = l_i'(t_q)
void lagrange(const std::vector<double>& z, const std::vector<double>& t, std::vector<double>& V,
              std::vector<double>& Dv);
Tables1D build_tables(int k, double h, double nu, double penalty_factor);

template <typename T>
void fill_cell_tables(const Tables1D& t, CellTables<T>* out);

struct Level {
  int n = 0, m = 0;
  double h = 0;
  int64_t nvel = 0, npress = 0, ntotal = 0;
  Tables1D t1d;
  CellTables<double>* tab64 = nullptr;  // device
  CellTables<float>* tab32 = nullptr;   // device
};

}  // namespace stk

struct stk_problem {
  int k = 0;
  double nu = 1.0;
  stk_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<stk::Level> levels;  // [0] coarsest
  std::string err;
};

namespace stk {

// Launchers (apply.cu).  y = alpha * A x + (b ? b : 0); returns a cudaError_t.
// stages: bit 0 = velocity rows, bit 1 = pressure rows (3 = the whole operator).
cudaError_t launch_apply(const stk_problem* P, int level, int dtype, const void* x, const void* b, void* y,
                         double alpha, int stages = 3);

}  // namespace stk
