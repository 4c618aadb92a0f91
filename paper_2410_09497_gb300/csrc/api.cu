// C ABI of libstokesmg: setup, teardown, layout queries and the operator
// entry points.  Every function returns a status code and never throws.
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace {

thread_local std::string g_setup_error;

int fail(stk_problem* P, int code, const std::string& msg) {
  if (P)
    P->err = msg;
  else
    g_setup_error = msg;
  return code;
}

int cuda_fail(stk_problem* P, cudaError_t e, const char* what) {
  return fail(P, STK_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_level(stk_problem* P, int level) {
  if (!P) return STK_EINVAL;
  if (level < 0 || level >= (int)P->levels.size())
    return fail(P, STK_EINVAL, "level out of range");
  return STK_OK;
}

int check_vec(stk_problem* P, const void* v, const char* name) {
  if (!v) return fail(P, STK_EINVAL, std::string(name) + " is NULL");
  if (!aligned16(v)) return fail(P, STK_EINVAL, std::string(name) + " is not 16-byte aligned");
  return STK_OK;
}

void free_level(stk::Level& L) {
  if (L.tab64) cudaFree(L.tab64);
  if (L.tab32) cudaFree(L.tab32);
  L.tab64 = nullptr;
  L.tab32 = nullptr;
}

}  // namespace

extern "C" {

int stk_default_options(stk_options* opt) {
  if (!opt) return STK_EINVAL;
  opt->precision = STK_PREC_FP64;
  opt->gmres_restart = 20;
  opt->max_iter = 200;
  opt->local_cg_mode = STK_CG_FIXED;
  opt->local_cg_iters = 15;
  opt->local_cg_tol = 1e-8;
  opt->penalty_factor = 1.0;
  opt->stream = nullptr;
  return STK_OK;
}

int stk_setup(int n, int k, double nu, const stk_options* opt, stk_problem** out) {
  if (!out) return fail(nullptr, STK_EINVAL, "out is NULL");
  *out = nullptr;
  if (k < 1 || k > stk::kMaxDegree) return fail(nullptr, STK_EINVAL, "degree k must be in 1..5");
  if (!(nu > 0.0)) return fail(nullptr, STK_EINVAL, "viscosity must be positive");
  std::vector<int> sizes;
  {
    int s = n;
    if (s < 2) return fail(nullptr, STK_EINVAL, "n must be at least 2");
    sizes.push_back(s);
    while (s % 2 == 0 && s > 3) {
      s /= 2;
      sizes.push_back(s);
    }
    if (s != 2 && s != 3) return fail(nullptr, STK_EINVAL, "n must be 2 or 3 times a power of two");
    if ((int64_t)n * (k + 1) > 1200) return fail(nullptr, STK_EINVAL, "mesh too large");
  }
  stk_problem* P = new (std::nothrow) stk_problem();
  if (!P) return fail(nullptr, STK_ENOMEM, "host allocation failed");
  P->k = k;
  P->nu = nu;
  if (opt)
    P->opt = *opt;
  else
    stk_default_options(&P->opt);
  if (!(P->opt.penalty_factor > 0.0)) {
    delete P;
    return fail(nullptr, STK_EINVAL, "penalty_factor must be positive");
  }
  P->stream = reinterpret_cast<cudaStream_t>(P->opt.stream);
  P->levels.resize(sizes.size());
  for (size_t i = 0; i < sizes.size(); ++i) {
    stk::Level& L = P->levels[sizes.size() - 1 - i];
    L.n = sizes[i];
    L.m = L.n * (k + 1);
    L.h = 1.0 / L.n;
    L.nvel = (int64_t)(L.m + 1) * L.m * L.m;
    L.npress = (int64_t)L.m * L.m * L.m;
    L.ntotal = 3 * L.nvel + L.npress;
    L.t1d = stk::build_tables(k, L.h, nu, P->opt.penalty_factor);
    stk::CellTables<double> h64;
    stk::CellTables<float> h32;
    stk::fill_cell_tables(L.t1d, &h64);
    stk::fill_cell_tables(L.t1d, &h32);
    cudaError_t e = cudaMalloc(&L.tab64, sizeof(h64));
    if (e == cudaSuccess) e = cudaMalloc(&L.tab32, sizeof(h32));
    if (e == cudaSuccess) e = cudaMemcpy(L.tab64, &h64, sizeof(h64), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.tab32, &h32, sizeof(h32), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      std::string msg = std::string("setup: ") + cudaGetErrorString(e);
      for (auto& l : P->levels) free_level(l);
      delete P;
      return fail(nullptr, e == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA, msg);
    }
  }
  *out = P;
  return STK_OK;
}

int stk_destroy(stk_problem* P) {
  if (!P) return STK_OK;
  cudaStreamSynchronize(P->stream);
  for (auto& L : P->levels) free_level(L);
  delete P;
  return STK_OK;
}

const char* stk_last_error(const stk_problem* P) { return P ? P->err.c_str() : g_setup_error.c_str(); }

int stk_num_levels(const stk_problem* P, int* nlevels) {
  if (!P || !nlevels) return STK_EINVAL;
  *nlevels = (int)P->levels.size();
  return STK_OK;
}

int stk_layout(const stk_problem* P, int level, int* n_cells, int64_t* n_vel_component, int64_t* n_pressure,
               int64_t* n_total) {
  if (!P) return STK_EINVAL;
  if (level < 0 || level >= (int)P->levels.size()) return STK_EINVAL;
  const stk::Level& L = P->levels[level];
  if (n_cells) *n_cells = L.n;
  if (n_vel_component) *n_vel_component = L.nvel;
  if (n_pressure) *n_pressure = L.npress;
  if (n_total) *n_total = L.ntotal;
  return STK_OK;
}

int stk_apply(stk_problem* P, int level, int dtype, const void* x, void* y) {
  int rc = check_level(P, level);
  if (rc) return rc;
  if (dtype != STK_F64 && dtype != STK_F32) return fail(P, STK_EINVAL, "dtype must be STK_F64 or STK_F32");
  if ((rc = check_vec(P, x, "x")) || (rc = check_vec(P, y, "y"))) return rc;
  if (x == y) return fail(P, STK_EINVAL, "x and y must not alias");
  cudaError_t e = stk::launch_apply(P, level, dtype, x, nullptr, y, 1.0);
  if (e != cudaSuccess) return cuda_fail(P, e, "apply");
  return STK_OK;
}

int stk_apply_stage(stk_problem* P, int level, int dtype, int stage, const void* x, void* y) {
  int rc = check_level(P, level);
  if (rc) return rc;
  if (dtype != STK_F64 && dtype != STK_F32) return fail(P, STK_EINVAL, "dtype must be STK_F64 or STK_F32");
  if (stage != 0 && stage != 1) return fail(P, STK_EINVAL, "stage must be 0 (velocity rows) or 1 (pressure rows)");
  if ((rc = check_vec(P, x, "x")) || (rc = check_vec(P, y, "y"))) return rc;
  if (x == y) return fail(P, STK_EINVAL, "x and y must not alias");
  cudaError_t e = stk::launch_apply(P, level, dtype, x, nullptr, y, 1.0, stage == 0 ? 1 : 2);
  if (e != cudaSuccess) return cuda_fail(P, e, "apply_stage");
  return STK_OK;
}

int stk_residual(stk_problem* P, int level, int dtype, const void* x, const void* b, void* r) {
  int rc = check_level(P, level);
  if (rc) return rc;
  if (dtype != STK_F64 && dtype != STK_F32) return fail(P, STK_EINVAL, "dtype must be STK_F64 or STK_F32");
  if ((rc = check_vec(P, x, "x")) || (rc = check_vec(P, b, "b")) || (rc = check_vec(P, r, "r"))) return rc;
  if (x == r) return fail(P, STK_EINVAL, "x and r must not alias");
  cudaError_t e = stk::launch_apply(P, level, dtype, x, b, r, -1.0);
  if (e != cudaSuccess) return cuda_fail(P, e, "residual");
  return STK_OK;
}

}  // extern "C"
