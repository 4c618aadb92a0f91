// C ABI of libstokesmg: setup, teardown, layout queries and the operator
// entry points.  Every function returns a status code and never throws.
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include <cublas_v2.h>

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
  if (L.ptab64) cudaFree(L.ptab64);
  if (L.ptab32) cudaFree(L.ptab32);
  L.tab64 = nullptr;
  L.tab32 = nullptr;
  L.ptab64 = nullptr;
  L.ptab32 = nullptr;
  for (void* p : {(void*)L.dirM64, (void*)L.dirM32, (void*)L.dirtab64, (void*)L.dirtab32})
    if (p) cudaFree(p);
  L.dirM64 = nullptr;
  L.dirM32 = nullptr;
  L.dirtab64 = nullptr;
  L.dirtab32 = nullptr;
  L.dir_ready = false;
  if (L.flat64) cudaFree(L.flat64);
  if (L.flat32) cudaFree(L.flat32);
  L.flat64 = nullptr;
  L.flat32 = nullptr;
  if (L.gemmR) cudaFree(L.gemmR);
  if (L.gemmP) cudaFree(L.gemmP);
  L.gemmR = nullptr;
  L.gemmP = nullptr;
  L.gemm_cap = 0;
}

void free_problem(stk_problem* P) {
  for (auto& L : P->levels) free_level(L);
  for (int d = 0; d < 2; ++d)
    for (auto* v : {&P->mg[d].r, &P->mg[d].b, &P->mg[d].x})
      for (void* p : *v)
        if (p) cudaFree(p);
  stk::KrylovWork& K = P->kry;
  if (K.solve_graph) cudaGraphExecDestroy(K.solve_graph);
  for (double* d : {K.V, K.Z, K.w, K.zbuf, K.partial, K.h})
    if (d) cudaFree(d);
  if (K.state) cudaFree(K.state);
  if (K.state_host) cudaFreeHost(K.state_host);
  for (cudaStream_t s : K.side)
    if (s) cudaStreamDestroy(s);
  if (P->blas) cublasDestroy(static_cast<cublasHandle_t>(P->blas));
  if (P->blas_ws) cudaFree(P->blas_ws);
  if (P->xfer64) cudaFree(P->xfer64);
  if (P->xfer32) cudaFree(P->xfer32);
  if (P->pmean_w) cudaFree(P->pmean_w);
  if (P->coarse_inv) cudaFree(P->coarse_inv);
  for (double* c : P->coarse3)
    if (c) cudaFree(c);
  for (int d = 0; d < 2; ++d)
    if (P->mg[d].graph) cudaGraphExecDestroy(P->mg[d].graph);
  delete P;
}

int check_dtype(stk_problem* P, int dtype) {
  if (dtype != STK_F64 && dtype != STK_F32) return fail(P, STK_EINVAL, "dtype must be STK_F64 or STK_F32");
  return STK_OK;
}

int check_3d(stk_problem* P, const char* what) {
  if (P->dim != 3) return fail(P, STK_EINVAL, std::string(what) + " is not available for two-dimensional problems");
  return STK_OK;
}

// x[i] = a deterministic value in [-1, 1) (a hash of i and the seed): the
// autotuner's smoothing input, nonzero so that no local solve stops early
__global__ void fill_pattern_kernel(void* x, int64_t n, int f32, unsigned seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + seed;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double v = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    if (f32)
      static_cast<float*>(x)[i] = (float)v;
    else
      static_cast<double*>(x)[i] = v;
  }
}

void fill_pattern(void* x, int64_t n, int dtype, unsigned seed, cudaStream_t s) {
  fill_pattern_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1216), 256, 0, s>>>(x, n, dtype == STK_F32, seed);
}

int check_mg(stk_problem* P) {
  if (P->levels[0].n != 2 && P->levels[0].n != 3)
    return fail(P, STK_ESTATE, "the V-cycle needs a hierarchy that coarsens to 2 or 3 cells per side");
  return STK_OK;
}

int status_of(stk_problem* P, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return STK_OK;
  if (e == cudaErrorMemoryAllocation) return fail(P, STK_ENOMEM, std::string(what) + ": out of device memory");
  return cuda_fail(P, e, what);
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
  opt->use_graphs = 1;
  opt->fused_smoother = 0;
  opt->direct_gemm = 2;
  return STK_OK;
}

int stk_cell_tables(int n, int k, double nu, double penalty_factor, double* out) {
  if (k < 1 || k > stk::kMaxDegree) return fail(nullptr, STK_EINVAL, "cell_tables: degree k must be in 1..5");
  if (n < 2) return fail(nullptr, STK_EINVAL, "cell_tables: n must be at least 2");
  if (!(nu > 0.0) || !(penalty_factor > 0.0))
    return fail(nullptr, STK_EINVAL, "cell_tables: viscosity and penalty factor must be positive");
  if (!out) return fail(nullptr, STK_EINVAL, "cell_tables: NULL output pointer");
  try {
    const stk::Tables1D t = stk::build_tables(k, 1.0 / n, nu, penalty_factor);
    for (const std::vector<double>* v : {&t.KC, &t.MC, &t.D, &t.LS[0], &t.LS[1], &t.LS[2], &t.LLO, &t.LHI, &t.S})
      out = std::copy(v->begin(), v->end(), out);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, STK_ENOMEM, "cell_tables: host allocation failed");
  }
  return STK_OK;
}

int stk_transfer_tables(int k, double* out) {
  if (k < 1 || k > stk::kMaxDegree) return fail(nullptr, STK_EINVAL, "transfer_tables: degree k must be in 1..5");
  if (!out) return fail(nullptr, STK_EINVAL, "transfer_tables: NULL output pointer");
  try {
    const std::vector<double> t = stk::build_transfer_tables(k);
    std::copy(t.begin(), t.end(), out);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, STK_ENOMEM, "transfer_tables: host allocation failed");
  }
  return STK_OK;
}

int stk_patch_eigen(int n, int k, double nu, double penalty_factor, int direction, double* S, double* lambda,
                    int* dim, int* even_odd) {
  if (k < 1 || k > stk::kMaxDegree) return fail(nullptr, STK_EINVAL, "patch_eigen: degree k must be in 1..5");
  if (n < 2) return fail(nullptr, STK_EINVAL, "patch_eigen: n must be at least 2");
  if (!(nu > 0.0) || !(penalty_factor > 0.0))
    return fail(nullptr, STK_EINVAL, "patch_eigen: viscosity and penalty factor must be positive");
  if (direction < 0 || direction > 4) return fail(nullptr, STK_EINVAL, "patch_eigen: direction must be in 0..4");
  if (!S || !lambda || !dim || !even_odd) return fail(nullptr, STK_EINVAL, "patch_eigen: NULL output pointer");
  try {
    const stk::PatchTables1D p = stk::build_patch_tables(stk::build_tables(k, 1.0 / n, nu, penalty_factor));
    const std::vector<double>& vs = direction == 0 ? p.SC : p.SD[direction - 1];
    const std::vector<double>& vl = direction == 0 ? p.LC : p.LD[direction - 1];
    std::copy(vs.begin(), vs.end(), S);
    std::copy(vl.begin(), vl.end(), lambda);
    *dim = (int)vl.size();
    *even_odd = (direction == 0 ? p.eo_c : p.eo_d[direction - 1]) ? 1 : 0;
  } catch (const std::bad_alloc&) {
    return fail(nullptr, STK_ENOMEM, "patch_eigen: host allocation failed");
  }
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
  if (P->opt.gmres_restart < 1 || P->opt.gmres_restart > 60 || P->opt.max_iter < 1 || P->opt.local_cg_iters < 0 ||
      (P->opt.precision != STK_PREC_FP64 && P->opt.precision != STK_PREC_MIXED) ||
      (P->opt.local_cg_mode != STK_CG_FIXED && P->opt.local_cg_mode != STK_CG_TOL &&
       P->opt.local_cg_mode != STK_LOCAL_DIRECT)) {
    delete P;
    return fail(nullptr, STK_EINVAL, "invalid options (restart in 1..60, max_iter >= 1, known modes)");
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
    L.htab64 = h64;
    L.htab32 = h32;
    stk::fill_contract_tables(L.t1d, &L.hce64);
    stk::fill_contract_tables(L.t1d, &L.hce32);
    const stk::PatchTables1D pt = stk::build_patch_tables(L.t1d);
    L.eo_interior = pt.eo_c && pt.eo_d[0];
    stk::PatchTables<double> p64;
    stk::PatchTables<float> p32;
    stk::fill_patch_tables(pt, &p64);
    stk::fill_patch_tables(pt, &p32);
    L.hptab64 = p64;
    L.hptab32 = p32;
    cudaError_t e = stk::dev_alloc(&L.tab64, sizeof(h64));
    if (e == cudaSuccess) e = stk::dev_alloc(&L.tab32, sizeof(h32));
    if (e == cudaSuccess) e = stk::dev_alloc(&L.ptab64, sizeof(p64));
    if (e == cudaSuccess) e = stk::dev_alloc(&L.ptab32, sizeof(p32));
    if (e == cudaSuccess) e = cudaMemcpy(L.tab64, &h64, sizeof(h64), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.tab32, &h32, sizeof(h32), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.ptab64, &p64, sizeof(p64), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.ptab32, &p32, sizeof(p32), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      std::string msg = std::string("setup: ") + cudaGetErrorString(e);
      free_problem(P);
      return fail(nullptr, e == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA, msg);
    }
  }
  {
    const std::vector<double> xt = stk::build_transfer_tables(k);
    std::vector<float> xt32(xt.begin(), xt.end());
    const std::vector<double>& S = P->levels.back().t1d.S;
    cudaError_t e = stk::dev_alloc(&P->xfer64, sizeof(double) * xt.size());
    if (e == cudaSuccess) e = stk::dev_alloc(&P->xfer32, sizeof(float) * xt.size());
    if (e == cudaSuccess) e = stk::dev_alloc(&P->pmean_w, sizeof(double) * S.size());
    if (e == cudaSuccess) e = cudaMemcpy(P->xfer64, xt.data(), sizeof(double) * xt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->xfer32, xt32.data(), sizeof(float) * xt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->pmean_w, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      std::string msg = std::string("setup: ") + cudaGetErrorString(e);
      free_problem(P);
      return fail(nullptr, e == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA, msg);
    }
  }
  *out = P;
  return STK_OK;
}

int stk_setup_planar(int n, int k, double nu, const stk_options* opt, stk_problem** out) {
  if (!out) return fail(nullptr, STK_EINVAL, "out is NULL");
  *out = nullptr;
  if (k < 1 || k > stk::kMaxPlanarDegree) return fail(nullptr, STK_EINVAL, "degree k must be in 1..8");
  if (!(nu > 0.0)) return fail(nullptr, STK_EINVAL, "viscosity must be positive");
  if (n < 2 || (n & (n - 1)) != 0) return fail(nullptr, STK_EINVAL, "n must be a power of two (n >= 2)");
  if ((int64_t)n * (k + 1) > 8192) return fail(nullptr, STK_EINVAL, "mesh too large");
  stk_problem* P = new (std::nothrow) stk_problem();
  if (!P) return fail(nullptr, STK_ENOMEM, "host allocation failed");
  P->dim = 2;
  P->k = k;
  P->nu = nu;
  if (opt)
    P->opt = *opt;
  else
    stk_default_options(&P->opt);
  if (!(P->opt.penalty_factor > 0.0) || P->opt.gmres_restart < 1 || P->opt.gmres_restart > 60 ||
      P->opt.max_iter < 1 || (P->opt.precision != STK_PREC_FP64 && P->opt.precision != STK_PREC_MIXED)) {
    delete P;
    return fail(nullptr, STK_EINVAL, "invalid options (penalty > 0, restart in 1..60, max_iter >= 1, known precision)");
  }
  P->stream = reinterpret_cast<cudaStream_t>(P->opt.stream);
  std::vector<int> sizes;
  for (int s2 = n; s2 >= 2; s2 /= 2) sizes.push_back(s2);
  P->levels.resize(sizes.size());
  try {
    for (size_t i = 0; i < sizes.size(); ++i) {
      stk::Level& L = P->levels[sizes.size() - 1 - i];
      L.n = sizes[i];
      L.m = L.n * (k + 1);
      L.h = 1.0 / L.n;
      L.nvel = (int64_t)(L.m + 1) * L.m;
      L.npress = (int64_t)L.m * L.m;
      L.ntotal = 2 * L.nvel + L.npress;
      L.t1d = stk::build_tables(k, L.h, nu, P->opt.penalty_factor);
    }
  } catch (const std::bad_alloc&) {
    delete P;
    return fail(nullptr, STK_ENOMEM, "host allocation failed");
  }
  cudaError_t e = stk::setup_planar(P);
  if (e == cudaSuccess) {
    const std::vector<double> xt = stk::build_transfer_tables(k);
    std::vector<float> xt32(xt.begin(), xt.end());
    const std::vector<double>& S = P->levels.back().t1d.S;
    e = stk::dev_alloc(&P->xfer64, sizeof(double) * xt.size());
    if (e == cudaSuccess) e = stk::dev_alloc(&P->xfer32, sizeof(float) * xt.size());
    if (e == cudaSuccess) e = stk::dev_alloc(&P->pmean_w, sizeof(double) * S.size());
    if (e == cudaSuccess) e = cudaMemcpy(P->xfer64, xt.data(), sizeof(double) * xt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->xfer32, xt32.data(), sizeof(float) * xt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->pmean_w, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    std::string msg = std::string("setup_planar: ") + cudaGetErrorString(e);
    free_problem(P);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA, msg);
  }
  *out = P;
  return STK_OK;
}

int stk_planar_errors(stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq,
                      const double* p_amp, const double* x, double* err_u, double* err_p) {
  if (!P) return STK_EINVAL;
  if (P->dim != 2) return fail(P, STK_EINVAL, "planar_errors needs a two-dimensional problem");
  if (!psi_freq || !psi_amp || !p_freq || !p_amp || !err_u || !err_p)
    return fail(P, STK_EINVAL, "NULL argument");
  int rc = check_vec(P, x, "x");
  if (rc) return rc;
  constexpr int kBlocks = 304;
  double* part = nullptr;
  cudaError_t e = stk::dev_alloc(&part, sizeof(double) * 2 * kBlocks);
  if (e == cudaSuccess) e = stk::launch_errors_planar(P, psi_freq, psi_amp, p_freq, p_amp, x, part, kBlocks);
  std::vector<double> h(2 * kBlocks, 0.0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, sizeof(double) * 2 * kBlocks, cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (part) cudaFree(part);
  if (e != cudaSuccess) return status_of(P, e, "planar_errors");
  double su = 0.0, sp = 0.0;
  for (int b = 0; b < kBlocks; ++b) {
    su += h[2 * b];
    sp += h[2 * b + 1];
  }
  *err_u = std::sqrt(su);
  *err_p = std::sqrt(sp);
  return STK_OK;
}

int stk_destroy(stk_problem* P) {
  if (!P) return STK_OK;
  cudaStreamSynchronize(P->stream);
  free_problem(P);
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

int stk_prolongate_add(stk_problem* P, int fine_level, int dtype, const void* xc, void* xf) {
  int rc = check_level(P, fine_level);
  if (rc) return rc;
  if (fine_level == 0) return fail(P, STK_EINVAL, "level 0 has no coarser level");
  if ((rc = check_dtype(P, dtype)) || (rc = check_vec(P, xc, "xc")) || (rc = check_vec(P, xf, "xf"))) return rc;
  return status_of(P, stk::launch_prolongate_add(P, fine_level, dtype, xc, xf), "prolongate_add");
}

int stk_restrict(stk_problem* P, int fine_level, int dtype, const void* rf, void* rc_out) {
  int rc = check_level(P, fine_level);
  if (rc) return rc;
  if (fine_level == 0) return fail(P, STK_EINVAL, "level 0 has no coarser level");
  if ((rc = check_dtype(P, dtype)) || (rc = check_vec(P, rf, "rf")) || (rc = check_vec(P, rc_out, "rc"))) return rc;
  return status_of(P, stk::launch_restrict(P, fine_level, dtype, rf, rc_out), "restrict");
}

int stk_smooth(stk_problem* P, int level, int dtype, void* x, const void* b) {
  int rc = check_level(P, level);
  if (rc) return rc;
  if ((rc = check_dtype(P, dtype)) || (rc = check_vec(P, x, "x")) || (rc = check_vec(P, b, "b"))) return rc;
  if (x == b) return fail(P, STK_EINVAL, "x and b must not alias");
  return status_of(P, stk::run_smooth(P, level, dtype, x, b), "smooth");
}

int stk_smooth_colour(stk_problem* P, int level, int dtype, int colour, void* x, const void* b) {
  int rc = check_level(P, level);
  if (rc) return rc;
  if ((rc = check_dtype(P, dtype)) || (rc = check_vec(P, x, "x")) || (rc = check_vec(P, b, "b"))) return rc;
  if (colour < 0 || colour >= (P->dim == 2 ? 4 : 8))
    return fail(P, STK_EINVAL, P->dim == 2 ? "colour must be in 0..3" : "colour must be in 0..7");
  if (x == b) return fail(P, STK_EINVAL, "x and b must not alias");
  return status_of(P, stk::run_smooth_colour(P, level, dtype, colour, x, b), "smooth_colour");
}

int stk_smooth_batch(stk_problem* const* problems, int count, const int* levels, int dtype, void* const* x,
                     const void* const* b) {
  if (!problems || count < 1 || !levels || !x || !b) return fail(nullptr, STK_EINVAL, "smooth_batch: empty or NULL arguments");
  if (dtype != STK_F64 && dtype != STK_F32) return fail(nullptr, STK_EINVAL, "dtype must be STK_F64 or STK_F32");
  for (int i = 0; i < count; ++i) {
    stk_problem* P = problems[i];
    if (!P) return fail(nullptr, STK_EINVAL, "smooth_batch: NULL problem");
    if (P->dim != 3) return fail(nullptr, STK_EINVAL, "smooth_batch: three-dimensional problems only");
    if (P->k != problems[0]->k) return fail(nullptr, STK_EINVAL, "smooth_batch: problems of different degrees");
    int rc;
    if ((rc = check_level(P, levels[i])) || (rc = check_vec(P, x[i], "x")) || (rc = check_vec(P, b[i], "b"))) {
      g_setup_error = "problem " + std::to_string(i) + ": " + P->err;
      return rc;
    }
    if (x[i] == b[i]) return fail(nullptr, STK_EINVAL, "smooth_batch: x and b must not alias");
    for (int j = 0; j < i; ++j)
      if (problems[j] == P) return fail(nullptr, STK_EINVAL, "smooth_batch: a problem appears twice");
  }
  const cudaError_t e = stk::run_smooth_batch(problems, levels, count, dtype, x, b);
  if (e != cudaSuccess) return fail(nullptr, e == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA,
                                    std::string("smooth_batch: ") + cudaGetErrorString(e));
  return STK_OK;
}

int stk_coarse_solve(stk_problem* P, int dtype, const void* b, void* x) {
  if (!P) return STK_EINVAL;
  int rc;
  if ((rc = check_mg(P)) || (rc = check_dtype(P, dtype)) || (rc = check_vec(P, b, "b")) || (rc = check_vec(P, x, "x")))
    return rc;
  if (x == b) return fail(P, STK_EINVAL, "x and b must not alias");
  return status_of(P, stk::run_coarse_solve(P, dtype, b, x), "coarse_solve");
}

int stk_vcycle(stk_problem* P, int dtype, const void* b, void* x) {
  if (!P) return STK_EINVAL;
  int rc;
  if ((rc = check_mg(P)) || (rc = check_dtype(P, dtype)) || (rc = check_vec(P, b, "b")) || (rc = check_vec(P, x, "x")))
    return rc;
  if (x == b) return fail(P, STK_EINVAL, "x and b must not alias");
  return status_of(P, stk::run_vcycle(P, dtype, b, x), "vcycle");
}

int stk_solve(stk_problem* P, const double* b, double* x, double rtol, stk_solve_info* info) {
  if (!P) return STK_EINVAL;
  int rc;
  if ((rc = check_mg(P)) || (rc = check_vec(P, b, "b")) || (rc = check_vec(P, x, "x"))) return rc;
  if ((const void*)x == (const void*)b) return fail(P, STK_EINVAL, "x and b must not alias");
  if (!(rtol > 0.0)) return fail(P, STK_EINVAL, "rtol must be positive");
  std::string err;
  rc = stk::run_solve(P, b, x, rtol, info, err);
  if (rc) return fail(P, rc, err);
  return STK_OK;
}

int stk_solve_batch(stk_problem* const* problems, int count, const double* const* b, double* const* x, double rtol,
                    stk_solve_info* infos) {
  if (!problems || count < 1 || !b || !x) return fail(nullptr, STK_EINVAL, "solve_batch: empty or NULL arguments");
  if (!(rtol > 0.0)) return fail(nullptr, STK_EINVAL, "rtol must be positive");
  for (int i = 0; i < count; ++i) {
    stk_problem* P = problems[i];
    if (!P) return fail(nullptr, STK_EINVAL, "solve_batch: NULL problem");
    // an in-place call would zero b with x at the start of the solve
    if ((const void*)x[i] == (const void*)b[i]) return fail(nullptr, STK_EINVAL, "solve_batch: x and b must not alias");
    int rc;
    if ((rc = check_mg(P)) || (rc = check_vec(P, b[i], "b")) || (rc = check_vec(P, x[i], "x"))) {
      g_setup_error = "problem " + std::to_string(i) + ": " + P->err;
      return rc;
    }
    for (int j = 0; j < i; ++j)
      if (problems[j] == P) return fail(nullptr, STK_EINVAL, "solve_batch: a problem appears twice");
  }
  std::string err;
  const int rc = stk::run_solve_batch(problems, count, b, x, rtol, infos, err);
  if (rc) return fail(nullptr, rc, err);
  return STK_OK;
}

// A V-cycle graph captured before a change of tuning replays the old launch
// shapes: drop it so that the next solve captures the new ones.
static void drop_graphs(stk_problem* P, int dtype) {
  stk::MgWork& W = P->mg[dtype];
  cudaStreamSynchronize(P->stream);
  if (W.graph) cudaGraphExecDestroy(W.graph);
  W.graph = nullptr;
  W.vcycle_runs = 0;
  if (P->kry.solve_graph) cudaGraphExecDestroy(P->kry.solve_graph);  // holds the V-cycle's launches too
  P->kry.solve_graph = nullptr;
}

int stk_autotune(stk_problem* P, int dtype) {
  if (!P) return STK_EINVAL;
  int rc = check_3d(P, "autotune");
  if (rc) return rc;
  rc = check_dtype(P, dtype);
  if (rc) return rc;
  const size_t es = dtype == STK_F64 ? 8 : 4;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (size_t l = 0; e == cudaSuccess && l < P->levels.size(); ++l) {
    stk::Level& L = P->levels[l];
    void *x = nullptr, *y = nullptr;
    e = stk::dev_alloc(&x, L.ntotal * es);
    if (e == cudaSuccess) e = stk::dev_alloc(&y, L.ntotal * es);
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, L.ntotal * es, P->stream);
    float best = 1e30f;
    int best_chunk = 0;
    // candidate run lengths of the persistent march: n, then halving to 2
    for (int chunk = L.n;; chunk = (chunk + 1) / 2) {
      if (e != cudaSuccess) break;
      L.apply_chunk[dtype] = chunk;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = stk::launch_apply(P, (int)l, dtype, x, nullptr, y, 1.0);
      if (e == cudaSuccess) e = cudaEventRecord(e0, P->stream);
      for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) e = stk::launch_apply(P, (int)l, dtype, x, nullptr, y, 1.0);
      if (e == cudaSuccess) e = cudaEventRecord(e1, P->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_chunk = chunk;
      }
      if (chunk <= 2) break;
    }
    L.apply_chunk[dtype] = best_chunk;
    // the smoother's form on the levels that are smoothed (all but the
    // coarsest): one step of each, on a deterministic nonzero x and b
    if (e == cudaSuccess && l > 0) {
      fill_pattern(x, L.ntotal, dtype, 1, P->stream);
      fill_pattern(y, L.ntotal, dtype, 2, P->stream);
      e = cudaGetLastError();
      float tf[2] = {1e30f, 1e30f};
      for (int form = 0; form < 2 && e == cudaSuccess; ++form) {
        L.fused_pick[dtype] = form;
        e = stk::run_smooth(P, (int)l, dtype, x, y);  // warm-up (builds Direct inverses if needed)
        if (e == cudaSuccess) e = cudaEventRecord(e0, P->stream);
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) e = stk::run_smooth(P, (int)l, dtype, x, y);
        if (e == cudaSuccess) e = cudaEventRecord(e1, P->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&tf[form], e0, e1);
      }
      L.fused_pick[dtype] = tf[1] < tf[0] ? 1 : 0;
      // then, in that form, the interior patches in their own launch or not
      float ts[2] = {1e30f, 1e30f};
      for (int sp = 0; sp < 2 && e == cudaSuccess && L.eo_interior; ++sp) {
        L.split_pick[dtype] = sp;
        e = stk::run_smooth(P, (int)l, dtype, x, y);
        if (e == cudaSuccess) e = cudaEventRecord(e0, P->stream);
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) e = stk::run_smooth(P, (int)l, dtype, x, y);
        if (e == cudaSuccess) e = cudaEventRecord(e1, P->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ts[sp], e0, e1);
      }
      if (L.eo_interior) L.split_pick[dtype] = ts[1] < ts[0] ? 1 : 0;
    }
    if (x) cudaFree(x);
    if (y) cudaFree(y);
  }
  drop_graphs(P, dtype);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return status_of(P, e, "autotune");
}

int stk_tuned_smoother(const stk_problem* P, int level, int dtype, int* fused) {
  if (!P || !fused || level < 0 || level >= (int)P->levels.size() || (dtype != STK_F64 && dtype != STK_F32))
    return STK_EINVAL;
  *fused = P->levels[level].fused_pick[dtype];
  return STK_OK;
}

int stk_tuned_split(const stk_problem* P, int level, int dtype, int* split) {
  if (!P || !split || level < 0 || level >= (int)P->levels.size() || (dtype != STK_F64 && dtype != STK_F32))
    return STK_EINVAL;
  *split = P->levels[level].split_pick[dtype];
  return STK_OK;
}

int stk_tuning(const stk_problem* P, int level, int dtype, int* cells_per_run) {
  if (!P || !cells_per_run || level < 0 || level >= (int)P->levels.size() || (dtype != STK_F64 && dtype != STK_F32))
    return STK_EINVAL;
  *cells_per_run = P->levels[level].apply_chunk[dtype];
  return STK_OK;
}

int stk_set_tuning(stk_problem* P, int level, int dtype, int cells_per_run) {
  if (!P) return STK_EINVAL;
  int rc = check_3d(P, "set_tuning");
  if (rc) return rc;
  if (level < 0 || level >= (int)P->levels.size() || (dtype != STK_F64 && dtype != STK_F32) || cells_per_run < 0)
    return fail(P, STK_EINVAL, "set_tuning: level, dtype or cells per run out of range");
  P->levels[level].apply_chunk[dtype] = cells_per_run;
  drop_graphs(P, dtype);
  return STK_OK;
}

int stk_rhs(stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq, const double* p_amp,
            double* b) {
  if (!P) return STK_EINVAL;
  if (!psi_freq || !psi_amp || !p_freq || !p_amp) return fail(P, STK_EINVAL, "coefficient arrays must not be NULL");
  int rc = check_vec(P, b, "b");
  if (rc) return rc;
  for (int i = 0; i < 27; ++i)
    if (psi_freq[i] < 1 || psi_freq[i] > 8) return fail(P, STK_EINVAL, "psi frequencies must be in 1..8");
  for (int i = 0; i < 9; ++i)
    if (p_freq[i] < 1 || p_freq[i] > 8) return fail(P, STK_EINVAL, "pressure frequencies must be in 1..8");
  if (P->dim == 2) return status_of(P, stk::launch_rhs_planar(P, psi_freq, psi_amp, p_freq, p_amp, b), "rhs");
  return status_of(P, stk::launch_rhs(P, psi_freq, psi_amp, p_freq, p_amp, b), "rhs");
}

}  // extern "C"
