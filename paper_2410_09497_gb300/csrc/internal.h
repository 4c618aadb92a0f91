// Internal declarations of libstokesmg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <memory>
#include <string>
#include <vector>

#include "stokesmg.h"

namespace stk {

// alloc.cu: all allocations of the library (with the host-side fault injector)
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t dev_alloc_async(void** p, size_t bytes, cudaStream_t s);
cudaError_t host_alloc_pinned(void** p, size_t bytes);
template <typename T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc(reinterpret_cast<void**>(p), bytes);
}
template <typename T>
cudaError_t dev_alloc_async(T** p, size_t bytes, cudaStream_t s) {
  return dev_alloc_async(reinterpret_cast<void**>(p), bytes, s);
}
template <typename T>
cudaError_t host_alloc_pinned(T** p, size_t bytes) {
  return host_alloc_pinned(reinterpret_cast<void**>(p), bytes);
}

// Raises a kernel's dynamic shared-memory limit to `bytes` (needed above
// 48 KB) once per device: the attribute belongs to the function on the device
// that is current, so `done` keeps one bit per device.  Two threads making the
// first call together both set it, which is harmless.
template <typename Kernel>
cudaError_t allow_dynamic_smem(Kernel* fn, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

constexpr int kMaxDegree = 5;
constexpr int kMaxC = kMaxDegree + 2;  // nodes of a cell in the continuous direction
constexpr int kMaxD = kMaxDegree + 1;  // nodes of a cell in a discontinuous direction

// 1D cell matrices of one level (Sec. 2.3 and Sec. 3.2), row-major, in the
// precision of the kernel that reads them.  Layout is fixed so a kernel can
// copy the whole struct into shared memory.
//   KC[i][j]  nu * int phi_i' phi_j'      continuous (Gauss-Lobatto) basis, (k+2)^2
//   MC[i][j]  int phi_i phi_j (no nu)     continuous basis, (k+2)^2
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

// The contraction along the continuous direction in even-odd form.  KC and
// MC are centro-symmetric and D is antisymmetric under the reflection of a
// cell (its Gauss-Lobatto and Gauss nodes are symmetric), so with the
// P = (k+2)/2 node pairs (a, k+1-a) of the continuous basis, sums
// ue[a] = u[a] + u[k+1-a] (and the centre node when k+2 is odd) and
// differences uo[a] = u[a] - u[k+1-a], and the same for the Q = (k+1)/2
// pressure pairs, the half-sums and half-differences of the outputs are
//   Ze[i] = sum_a EK[i][a] ue[a] + EM[i][a] te[a] + sum_q ED[i][q] po[q]
//   Zo[i] = sum_a OK[i][a] uo[a] + OM[i][a] to[a] + sum_q OD[i][q] pe[q]
// and z[i] = Ze[i] + Zo[i], z[k+1-i] = Ze[i] - Zo[i] (the centre output is
// Ze[P]): about half the products of the dense form.  Row-major with row
// length kMaxC (EK, EM, OK, OM) or kMaxD (ED, OD).
template <typename T>
struct ContractTables {
  T EK[kMaxC * kMaxC];
  T EM[kMaxC * kMaxC];
  T OK[kMaxC * kMaxC];
  T OM[kMaxC * kMaxC];
  T ED[kMaxC * kMaxD];
  T OD[kMaxC * kMaxD];
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

constexpr int kMaxPatchJobs = 64;  // problems per multi-problem patch launch
constexpr int kMaxPC = 2 * kMaxDegree + 1;  // patch-interior nodes, continuous direction
constexpr int kMaxPD = 2 * kMaxDegree + 2;  // patch nodes, discontinuous direction

// Fast-diagonalization data of the vertex-patch local solver (Sec. 3.2) for
// one level, in kernel precision:
//   SC[i][j], LC[j]  eigenvectors (columns) / eigenvalues of the continuous direction
//   SD[t][i][j], LD[t][j]  the same for a discontinuous direction of boundary type t
//   DL[q][a]  local divergence factor (2k+2 pressure x 2k+1 velocity nodes)
//   W[j]      diagonal patch mass of a discontinuous direction
//   EC[q][j]  = sum_a DL[q][a] SC[a][j]: the divergence factor in the eigenbasis
//   FM[t][q][j] = W[q] SD[t][q][j]: the mass factor in the eigenbasis
// The four transform matrices are stored with rows of kRowStride entries
// (zero padded, 16-byte aligned) so that kernels read a row with vector loads.
// Kernels treat every transform as (2k+2) x (2k+2): SC and EC carry a zero row
// / column 2k+1 and LC[2k+1] = 1, so a padded node of a velocity component's
// continuous direction stays exactly zero through every pass.
constexpr int kRowStride = 12;
template <typename T>
struct PatchTables {
  alignas(16) T SC[kMaxPD * kRowStride];
  alignas(16) T SD[4][kMaxPD * kRowStride];
  alignas(16) T EC[kMaxPD * kRowStride];
  alignas(16) T FM[4][kMaxPD * kRowStride];
  T LC[kMaxPD];
  T LD[4][kMaxPD];
  T DL[kMaxPD * kMaxPC];
  T W[kMaxPD];
  T inv_nu;
  // 1 when the eigenvectors of SC / SD[t] are ordered even (symmetric under
  // the patch reflection) first, odd after: the kernels then transform lines
  // in the even-odd form (half the products).  Holds for SC and for the
  // reflection-symmetric types 0 and 3.
  int eo_c;
  int eo_d[4];
};

struct PatchTables1D {
  int k = 0;
  double nu = 1.0;
  std::vector<double> SC, LC, SD[4], LD[4], DL, W;
  // even-odd ordering (see sort_by_parity): eigenvectors symmetric under the
  // reflection of the patch come first, antisymmetric ones after
  bool eo_c = false, eo_d[4] = {false, false, false, false};
};

void generalized_eigen(int n, const std::vector<double>& K, const std::vector<double>& M, std::vector<double>& S,
                       std::vector<double>& lam);
struct Tables1D;
PatchTables1D build_patch_tables(const Tables1D& t);
template <typename T>
void fill_patch_tables(const PatchTables1D& p, PatchTables<T>* out);
// PC[2][k+2][k+2] followed by PD[2][k+1][k+1] (transfer.cu)
std::vector<double> build_transfer_tables(int k);

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w);
// values V[i*np+q] = l_i(t_q) and derivatives Dv[i*np+q] = l_i'(t_q)
void lagrange(const std::vector<double>& z, const std::vector<double>& t, std::vector<double>& V,
              std::vector<double>& Dv);
Tables1D build_tables(int k, double h, double nu, double penalty_factor);

template <typename T>
void fill_cell_tables(const Tables1D& t, CellTables<T>* out);
template <typename T>
void fill_contract_tables(const Tables1D& t, ContractTables<T>* out);

struct Level {
  int n = 0, m = 0;
  double h = 0;
  int64_t nvel = 0, npress = 0, ntotal = 0;
  Tables1D t1d;
  CellTables<double>* tab64 = nullptr;  // device
  CellTables<float>* tab32 = nullptr;   // device
  CellTables<double> htab64{};          // host copies, passed to kernels by value
  CellTables<float> htab32{};
  ContractTables<double> hce64{};       // even-odd contraction tables, by value
  ContractTables<float> hce32{};
  int apply_chunk[2] = {0, 0};          // cells per run of the apply's velocity march ([dtype]); 0 = default
  int fused_pick[2] = {-1, -1};         // smoother form chosen by stk_autotune ([dtype]); -1 = the option's
  int split_pick[2] = {-1, -1};         // interior patches in their own launch, chosen by stk_autotune ([dtype]); -1 = by count
  PatchTables<double>* ptab64 = nullptr;  // device
  PatchTables<float>* ptab32 = nullptr;   // device
  PatchTables<double> hptab64;            // host copies (the interior kernel's matrices go by value)
  PatchTables<float> hptab32;
  bool eo_interior = false;  // continuous and interior 1D eigenbases both in even-odd order
  // Direct local solver (built on first use): (S + a 1 1^T)^{-1} of every patch
  // type of the level, column-major (2k+2)^3 squared, FP64 and FP32 copies, and
  // device tables of 64 pointers indexed by t0 + 4 t1 + 16 t2 (NULL: absent)
  bool dir_ready = false;
  double* dirM64 = nullptr;
  float* dirM32 = nullptr;
  const double** dirtab64 = nullptr;
  const float** dirtab32 = nullptr;
  const float* dir32_host[64] = {};  // the FP32 inverses' device addresses, per type, on the host
  // FP32 Direct as one GEMM per colour: the interior patches' R and P
  // (gemm_cap patches of (2k+2)^3 entries each)
  float* gemmR = nullptr;
  float* gemmP = nullptr;
  int64_t gemm_cap = 0;
  // two dimensions: the 1D cell tables flattened with runtime sizes (the
  // order of stk_cell_tables), device copies in both precisions
  double* flat64 = nullptr;
  float* flat32 = nullptr;
};

// Exact local solver of the 2D vertex patches (2 x 2 cells): for every patch
// type (boundary type t0 + 4 t1 per direction) the pseudo-inverse of the patch
// matrix with the pressure mean fixed, at h = 1 (the velocity block does not
// depend on h in two dimensions and the divergence blocks scale with h; the
// kernels rescale the pressure rows and columns by 1/h), column-major, FP64
// and FP32.  Shared by the problems of a process with the same device,
// degree, viscosity and penalty factor.
struct PlanarInverses {
  int nloc = 0;
  double* m64[16] = {};
  float* m32[16] = {};
  const double** tab64 = nullptr;  // device arrays of the 16 pointers
  const float** tab32 = nullptr;
  ~PlanarInverses();
};
constexpr int kMaxPlanarDegree = 8;

struct MgWork {
  bool ready = false;
  std::vector<void*> r, b, x;  // per level: residual, right-hand side, solution
  int vcycle_runs = 0;          // V-cycles run on the finest-level buffers
  cudaGraphExec_t graph = nullptr;  // captured V-cycle on b.back() -> x.back()
};

struct KrylovWork {
  bool ready = false;
  double* V = nullptr;     // (restart + 1) basis vectors
  double* Z = nullptr;     // restart preconditioned vectors
  double* w = nullptr;     // the new Arnoldi vector
  double* zbuf = nullptr;  // FP64 copy of the FP32 V-cycle's output (mixed precision)
  double* partial = nullptr;
  double* h = nullptr;     // Gram-Schmidt coefficients and norms
  void* state = nullptr;       // device state of the FGMRES recurrence (solver.cu)
  void* state_host = nullptr;  // pinned copy
  cudaStream_t side[2] = {nullptr, nullptr};  // capture streams of the loop bodies
  cudaGraphExec_t solve_graph = nullptr;       // the whole solve for (key_b, key_x, key_rtol)
  const double* key_b = nullptr;
  double* key_x = nullptr;
  double key_rtol = 0;
};

struct Coarse3Factors;  // coarse3.cu

}  // namespace stk

struct stk_problem {
  int dim = 3;  // 3: the unit cube; 2: the unit square (Table 1)
  int k = 0;
  double nu = 1.0;
  stk_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<stk::Level> levels;  // [0] coarsest
  double* xfer64 = nullptr;        // device transfer tables (build_transfer_tables)
  float* xfer32 = nullptr;
  double* pmean_w = nullptr;       // device Gauss weights x h of the finest level (pressure mean)
  double* coarse_inv = nullptr;    // dense pseudo-inverse of the 2^3 coarse problem, patch order
  double* coarse3[3] = {nullptr, nullptr, nullptr};  // FP64 b, x, r of a 3^3 coarse mesh
  std::shared_ptr<stk::Coarse3Factors> coarse3f;      // dense factors of the 3^3 coarse problem (shared)
  std::shared_ptr<stk::PlanarInverses> pinv2;         // 2D patch inverses (shared)
  void* blas = nullptr;            // cuBLAS handle of the Direct solver's GEMM (created on first use)
  void* blas_ws = nullptr;         // its workspace
  size_t blas_ws_bytes = 0;
  stk::MgWork mg[2];               // [STK_F64], [STK_F32]
  stk::KrylovWork kry;
  std::string err;
};

namespace stk {

// Launchers (apply.cu).  y = alpha * A x + (b ? b : 0); returns a cudaError_t.
// stages: bit 0 = velocity rows, bit 1 = pressure rows (3 = the whole operator).
cudaError_t launch_apply(const stk_problem* P, int level, int dtype, const void* x, const void* b, void* y,
                         double alpha, int stages = 3);
// the same on a given stream
cudaError_t launch_apply_on(const stk_problem* P, int level, int dtype, const void* x, const void* b, void* y,
                            double alpha, int stages, cudaStream_t stream);
// xf += I^up xc (xc on fine_level - 1); rc = I^down rf (rc is overwritten).
cudaError_t launch_prolongate_add(const stk_problem* P, int fine_level, int dtype, const void* xc, void* xf);
cudaError_t launch_restrict(const stk_problem* P, int fine_level, int dtype, const void* rf, void* rc);
// smoother.cu
int patch_local_size(int k);
cudaError_t launch_patch_colour(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x);
// the fused colour (patch residual computed in the kernel): xout = xin + the
// colour's corrections at its patch DoFs; xin and xout must not alias
cudaError_t launch_patch_colour_fused(const stk_problem* P, int level, int dtype, int colour, const void* xin,
                                      const void* b, void* xout);
// xout = xin at every entry no patch of the colour owns
cudaError_t launch_copy_unowned(const stk_problem* P, int level, int dtype, int colour, const void* xin, void* xout);
cudaError_t launch_patch_colour_cg(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x,
                                   int cg_tol_mode, int cg_iters, double cg_tol);
cudaError_t launch_coarse_columns(const stk_problem* P, double* cols, int max_iter, double tol);
// the local inverses of the Direct solver of a level (smoother.cu); synchronous
cudaError_t ensure_direct(stk_problem* P, int level);
// coarse3.cu: M <- (M + a 1 1^T)^{-1}, a = trace(M) / n^2, for a symmetric
// positive semidefinite M (n x n, row stride ld) whose null space is the
// constants; by Gauss-Jordan elimination on the stream
cudaError_t invert_shifted(double* M, int64_t n, int64_t ld, cudaStream_t s);
// one colour of `count` problems of the same degree (levels[i] of problem i),
// kMaxPatchJobs problems per launch, on `stream`; local-solver options of Ps[0]
cudaError_t launch_patch_colour_multi(const stk_problem* const* Ps, const int* levels, int count, int dtype,
                                      int colour, void* const* r, void* const* x, cudaStream_t stream);
cudaError_t launch_coarse_solve(const stk_problem* P, int dtype, const void* b, void* x);
// coarse3.cu: exact solve on a 3^3 coarse mesh.  acquire_coarse3 builds (or
// takes from the cache) the dense factors, using P->coarse3 as probes and
// synchronizing the stream; coarse3_solve maps P->coarse3[0] (pressure rows
// summing to zero) to P->coarse3[1], with P->coarse3[2] as scratch.
cudaError_t acquire_coarse3(stk_problem* P);
cudaError_t coarse3_solve(stk_problem* P);
// solver.cu
cudaError_t ensure_mg_workspace(stk_problem* P, int dtype);
cudaError_t ensure_coarse(stk_problem* P);
cudaError_t run_smooth(stk_problem* P, int level, int dtype, void* x, const void* b);
cudaError_t run_smooth_colour(stk_problem* P, int level, int dtype, int colour, void* x, const void* b);
cudaError_t run_smooth_batch(stk_problem* const* Ps, const int* levels, int count, int dtype, void* const* x,
                             const void* const* b);
cudaError_t run_vcycle(stk_problem* P, int dtype, const void* b, void* x);
cudaError_t run_coarse_solve(stk_problem* P, int dtype, const void* b, void* x);
int run_solve(stk_problem* P, const double* b, double* x, double rtol, stk_solve_info* info, std::string& err);
int run_solve_batch(stk_problem* const* Ps, int count, const double* const* b, double* const* x, double rtol,
                    stk_solve_info* infos, std::string& err);
// rhs.cu
cudaError_t launch_rhs(const stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq,
                       const double* p_amp, double* b);
// planar.cu: the method on the unit square (n = 2^L cells per side, k = 1..8)
cudaError_t setup_planar(stk_problem* P);
cudaError_t launch_apply_planar(const stk_problem* P, int level, int dtype, const void* x, const void* b, void* y,
                                int stages, cudaStream_t s);
cudaError_t launch_prolongate_add_planar(const stk_problem* P, int fine_level, int dtype, const void* xc, void* xf);
cudaError_t launch_restrict_planar(const stk_problem* P, int fine_level, int dtype, const void* rf, void* rc);
// one colour of 2D patch solves (exact local solver): x += R_j^T A_j^+ R_j r
cudaError_t launch_patch_colour_planar(const stk_problem* P, int level, int dtype, int colour, const void* r, void* x);
cudaError_t launch_coarse_solve_planar(const stk_problem* P, int dtype, const void* b, void* x);
cudaError_t launch_pressure_mean_planar(stk_problem* P, double* x, double* partial, int nblocks);
cudaError_t launch_rhs_planar(const stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq,
                              const double* p_amp, double* b);
cudaError_t launch_errors_planar(const stk_problem* P, const int* psi_freq, const double* psi_amp, const int* p_freq,
                                 const double* p_amp, const double* x, double* partial, int nblocks);

}  // namespace stk
