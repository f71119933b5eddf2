// Internal declarations of the tensor-product Schwarz smoother library.
//
// Layout conventions (all device arrays):
//  * DoF vectors: cell-major (cells lexicographic, x fastest), then the
//    (k+1)^d nodal values of the cell, x fastest (eq. discFEspace, eq. multiindex).
//  * 1D matrices: row-major n x n with the TEST index first, so that
//    (A u)_i = sum_j A[i*n + j] u_j.
//  * Patch tensors: n^d values, patch-local 1D index p_t = c_t (k+1) + i_t with
//    c_t in {0,1} the cell of the patch along t (vertex patches, Sec. 3.2) or
//    p_t = i_t (cells).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tpss.h"

namespace tpss {

constexpr int kMaxDegree = 15;
constexpr int kMaxMixedDegree = 7;        // FP32 / TF32 / BF16 smoothers and batches
constexpr int kMaxN1 = kMaxDegree + 1;    // (k+1)
constexpr int kMaxNP = 2 * kMaxN1;        // 2(k+1): vertex patch 1D size
constexpr int kMaxNQ = kMaxN1 + 1;        // Gauss points of the right-hand side rule

// thread-local message for tpss_last_error()
void set_error(const std::string& msg);
void clear_error();

#define TPSS_CHECK_CUDA(call)                                                         \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      ::tpss::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
      return TPSS_ECUDA;                                                              \
    }                                                                                 \
  } while (0)

#define TPSS_CHECK_LAUNCH()                                                           \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess) {                                                          \
      ::tpss::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));     \
      return TPSS_ECUDA;                                                              \
    }                                                                                 \
  } while (0)

#define TPSS_REQUIRE(cond, msg)                                                       \
  do {                                                                                \
    if (!(cond)) {                                                                    \
      ::tpss::set_error(msg);                                                         \
      return TPSS_EINVAL;                                                             \
    }                                                                                 \
  } while (0)

#define TPSS_TRY(expr)                                                                \
  do {                                                                                \
    tpss_status s_ = (expr);                                                          \
    if (s_ < 0) return s_;                                                            \
  } while (0)

// 1D reference data on [0,1], computed on the device by setup_basis_kernel.
struct Basis1D {
  int k, n1, nq_rhs;
  double nodes[kMaxN1];                 // Gauss-Lobatto points
  double xq[kMaxN1], wq[kMaxN1];        // (k+1)-point Gauss rule
  double xr[kMaxNQ], wr[kMaxNQ];        // (k+2)-point Gauss rule (right-hand side)
  double Vr[kMaxNQ * kMaxN1];           // Vr[q*n1+i] = phi_i(xr_q)
  double d0[kMaxN1], d1[kMaxN1];        // phi_i'(0), phi_i'(1)
  double Mhat[kMaxN1 * kMaxN1];         // sum_q wq phi_i phi_j
  double Lhat[kMaxN1 * kMaxN1];         // sum_q wq phi_i' phi_j'
  double Pc[2][kMaxN1 * kMaxN1];        // Pc[s][i*n1+j] = phi_j((x_i + s)/2)
  double Vq[kMaxN1 * kMaxN1];           // Vq[q*n1+i] = phi_i(xq_q)  (compact, stride n1)
  double Dq[kMaxN1 * kMaxN1];           // Dq[q*n1+i] = phi_i'(xq_q)
  int status;                           // 0 ok, else Newton failed to converge
};

// 1D matrices of one cell of width h in a line of cells (eq. 1Dsipg with the
// Nitsche terms of eq. 1Dnitsche): entry (i, j) of M and A.  hl / hr are the
// neighbours' widths (h where absent), gpk = gamma_hat P(k) of eq. penalty;
// eta = 1/2 on interior faces (the 1/sqrt(2) averages of eq. bfsipg), 1 on the
// boundary.
__device__ __forceinline__ void op1d_entry(const Basis1D* B, double h, double hl, double hr, bool has_l,
                                           bool has_r, double gpk, int i, int j, double* m, double* a) {
  const int n1 = B->n1, k = B->k;
  const double gl = gpk * (1.0 / h + 1.0 / hl), gr = gpk * (1.0 / h + 1.0 / hr);
  const double el = has_l ? 0.5 : 1.0, er = has_r ? 0.5 : 1.0;
  *m = h * B->Mhat[i * n1 + j];
  double v = B->Lhat[i * n1 + j] / h;
  // left face p = 0: G[i][j] = -eta/h phi_j'(0) phi_i(0)
  v += el * gl * (i == 0 && j == 0 ? 1.0 : 0.0);
  v += el / h * ((i == 0 ? B->d0[j] : 0.0) + (j == 0 ? B->d0[i] : 0.0));
  // right face p = 1: G[i][j] = +eta/h phi_j'(1) phi_i(1)
  v += er * gr * (i == k && j == k ? 1.0 : 0.0);
  v -= er / h * ((i == k ? B->d1[j] : 0.0) + (j == k ? B->d1[i] : 0.0));
  *a = v;
}

// Number of face-coupling coefficients stored per cell position:
// {cR0, cR1, cRd, cL0, cL1, cLd} (see operator.cu for their meaning).
constexpr int kFaceCoef = 6;

// Per-level 1D operator data for one scalar type.
template <typename T>
struct LevelOps {
  T* M[3] = {nullptr, nullptr, nullptr};     // [nc][n1*n1]   M_t(c) = h_c Mhat
  T* A[3] = {nullptr, nullptr, nullptr};     // [nc][n1*n1]   A_t(c) of eq. 1Dsipg
  T* F[3] = {nullptr, nullptr, nullptr};     // [nc][kFaceCoef]
  T* d0 = nullptr;                           // [n1]
  T* d1 = nullptr;                           // [n1]
  T* Pc = nullptr;                           // [2][n1*n1]
  T* Vr = nullptr;                           // unused for float
};

struct Level {
  int nc[3] = {1, 1, 1};
  int64_t ncells = 0;
  int64_t ndofs = 0;
  std::vector<double> widths[3];             // host copies
  double* d_widths[3] = {nullptr, nullptr, nullptr};
  double* d_verts = nullptr;                 // mapped 2D meshes: [(nc1+1)][(nc0+1)] points (x, y)
  double* d_geo = nullptr;                   // mapped meshes: per-cell geometry (GeoLayout / Geo3Layout)
  float* d_geo32 = nullptr;                  // its FP32 copy (mixed-precision V-cycle)
  LevelOps<double> op64;
  LevelOps<float> op32;
  // scratch: operator intermediates and residual, nrhs_cap right-hand sides
  int nrhs_cap = 0;
  double* t64[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  float* t32[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

// Multigrid state of one context (solver.cu).
struct MGState {
  tpss_mg_params params{};
  int mixed = 0;                         // 1: V-cycle in FP32
  std::vector<tpss_patches*> patches;    // per level, [0] unused
  int64_t n0 = 0;
  double* coarse_inv = nullptr;          // [n0][n0]
  std::vector<double*> b64, x64;         // per level right-hand side / solution
  std::vector<float*> b32, x32;
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *zold = nullptr;
  double* gj_tmp = nullptr;              // 2 n0
  int gm_restart = 0;                    // GMRES basis: (restart+1) V vectors, restart Z vectors
  double* gm_V = nullptr;
  double* gm_Z = nullptr;
  double* gm_h = nullptr;                // device scalars (2 (restart+1))
  tpss_patches* coarse_fd = nullptr;     // exact coarse solve by fast diagonalization (else coarse_inv)
  tpss_patches* coarse_acs = nullptr;    // Chebyshev coarse solve: additive cell smoother on level 0
  double cheb_a = 0.0, cheb_b = 0.0;     // spectral interval of P A_0 used by the iteration
  int cheb_m = 0;                        // Chebyshev steps per coarse solve
  double* cheb_vec = nullptr;            // 4 level-0 vectors
  cudaGraphExec_t cheb_exec = nullptr;   // captured steps for the (f, x) pair below
  const void* cheb_gf = nullptr;
  void* cheb_gx = nullptr;
  tpss_patches* coarse_acs32 = nullptr;  // mixed V-cycle on mapped meshes: FP32 Chebyshev steps
  float* cheb_vec32 = nullptr;           // 3 level-0 vectors
  cudaGraphExec_t cheb_exec32 = nullptr;
  const void* cheb_gf32 = nullptr;
  void* cheb_gx32 = nullptr;
  cudaStream_t cheb_capture = nullptr;   // private non-blocking stream for the capture
  float* ir_vec = nullptr;               // iterative refinement: 5 finest-level FP32 vectors
  double* en_vec = nullptr;              // energy-norm PCG: e and A e on the finest level
};

}  // namespace tpss

struct tpss_ctx {
  int dim = 0, k = 0, n1 = 0, nloc = 0, nlevels = 0;
  double gamma_hat = 1.0;
  int penalty_poly = 0;
  cudaStream_t stream = nullptr;
  tpss::Basis1D* d_basis = nullptr;
  tpss::Basis1D h_basis{};
  std::vector<tpss::Level> levels;
  tpss::MGState* mg = nullptr;
  double* d_scalars = nullptr;               // small device scratch for reductions
  double* d_partials = nullptr;
  int num_sms = 0;
  int mapped = 0;                            // 1: 2D bilinear quadrilateral mesh (mapped.cu)
};

struct tpss_patches {
  tpss_ctx* ctx = nullptr;
  int level = 0, kind = 0, precision = 0;
  int n = 0;                       // 1D subdomain size
  int per_sub = 0;                 // 1: eigendata per subdomain (mapped cells), not per position
  int npos[3] = {1, 1, 1};         // positions per direction
  int64_t nsub = 0;                // number of subdomains
  double* d_A[3] = {nullptr, nullptr, nullptr};   // [npos][n*n]
  double* d_M[3] = {nullptr, nullptr, nullptr};
  double* d_Z[3] = {nullptr, nullptr, nullptr};
  double* d_lam[3] = {nullptr, nullptr, nullptr}; // [npos][n]
  float* d_Z32[3] = {nullptr, nullptr, nullptr};
  float* d_lam32[3] = {nullptr, nullptr, nullptr};
  double* d_inv = nullptr;         // [nsub][n^d] 1/(sum of lambdas), FP64 path (n <= 16 in 3D)
  float* d_inv32 = nullptr;        // FP32 copy, surrogate cell solvers (mapped meshes) in FP32
  double* d_scratch = nullptr;     // 3D FP64 n > 16: [scratch_ctas][n^3] tensor slabs (one per cluster)
  int scratch_ctas = 0;
  int large_cluster = 0;           // CTAs per subdomain in that kernel: 0 = chosen per launch
  // colorings: packed positions (p_x | p_y << 10 | p_z << 20) grouped by color
  int* d_add_list = nullptr;
  std::vector<int> add_offsets;    // ncolors_add + 1
  int* d_mul_list = nullptr;
  std::vector<int> mul_offsets;    // ncolors_mul + 1
  int mul_colors_default = 0;
  int* d_mul8_list = nullptr;      // alternative 2^d-color multiplicative list (vertex)
  std::vector<int> mul8_offsets;
  int mul_colors_active = 0;
  int mult_update = 1;             // multiplicative sweep: update the residual per color (else recompute)
  int* d_lex_list = nullptr;       // every subdomain, lexicographic (x fastest)
  // 3D vertex patches: additive colors plane by plane, sorted (p_z, color,
  // p_y, p_x); plane_offsets[4 p_z + c] starts the c-th of the 4 colors
  // present in plane p_z
  int* d_plane_list = nullptr;
  std::vector<int> plane_offsets;
  int additive_schedule = 0;       // FP32-vector 3D additive: tpss_additive_schedule (BF16 3D vertex, k >= 4: TCGEN05)
  void* d_bop = nullptr;           // tcgen05 smoother: BF16 / TF32 B operands per direction and position
  int* h_fail_flag = nullptr;      // tcgen05 smoother: host-mapped word set when an MMA wait expires
  int* d_fail_flag = nullptr;      // its device address
  int expire_test = 0;             // test hook: the next tcgen05 call lets its first waits expire
  cudaStream_t aux_stream = nullptr;   // additive passes: second half of the right-hand sides
  cudaEvent_t fork_event = nullptr, join_event = nullptr;
  // per multiplicative color: cells outside the color with a face to it,
  // {cell index, face mask (bit 2t+side: neighbour at -1 / +1 along t)}
  int2* d_flux_list = nullptr;
  std::vector<int> flux_offsets;
};

namespace tpss {

inline int pack_pos(int px, int py, int pz) { return px | (py << 10) | (pz << 20); }
__host__ __device__ inline int unpack_x(int v) { return v & 1023; }
__host__ __device__ inline int unpack_y(int v) { return (v >> 10) & 1023; }
__host__ __device__ inline int unpack_z(int v) { return (v >> 20) & 1023; }

// device allocation helpers (return TPSS_ENOMEM with a message)
tpss_status dalloc(void** p, size_t bytes);
template <typename T>
tpss_status dalloc_t(T** p, size_t count) {
  return dalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}
void dfree(void* p);

// ---- operator.cu
template <typename T>
tpss_status apply_operator_t(tpss_ctx* ctx, int level, int nrhs, const T* u, T* out,
                             const T* rhs_for_residual);
tpss_status ensure_level_scratch(tpss_ctx* ctx, int level, int nrhs);

// ---- smoother.cu
// x += omega sum_j R_j^T A_j^{-1} R_j r over one color's list; if d is not
// null, d = omega A_j^{-1} R_j r is also written on the subdomains' DoFs and
// r (then writable) is scaled by 1 - omega there (the residual after the
// color on its own cells, for the multiplicative residual update).
template <typename T>
tpss_status patch_pass(tpss_patches* P, const int* list, int count, T omega, int nrhs,
                       const T* r, T* x, cudaStream_t s, T* d = nullptr);

// ---- smoother_mult.cu: residual update after one multiplicative color
template <typename T>
tpss_status mult_residual_update(tpss_patches* P, int color, int nrhs, const T* dx, T* r, cudaStream_t s);

// ---- smoother_tc.cu (TF32 / BF16 tensor-core contractions)
tpss_status patch_pass_tc(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                          float* x, cudaStream_t s, float* d = nullptr);

// ---- smoother_bf16.cu (3D BF16 tensor-core path; TPSS_EINVAL for uncovered shapes)
// rpc: right-hand sides per CTA (0 = all of them in every CTA)
tpss_status patch_pass_bf16(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                            float* x, cudaStream_t s, float* d = nullptr, int rpc = 0);
tpss_status patch_pass_bf16_atomic(tpss_patches* P, const int* list, int count, float omega, int nrhs,
                                   const float* r, float* x, cudaStream_t s);
// ---- smoother_stream.cu (3D BF16 vertex patches, column-streaming schedule:
// the whole additive pass, x written without clearing when x_is_zero)
tpss_status patch_pass_bf16_stream(tpss_patches* P, float omega, int nrhs, const float* r, float* x, int x_is_zero,
                                   cudaStream_t s);
// ---- smoother_tc05.cu (the same schedule with tcgen05 MMAs, BF16 or TF32;
// TPSS_ETIMEOUT if an earlier launch on P gave up waiting for its MMAs)
tpss_status patch_pass_tc05(tpss_patches* P, float omega, int nrhs, const float* r, float* x, int x_is_zero,
                            cudaStream_t s);
// its per-position operands and failure flag, built at setup (BF16 and TF32 3D vertex patches)
tpss_status tc05_prepare(tpss_patches* P);

// ---- smoother_large.cu (3D FP64 vertex patches with n > 16, per-CTA scratch slabs)
tpss_status patch_large_ctas(int n, int num_sms, int* max_ctas);
tpss_status patch_pass_large(tpss_patches* P, const int* list, int count, double omega, int nrhs,
                             const double* r, double* x, cudaStream_t s, double* d);
// subdomain sizes above this take the large-patch kernel in 3D
constexpr int kMaxSharedPatchN = 16;

// ---- smoother.cu: additive pass over every color (x_is_zero: x starts at 0)
template <typename T>
tpss_status smooth_additive_t(tpss_patches* P, T omega, int nrhs, const T* b, T* x, int x_is_zero);

// ---- transfer.cu
template <typename T>
tpss_status prolongate_add_t(tpss_ctx* ctx, int fine_level, int nrhs, const T* coarse, T* fine);
template <typename T>
tpss_status restrict_t(tpss_ctx* ctx, int fine_level, int nrhs, const T* fine, T* coarse);

// ---- mapped.cu (2D meshes of bilinear quadrilaterals, FP64)
constexpr int kMaxMappedDegree3 = 7;    // 3D mapped meshes (2D: kMaxDegree in FP64, kMaxMixedDegree in FP32)
template <typename T>
tpss_status mapped_apply_t(tpss_ctx* ctx, int level, int nrhs, const T* u, T* out, const T* rhs);
// surrogate cell solvers: fills P->d_A, d_M, d_Z, d_lam (per cell) and d_inv
tpss_status mapped_cell_eigendata(tpss_ctx* ctx, tpss_patches* P, int* d_err);
tpss_status mapped_rhs(tpss_ctx* ctx, int level, int kind, double* b);
// residual + surrogate cell solve + update, one launch, for the cells of
// `list` (packed positions; null: all cells of the level): mode 0 out = x +
// omega z, mode 1 d = c1 d + c2 z and out = x + d, z = P_K (b - A x)_K; out
// may alias x only for cells that are not face neighbours of one another
template <typename T>
tpss_status mapped_fused_t(tpss_patches* P, const int* list, int64_t count, int nrhs, const T* x, const T* b, T* out,
                           T* d, int mode, T omega, T c1, T c2);
// ---- mapped3.cu (3D meshes of trilinear hexahedra)
tpss_status mapped3_refine(const double* coarse, int nx, int ny, int nz, double* fine, cudaStream_t s);
tpss_status mapped3_setup_level(tpss_ctx* ctx, int level, double gpk);
template <typename T>
tpss_status mapped3_apply_t(tpss_ctx* ctx, int level, int nrhs, const T* u, T* out, const T* rhs);
tpss_status mapped3_surrogate_widths(tpss_ctx* ctx, int level, double* h);
tpss_status mapped3_inv_table(tpss_ctx* ctx, tpss_patches* P);
tpss_status mapped3_rhs(tpss_ctx* ctx, int level, double* b);
template <typename T>
tpss_status mapped3_fused_t(tpss_patches* P, const int* list, int64_t count, int nrhs, const T* x, const T* b, T* out,
                            T* d, int mode, T omega, T c1, T c2);
// per-precision views of the mapped data (nullptr where not built)
template <typename T>
inline const T* geo_of(const Level& L);
template <>
inline const double* geo_of<double>(const Level& L) { return L.d_geo; }
template <>
inline const float* geo_of<float>(const Level& L) { return L.d_geo32; }
template <typename T>
inline const T* patch_Z(const tpss_patches* P, int t);
template <>
inline const double* patch_Z<double>(const tpss_patches* P, int t) { return P->d_Z[t]; }
template <>
inline const float* patch_Z<float>(const tpss_patches* P, int t) { return P->d_Z32[t]; }
template <typename T>
inline const T* patch_inv(const tpss_patches* P);
template <>
inline const double* patch_inv<double>(const tpss_patches* P) { return P->d_inv; }
template <>
inline const float* patch_inv<float>(const tpss_patches* P) { return P->d_inv32; }

// ---- setup.cu
__global__ void gen_eig_kernel(const double* __restrict__ Aall, const double* __restrict__ Mall, int nprob, int n,
                               double* __restrict__ Zall, double* __restrict__ lamall, int* __restrict__ err);
tpss_status create_patches(tpss_ctx* ctx, int level, int kind, int precision, tpss_patches** out);

// ---- solver.cu
void destroy_mg(tpss_ctx* ctx);

}  // namespace tpss
