// Multigrid V-cycle (Alg. 1), exact coarse solve, preconditioned CG (Sec. 2.4)
// and the right-hand side of eq. sipg.
//
// Coarse level: the level-0 matrix is assembled by applying the matrix-free
// operator to the unit vectors (batched as right-hand sides) and inverted in
// place by Gauss-Jordan elimination without pivoting (the matrix is SPD);
// the coarse solve is then one dense matrix-vector product.  The paper uses a
// Chebyshev iteration preconditioned by the additive cell smoother there; an
// exact solve is the reading taken here.
//
// CG: all scalars (alpha, beta, inner products) stay on the device; partial
// sums per block are reduced by a second single-block kernel in a fixed
// order, so results are deterministic.  The host reads ||r||^2 and p^T A p
// once per iteration to test convergence and breakdown.
#include <algorithm>
#include <cmath>

#include "tpss_internal.cuh"

namespace tpss {

template <typename T>
tpss_status smooth_additive_t(tpss_patches* P, T omega, int nrhs, const T* b, T* x, int x_is_zero);
template <typename T>
tpss_status smooth_multiplicative_t(tpss_patches* P, T omega, int reverse, int nrhs, const T* b, T* x);

void destroy_mg(tpss_ctx* ctx) {
  MGState* mg = ctx->mg;
  if (!mg) return;
  for (auto* P : mg->patches)
    if (P) tpss_patches_destroy(P);
  if (mg->coarse_fd) tpss_patches_destroy(mg->coarse_fd);
  if (mg->coarse_acs) tpss_patches_destroy(mg->coarse_acs);
  if (mg->coarse_acs32) tpss_patches_destroy(mg->coarse_acs32);
  dfree(mg->cheb_vec32);
  if (mg->cheb_exec32) cudaGraphExecDestroy(mg->cheb_exec32);
  dfree(mg->cheb_vec);
  if (mg->cheb_exec) cudaGraphExecDestroy(mg->cheb_exec);
  if (mg->cheb_capture) cudaStreamDestroy(mg->cheb_capture);
  dfree(mg->ir_vec);
  dfree(mg->coarse_inv);
  dfree(mg->gj_tmp);
  for (auto* v : mg->b64) dfree(v);
  for (auto* v : mg->x64) dfree(v);
  for (auto* v : mg->b32) dfree(v);
  for (auto* v : mg->x32) dfree(v);
  dfree(mg->r); dfree(mg->z); dfree(mg->p); dfree(mg->q); dfree(mg->zold);
  dfree(mg->gm_V); dfree(mg->gm_Z); dfree(mg->gm_h);
  dfree(mg->en_vec);
  delete mg;
  ctx->mg = nullptr;
}

// ------------------------------------------------------------- reductions
constexpr int kRedThreads = 256;
constexpr int kRedBlocksMax = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double ws[32];
  v = warp_sum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) ws[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) / 32;
  v = threadIdx.x < nw ? ws[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

template <typename T>
__global__ void dot_partial_kernel(const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                                   double* __restrict__ partials) {
  double s = 0.0;   // FP64 accumulation for FP32 vectors too
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)x[i], (double)y[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void dot_final_kernel(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partials[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

template <typename T>
static tpss_status dot(tpss_ctx* ctx, const T* x, const T* y, int64_t n, double* out) {
  int nb = (int)std::min<int64_t>((n + kRedThreads * 4 - 1) / (kRedThreads * 4), kRedBlocksMax);
  if (nb < 1) nb = 1;
  dot_partial_kernel<T><<<nb, kRedThreads, 0, ctx->stream>>>(x, y, n, ctx->d_partials);
  dot_final_kernel<<<1, kRedThreads, 0, ctx->stream>>>(ctx->d_partials, nb, out);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// scalars: 0 rz, 1 pq, 2 rr, 3 rz_new, 4 r.zold, 5 rr0
template <typename T>
__global__ void cg_xr_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                             const T* __restrict__ q, int64_t n, const double* __restrict__ s) {
  const T alpha = (T)(s[0] / s[1]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

template <typename T>
__global__ void cg_p_kernel(T* __restrict__ p, const T* __restrict__ z, int64_t n,
                            const double* __restrict__ s, int flexible) {
  const T beta = (T)((s[3] - (flexible ? s[4] : 0.0)) / s[0]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// dst = s * src (types may differ)
template <typename S, typename D>
__global__ void scaled_convert_kernel(const S* __restrict__ src, D* __restrict__ dst, double s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = static_cast<D>(s * (double)src[i]);
}
// x += s * e (e in FP32)
__global__ void add_scaled_f32_kernel(double* __restrict__ x, const float* __restrict__ e, double s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(s, (double)e[i], x[i]);
}

__global__ void cg_shift_kernel(double* s) { s[0] = s[3]; }

template <typename S, typename D>
__global__ void copy_convert_kernel(const S* __restrict__ a, D* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = static_cast<D>(a[i]);
}

static int grid_for(tpss_ctx* ctx, int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)ctx->num_sms * 8;
  return (int)std::max<int64_t>(1, std::min(b, cap));
}

// ----------------------------------------------------------- coarse solve
__global__ void unit_vectors_kernel(double* __restrict__ E, int64_t n, int64_t c0, int ncols) {
  const int64_t total = n * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / n, row = e % n;
    E[e] = (row == c0 + col) ? 1.0 : 0.0;
  }
}

__global__ void gj_save_kernel(const double* __restrict__ A, int64_t n, int64_t j, double* __restrict__ tmp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    tmp[i] = A[i * n + j];       // column j
    tmp[n + i] = A[j * n + i];   // row j
  }
}

__global__ void gj_update_kernel(double* __restrict__ A, int64_t n, int64_t j, const double* __restrict__ tmp) {
  const double p = tmp[j];
  const double ip = 1.0 / p;
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, l = e % n;
    double v;
    if (i == j && l == j) v = ip;
    else if (i == j) v = tmp[n + l] * ip;
    else if (l == j) v = -tmp[i] * ip;
    else v = A[e] - tmp[i] * tmp[n + l] * ip;
    A[e] = v;
  }
}

// y = Ainv b, one warp per row, FP64 accumulation; S/D input/output types.
template <typename S, typename D>
__global__ void dense_mv_kernel(const double* __restrict__ A, const S* __restrict__ b, D* __restrict__ y, int64_t n) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (row >= n) return;
  double s = 0.0;
  for (int64_t c = lane; c < n; c += 32) s = fma(A[row * n + c], (double)b[c], s);
  s = warp_sum(s);
  if (lane == 0) y[row] = (D)s;
}

// Level 0 is a single subdomain (1 cell, or 2 cells = one vertex patch, per
// direction): its fast-diagonalization inverse is A_0^{-1}.
static bool coarse_is_one_subdomain(const tpss_ctx* ctx, int* kind) {
  const Level& L0 = ctx->levels[0];
  bool ones = true, twos = true;
  for (int t = 0; t < ctx->dim; ++t) {
    ones = ones && L0.nc[t] == 1;
    twos = twos && L0.nc[t] == 2;
  }
  *kind = ones ? TPSS_CELL : TPSS_VERTEX_PATCH;
  return ones || twos;
}

constexpr int64_t kDenseCoarseAuto = 4096;   // AUTO: dense inverse up to this size

// ------------------------------------------- Chebyshev coarse solver (Sec. 2.4)
// The paper solves the coarse problem to a relative accuracy of 1e-8 with a
// Chebyshev iteration preconditioned by the additive cell smoother (P, omega
// = 1).  Spectral interval of P A_0: Lanczos matrix of 50 PCG steps from a
// SplitMix64 start vector, its extreme Ritz values widened to [0.8, 1.1] x;
// steps: the smallest m with 2 q^m / (1 + q^2m) <= 1e-8,
// q = (sqrt(kappa) - 1)/(sqrt(kappa) + 1), kappa = b/a.  Three-term recurrence
//   theta = (b+a)/2, delta = (b-a)/2, sigma = theta/delta, rho_0 = 1/sigma,
//   d_0 = P f / theta, x_1 = d_0, and for k >= 1: r_k = f - A x_k,
//   rho_k = 1/(2 sigma - rho_(k-1)), d_k = rho_k rho_(k-1) d_(k-1) + (2 rho_k/delta) P r_k,
//   x_(k+1) = x_k + d_k.
constexpr int kChebLanczosSteps = 50;
constexpr double kChebLow = 0.8, kChebHigh = 1.1, kChebTol = 1e-8;

static uint64_t splitmix64(uint64_t i) {   // output i of SplitMix64 from state 0
  uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Number of eigenvalues of the symmetric tridiagonal (diag, off) below x
// (Sturm sequence of the LDL^T pivots).
static int sturm_count(const std::vector<double>& diag, const std::vector<double>& off, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t j = 0; j < diag.size(); ++j) {
    const double o2 = j > 0 ? off[j - 1] * off[j - 1] : 0.0;
    q = diag[j] - x - (j > 0 ? o2 / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// i-th smallest eigenvalue (0-based) by bisection inside the Gershgorin interval
static double tridiag_eig(const std::vector<double>& diag, const std::vector<double>& off, int i) {
  double lo = 1e300, hi = -1e300;
  for (size_t j = 0; j < diag.size(); ++j) {
    const double rad = (j > 0 ? std::fabs(off[j - 1]) : 0.0) + (j + 1 < diag.size() ? std::fabs(off[j]) : 0.0);
    lo = std::min(lo, diag[j] - rad);
    hi = std::max(hi, diag[j] + rad);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(diag, off, mid) > i) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, double a, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}
__global__ void xpay_kernel(double* __restrict__ p, const double* __restrict__ z, double b, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    p[e] = fma(b, p[e], z[e]);
}
// d = c1 d + c2 z; x += d
__global__ void cheb_step_kernel(double* __restrict__ x, double* __restrict__ d, const double* __restrict__ z,
                                 double c1, double c2, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double dn = fma(c1, d[e], c2 * z[e]);
    d[e] = dn;
    x[e] += dn;
  }
}

static tpss_status chebyshev_setup(tpss_ctx* ctx, MGState* mg) {
  const int64_t n = mg->n0;
  cudaStream_t s = ctx->stream;
  TPSS_TRY(create_patches(ctx, 0, TPSS_CELL, TPSS_FP64, &mg->coarse_acs));
  TPSS_TRY(dalloc_t(&mg->cheb_vec, (size_t)4 * n));
  double* r = mg->cheb_vec;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  {
    std::vector<double> sv((size_t)n);
    for (int64_t i = 0; i < n; ++i) sv[i] = 2.0 * ((double)(splitmix64((uint64_t)i) >> 11) * 0x1.0p-53) - 1.0;
    TPSS_CHECK_CUDA(cudaMemcpyAsync(r, sv.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  double* sc = ctx->d_scalars;
  auto host_dot = [&](const double* a, const double* b, double* out) -> tpss_status {
    TPSS_TRY(dot(ctx, a, b, n, sc + 7));
    TPSS_CHECK_CUDA(cudaMemcpyAsync(out, sc + 7, sizeof(double), cudaMemcpyDeviceToHost, s));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
    return TPSS_OK;
  };
  const int g = grid_for(ctx, n);
  TPSS_TRY(smooth_additive_t<double>(mg->coarse_acs, 1.0, 1, r, z, 1));   // z = P r
  TPSS_CHECK_CUDA(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double rz = 0.0;
  TPSS_TRY(host_dot(r, z, &rz));
  std::vector<double> alphas, betas;
  const int steps = (int)std::min<int64_t>(n, kChebLanczosSteps);
  for (int j = 0; j < steps && rz > 0.0; ++j) {
    TPSS_TRY(apply_operator_t<double>(ctx, 0, 1, p, q, nullptr));
    double pq = 0.0;
    TPSS_TRY(host_dot(p, q, &pq));
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    axpy_kernel<<<g, 256, 0, s>>>(r, q, -alpha, n);
    TPSS_CHECK_LAUNCH();
    TPSS_TRY(smooth_additive_t<double>(mg->coarse_acs, 1.0, 1, r, z, 1));
    double rz_new = 0.0;
    TPSS_TRY(host_dot(r, z, &rz_new));
    alphas.push_back(alpha);
    betas.push_back(rz_new / rz);
    if (!(rz_new > 0.0)) break;
    xpay_kernel<<<g, 256, 0, s>>>(p, z, rz_new / rz, n);
    TPSS_CHECK_LAUNCH();
    rz = rz_new;
  }
  const int m = (int)alphas.size();
  TPSS_REQUIRE(m >= 1, "tpss_mg_setup: Chebyshev coarse solver: no Lanczos step");
  std::vector<double> diag(m), off(m > 1 ? m - 1 : 0);
  for (int j = 0; j < m; ++j) {
    diag[j] = 1.0 / alphas[j] + (j > 0 ? betas[j - 1] / alphas[j - 1] : 0.0);
    if (j + 1 < m) off[j] = std::sqrt(betas[j]) / alphas[j];
  }
  const double tmin = tridiag_eig(diag, off, 0), tmax = tridiag_eig(diag, off, m - 1);
  TPSS_REQUIRE(tmin > 0.0 && std::isfinite(tmax), "tpss_mg_setup: Chebyshev coarse solver: bad spectral estimate");
  mg->cheb_a = kChebLow * tmin;
  mg->cheb_b = kChebHigh * tmax;
  const double kappa = mg->cheb_b / mg->cheb_a, qq = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
  int steps_needed = 0;
  double qm = 1.0;
  while (2.0 * qm / (1.0 + qm * qm) > kChebTol && steps_needed < 100000) {
    qm *= qq;
    ++steps_needed;
  }
  mg->cheb_m = steps_needed;
  return TPSS_OK;
}

template <typename T>
static tpss_status chebyshev_body(tpss_ctx* ctx, MGState* mg, const T* f, T* x);

template <>
tpss_status chebyshev_body<double>(tpss_ctx* ctx, MGState* mg, const double* f, double* x) {
  const int64_t n = mg->n0;
  cudaStream_t s = ctx->stream;
  double* r = mg->cheb_vec;
  double* z = r + n;
  double* d = z + n;
  const double a = mg->cheb_a, b = mg->cheb_b;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int g = grid_for(ctx, n);
  if (mg->cheb_m < 1) {
    TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    return TPSS_OK;
  }
  TPSS_TRY(smooth_additive_t<double>(mg->coarse_acs, 1.0 / theta, 1, f, d, 1));   // d_0 = P f / theta
  TPSS_CHECK_CUDA(cudaMemcpyAsync(x, d, n * sizeof(double), cudaMemcpyDeviceToDevice, s));   // x_1
  if (ctx->mapped) {
    // one launch per step (residual, surrogate cell solves, recurrence), the
    // iterate alternating between x and r
    double* xc = x;
    double* xn = r;
    for (int k = 1; k < mg->cheb_m; ++k) {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      TPSS_TRY(mapped_fused_t<double>(mg->coarse_acs, nullptr, mg->coarse_acs->nsub, 1, xc, f, xn, d, 1, 0.0,
                                      rho_new * rho, 2.0 * rho_new / delta));
      std::swap(xc, xn);
      rho = rho_new;
    }
    if (xc != x) TPSS_CHECK_CUDA(cudaMemcpyAsync(x, xc, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return TPSS_OK;
  }
  for (int k = 1; k < mg->cheb_m; ++k) {
    TPSS_TRY(apply_operator_t<double>(ctx, 0, 1, x, r, f));                // r_k = f - A x_k
    TPSS_TRY(smooth_additive_t<double>(mg->coarse_acs, 1.0, 1, r, z, 1));  // z = P r_k
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    cheb_step_kernel<<<g, 256, 0, s>>>(x, d, z, rho_new * rho, 2.0 * rho_new / delta, n);
    TPSS_CHECK_LAUNCH();
    rho = rho_new;
  }
  return TPSS_OK;
}

// FP32 steps for the mixed V-cycle on mapped meshes: the FP64 interval and
// step count with the FP32 surrogate cell solvers and operator
template <>
tpss_status chebyshev_body<float>(tpss_ctx* ctx, MGState* mg, const float* f, float* x) {
  const int64_t n = mg->n0;
  cudaStream_t s = ctx->stream;
  float* r = mg->cheb_vec32;
  float* d = r + 2 * n;
  const double a = mg->cheb_a, b = mg->cheb_b;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (mg->cheb_m < 1) {
    TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(float), s));
    return TPSS_OK;
  }
  TPSS_TRY(smooth_additive_t<float>(mg->coarse_acs32, (float)(1.0 / theta), 1, f, d, 1));   // d_0 = P f / theta
  TPSS_CHECK_CUDA(cudaMemcpyAsync(x, d, n * sizeof(float), cudaMemcpyDeviceToDevice, s));     // x_1
  float* xc = x;
  float* xn = r;
  for (int k = 1; k < mg->cheb_m; ++k) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    TPSS_TRY(mapped_fused_t<float>(mg->coarse_acs32, nullptr, mg->coarse_acs32->nsub, 1, xc, f, xn, d, 1, 0.0f,
                                   (float)(rho_new * rho), (float)(2.0 * rho_new / delta)));
    std::swap(xc, xn);
    rho = rho_new;
  }
  if (xc != x) TPSS_CHECK_CUDA(cudaMemcpyAsync(x, xc, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return TPSS_OK;
}

template <typename T>
struct ChebGraph;
template <>
struct ChebGraph<double> {
  static cudaGraphExec_t& exec(MGState* m) { return m->cheb_exec; }
  static const void*& f(MGState* m) { return m->cheb_gf; }
  static void*& x(MGState* m) { return m->cheb_gx; }
};
template <>
struct ChebGraph<float> {
  static cudaGraphExec_t& exec(MGState* m) { return m->cheb_exec32; }
  static const void*& f(MGState* m) { return m->cheb_gf32; }
  static void*& x(MGState* m) { return m->cheb_gx32; }
};

// The m steps are ~m to 3m small launches on level 0 (launch-bound): they
// are captured once per (f, x) pair into a CUDA graph on a private stream
// (the library's stream may be the legacy default stream, which cannot
// capture) and replayed on the library's stream.  If capture is not possible
// the steps run directly.
template <typename T>
static tpss_status chebyshev_apply(tpss_ctx* ctx, MGState* mg, const T* f, T* x) {
  using Gr = ChebGraph<T>;
  if (mg->cheb_m < 1) {
    TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, mg->n0 * sizeof(T), ctx->stream));
    return TPSS_OK;
  }
  cudaGraphExec_t& exec = Gr::exec(mg);
  if (!(exec && Gr::f(mg) == f && Gr::x(mg) == x)) {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    if (!mg->cheb_capture && cudaStreamCreateWithFlags(&mg->cheb_capture, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      mg->cheb_capture = nullptr;
      return chebyshev_body<T>(ctx, mg, f, x);
    }
    cudaStream_t orig = ctx->stream;
    ctx->stream = mg->cheb_capture;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(mg->cheb_capture, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const tpss_status st = chebyshev_body<T>(ctx, mg, f, x);
      ok = cudaStreamEndCapture(mg->cheb_capture, &graph) == cudaSuccess && st == TPSS_OK;
    }
    ctx->stream = orig;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    clear_error();
    if (!ok) {
      exec = nullptr;
      return chebyshev_body<T>(ctx, mg, f, x);
    }
    Gr::f(mg) = f;
    Gr::x(mg) = x;
  }
  TPSS_CHECK_CUDA(cudaGraphLaunch(exec, ctx->stream));
  return TPSS_OK;
}

static tpss_status coarse_setup(tpss_ctx* ctx, MGState* mg) {
  const Level& L0 = ctx->levels[0];
  const int64_t n = L0.ndofs;
  mg->n0 = n;
  int kind = TPSS_CELL;
  const bool fd_ok = !mg->mixed && !ctx->mapped && coarse_is_one_subdomain(ctx, &kind);
  const int choice = mg->params.coarse_solver;
  if (choice == TPSS_COARSE_CHEBYSHEV || (choice == TPSS_COARSE_AUTO && ctx->mapped && n > kDenseCoarseAuto)) {
    TPSS_REQUIRE(!mg->mixed || ctx->mapped,
                 "tpss_mg_setup: the Chebyshev coarse solver needs an FP64 V-cycle on Cartesian meshes");
    TPSS_TRY(chebyshev_setup(ctx, mg));
    if (mg->mixed) {   // mapped meshes: the same iteration in FP32 inside the FP32 V-cycle
      TPSS_TRY(create_patches(ctx, 0, TPSS_CELL, TPSS_FP32, &mg->coarse_acs32));
      TPSS_TRY(dalloc_t(&mg->cheb_vec32, 3 * (size_t)n));
    }
    return TPSS_OK;
  }
  if (choice == TPSS_COARSE_FD || (choice == TPSS_COARSE_AUTO && fd_ok && n > kDenseCoarseAuto)) {
    TPSS_REQUIRE(fd_ok, "tpss_mg_setup: the fast-diagonalization coarse solve needs an FP64 V-cycle and "
                        "1 or 2 cells per direction on level 0");
    return create_patches(ctx, 0, kind, TPSS_FP64, &mg->coarse_fd);
  }
  TPSS_REQUIRE(n <= 16384, "tpss_mg_setup: coarse level too large for the dense coarse solver");
  TPSS_TRY(dalloc_t(&mg->coarse_inv, (size_t)n * n));
  TPSS_TRY(dalloc_t(&mg->gj_tmp, (size_t)2 * n));
  // assemble A_0 column blocks: A_0 e_c for c in [c0, c0 + nc)
  const int chunk = (int)std::min<int64_t>(n, 256);
  double* E = nullptr;
  TPSS_TRY(dalloc_t(&E, (size_t)n * chunk));
  for (int64_t c0 = 0; c0 < n; c0 += chunk) {
    const int nc = (int)std::min<int64_t>(chunk, n - c0);
    unit_vectors_kernel<<<grid_for(ctx, n * nc), 256, 0, ctx->stream>>>(E, n, c0, nc);
    tpss_status st = apply_operator_t<double>(ctx, 0, nc, E, mg->coarse_inv + c0 * n, nullptr);
    if (st != TPSS_OK) {
      dfree(E);
      return st;
    }
  }
  // columns were written as rows (A_0 symmetric): coarse_inv holds A_0
  cudaStreamSynchronize(ctx->stream);
  dfree(E);
  for (int64_t j = 0; j < n; ++j) {
    gj_save_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(mg->coarse_inv, n, j, mg->gj_tmp);
    gj_update_kernel<<<grid_for(ctx, n * n), 256, 0, ctx->stream>>>(mg->coarse_inv, n, j, mg->gj_tmp);
  }
  TPSS_CHECK_LAUNCH();
  TPSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  return TPSS_OK;
}

template <typename S, typename D>
static tpss_status coarse_apply(tpss_ctx* ctx, MGState* mg, const S* b, D* x) {
  if (mg->coarse_fd || mg->coarse_acs) {   // FP64, or FP32 Chebyshev on mapped meshes
    if constexpr (sizeof(S) == sizeof(double) && sizeof(D) == sizeof(double)) {
      if (mg->coarse_fd) return smooth_additive_t<double>(mg->coarse_fd, 1.0, 1, b, x, 1);
      return chebyshev_apply<double>(ctx, mg, b, x);
    }
    if constexpr (sizeof(S) == sizeof(float) && sizeof(D) == sizeof(float)) {
      if (mg->coarse_acs32) return chebyshev_apply<float>(ctx, mg, b, x);
    }
    set_error("coarse solve: the fast-diagonalization and Chebyshev coarse solvers are FP64 only");
    return TPSS_EINVAL;
  }
  const int64_t n = mg->n0;
  const int threads = 256;
  const int64_t blocks = (n * 32 + threads - 1) / threads;
  dense_mv_kernel<S, D><<<(unsigned)blocks, threads, 0, ctx->stream>>>(mg->coarse_inv, b, x, n);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// ---------------------------------------------------------------- V-cycle
template <typename T>
static std::vector<T*>& bvec(MGState* mg);
template <>
std::vector<double*>& bvec<double>(MGState* mg) { return mg->b64; }
template <>
std::vector<float*>& bvec<float>(MGState* mg) { return mg->b32; }
template <typename T>
static std::vector<T*>& xvec(MGState* mg);
template <>
std::vector<double*>& xvec<double>(MGState* mg) { return mg->x64; }
template <>
std::vector<float*>& xvec<float>(MGState* mg) { return mg->x32; }
template <typename T>
static T* resid(Level& L);
template <>
double* resid<double>(Level& L) { return L.t64[4]; }
template <>
float* resid<float>(Level& L) { return L.t32[4]; }

template <typename T>
static tpss_status smooth(tpss_ctx* ctx, MGState* mg, int l, const T* b, T* x, bool x_zero, bool post) {
  tpss_patches* P = mg->patches[l];
  const int kind = mg->params.smoother;
  const T omega = (T)mg->params.omega;
  const int steps = mg->params.smoothing_steps > 0 ? mg->params.smoothing_steps : 1;   // m of Sec. 4
  for (int m = 0; m < steps; ++m) {
    const bool zero = x_zero && m == 0;
    if (kind == TPSS_ACS || kind == TPSS_AVS) {
      TPSS_TRY(smooth_additive_t<T>(P, omega, 1, b, x, zero ? 1 : 0));
      continue;
    }
    if (zero) TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, (size_t)ctx->levels[l].ndofs * sizeof(T), ctx->stream));
    const bool reverse = post && !mg->params.nonsymmetric;
    TPSS_TRY(smooth_multiplicative_t<T>(P, omega, reverse ? 1 : 0, 1, b, x));
  }
  return TPSS_OK;
}

// x_l = MG_l(0, b_l) (Alg. 1); b, x are level-l vectors.
template <typename T>
static tpss_status vcycle_t(tpss_ctx* ctx, MGState* mg, int l, const T* b, T* x) {
  if (l == 0) return coarse_apply<T, T>(ctx, mg, b, x);
  Level& L = ctx->levels[l];
  TPSS_TRY(smooth<T>(ctx, mg, l, b, x, true, false));                       // pre-smoothing
  T* r = resid<T>(L);
  TPSS_TRY(apply_operator_t<T>(ctx, l, 1, x, r, b));                        // r = b - A x
  T* bc = bvec<T>(mg)[l - 1];
  T* xc = xvec<T>(mg)[l - 1];
  TPSS_TRY(restrict_t<T>(ctx, l, 1, r, bc));                                 // restriction
  TPSS_TRY(vcycle_t<T>(ctx, mg, l - 1, bc, xc));                             // recursion
  TPSS_TRY(prolongate_add_t<T>(ctx, l, 1, xc, x));                          // prolongation
  TPSS_TRY(smooth<T>(ctx, mg, l, b, x, false, true));                       // post-smoothing
  return TPSS_OK;
}

// z = B r on the finest level (FP64 in and out; FP32 inside when mixed)
static tpss_status precondition(tpss_ctx* ctx, MGState* mg, const double* r, double* z) {
  const int L = ctx->nlevels - 1;
  const int64_t n = ctx->levels[L].ndofs;
  if (!mg->mixed) return vcycle_t<double>(ctx, mg, L, r, z);
  float* bf = mg->b32[L];
  float* xf = mg->x32[L];
  copy_convert_kernel<double, float><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(r, bf, n);
  TPSS_TRY(vcycle_t<float>(ctx, mg, L, bf, xf));
  copy_convert_kernel<float, double><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(xf, z, n);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// ------------------------------------------------------------------ GMRES
// partial sums of <V_i, w> for i < j: grid (chunks, j)
__global__ void multi_dot_kernel(const double* __restrict__ V, const double* __restrict__ w, int64_t n,
                                 double* __restrict__ partials, int chunks) {
  const int i = blockIdx.y;
  const double* v = V + (int64_t)i * n;
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s = fma(v[e], w[e], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partials[(int64_t)i * chunks + blockIdx.x] = s;
}

__global__ void multi_final_kernel(const double* __restrict__ partials, int chunks, double* __restrict__ out) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) s += partials[(int64_t)i * chunks + c];
  s = block_sum(s);
  if (threadIdx.x == 0) out[i] = s;
}

// w += sign * sum_{i < j} c_i V_i
__global__ void multi_axpy_kernel(double* __restrict__ w, const double* __restrict__ V, const double* __restrict__ c,
                                  int j, int64_t n, double sign) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[e];
    for (int i = 0; i < j; ++i) acc = fma(sign * c[i], V[(int64_t)i * n + e], acc);
    w[e] = acc;
  }
}

__global__ void scale_copy_kernel(double* __restrict__ dst, const double* __restrict__ src, double s, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = s * src[e];
}

// ------------------------------------------------------------ right-hand side
// kind 0: f = d pi^2 prod sin(pi x_t), g = 0;  kind 1: Gaussian bells (Sec. 2.4)
struct RhsArgs {
  const Basis1D* B;
  const double* w[3];
  int nc[3];
  int dim;
  int kind;
  double gpk;   // gamma_hat * P(k)
  double* b;
};

__device__ double bells_u(const double* x, int dim, double* lap) {
  // u = 1/(sqrt(2 pi) sigma) sum_i exp(-|x - x_i|^2 / sigma^2); lap = Laplace(u)
  const double sigma = 1.0 / 3.0, s2 = sigma * sigma;
  const double c = 1.0 / (sqrt(2.0 * 3.14159265358979323846) * sigma);
  const double src[3][3] = {{0.0, 0.0, 0.0}, {0.25, 0.85, 0.85}, {0.6, 0.4, 0.4}};
  double u = 0.0, l = 0.0;
  for (int i = 0; i < 3; ++i) {
    double r2 = 0.0;
    for (int t = 0; t < dim; ++t) r2 += (x[t] - src[i][t]) * (x[t] - src[i][t]);
    const double e = exp(-r2 / s2);
    u += e;
    l += e * (4.0 * r2 / (s2 * s2) - 2.0 * dim / s2);
  }
  *lap = c * l;
  return c * u;
}

__global__ void rhs_kernel(RhsArgs a) {
  extern __shared__ double sm[];
  const Basis1D* B = a.B;
  const int n1 = B->n1, nq = B->nq_rhs, dim = a.dim;
  const int64_t cell = blockIdx.x;
  int cm[3] = {0, 0, 0};
  int64_t rest = cell;
  for (int t = 0; t < dim; ++t) {
    cm[t] = (int)(rest % a.nc[t]);
    rest /= a.nc[t];
  }
  double lo[3] = {0, 0, 0}, h[3] = {1, 1, 1};
  for (int t = 0; t < dim; ++t) {
    double s = 0.0;
    for (int c = 0; c < cm[t]; ++c) s += a.w[t][c];
    lo[t] = s;
    h[t] = a.w[t][cm[t]];
  }
  const int nqd = dim == 3 ? nq * nq * nq : nq * nq;
  const int nloc = dim == 3 ? n1 * n1 * n1 : n1 * n1;
  double* F = sm;             // nq^d
  double* G = F + nqd;        // workspace nq^d
  double* H = G + nqd;
  double jac = 1.0;
  for (int t = 0; t < dim; ++t) jac *= h[t];
  for (int e = threadIdx.x; e < nqd; e += blockDim.x) {
    const int q0 = e % nq, q1 = (e / nq) % nq, q2 = dim == 3 ? e / (nq * nq) : 0;
    const int qq[3] = {q0, q1, q2};
    double x[3] = {0, 0, 0}, wt = jac;
    for (int t = 0; t < dim; ++t) {
      x[t] = lo[t] + h[t] * B->xr[qq[t]];
      wt *= B->wr[qq[t]];
    }
    double f;
    if (a.kind == 0) {
      const double pi = 3.14159265358979323846;
      f = dim * pi * pi;
      for (int t = 0; t < dim; ++t) f *= sin(pi * x[t]);
    } else {
      double lap;
      bells_u(x, dim, &lap);
      f = -lap;
    }
    F[e] = wt * f;
  }
  __syncthreads();
  // sum factorization: contract q0 -> i0, q1 -> i1, (q2 -> i2) with Vr[q][i]
  const double* Vr = B->Vr;
  if (dim == 3) {
    for (int e = threadIdx.x; e < n1 * nq * nq; e += blockDim.x) {
      const int i0 = e % n1, q1 = (e / n1) % nq, q2 = e / (n1 * nq);
      double s = 0.0;
      for (int q0 = 0; q0 < nq; ++q0) s += Vr[q0 * n1 + i0] * F[q0 + nq * (q1 + nq * q2)];
      G[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n1 * n1 * nq; e += blockDim.x) {
      const int i0 = e % n1, i1 = (e / n1) % n1, q2 = e / (n1 * n1);
      double s = 0.0;
      for (int q1 = 0; q1 < nq; ++q1) s += Vr[q1 * n1 + i1] * G[i0 + n1 * (q1 + nq * q2)];
      H[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nloc; e += blockDim.x) {
      const int i2 = e / (n1 * n1);
      double s = 0.0;
      for (int q2 = 0; q2 < nq; ++q2) s += Vr[q2 * n1 + i2] * H[(e % (n1 * n1)) + n1 * n1 * q2];
      G[e] = s;
    }
  } else {
    for (int e = threadIdx.x; e < n1 * nq; e += blockDim.x) {
      const int i0 = e % n1, q1 = e / n1;
      double s = 0.0;
      for (int q0 = 0; q0 < nq; ++q0) s += Vr[q0 * n1 + i0] * F[q0 + nq * q1];
      G[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nloc; e += blockDim.x) {
      const int i0 = e % n1, i1 = e / n1;
      double s = 0.0;
      for (int q1 = 0; q1 < nq; ++q1) s += Vr[q1 * n1 + i1] * G[i0 + n1 * q1];
      H[e] = s;
    }
  }
  __syncthreads();
  const double* res = dim == 3 ? G : H;
  // boundary terms int (gamma g v - g n.grad v) for kind 1
  for (int e = threadIdx.x; e < nloc; e += blockDim.x) {
    double v = res[e];
    if (a.kind == 1) {
      const int ii[3] = {e % n1, (e / n1) % n1, dim == 3 ? e / (n1 * n1) : 0};
      for (int t = 0; t < dim; ++t)
        for (int side = 0; side < 2; ++side) {
          const bool bnd = side == 0 ? cm[t] == 0 : cm[t] == a.nc[t] - 1;
          if (!bnd) continue;
          const double gam = a.gpk * 2.0 / h[t];
          const double nsign = side == 1 ? 1.0 : -1.0;
          const double phit = (ii[t] == (side == 1 ? n1 - 1 : 0)) ? 1.0 : 0.0;
          const double dphit = (side == 1 ? B->d1[ii[t]] : B->d0[ii[t]]) / h[t];
          const int o1 = t == 0 ? 1 : 0, o2 = t == 2 ? 1 : 2;
          const int nq2 = dim == 3 ? nq : 1;
          for (int qa = 0; qa < nq; ++qa)
            for (int qb = 0; qb < nq2; ++qb) {
              double x[3];
              x[t] = lo[t] + h[t] * side;
              x[o1] = lo[o1] + h[o1] * B->xr[qa];
              double wt = B->wr[qa] * h[o1];
              double other = Vr[qa * n1 + ii[o1]];
              if (dim == 3) {
                x[o2] = lo[o2] + h[o2] * B->xr[qb];
                wt *= B->wr[qb] * h[o2];
                other *= Vr[qb * n1 + ii[o2]];
              }
              double lap;
              const double g = bells_u(x, dim, &lap);
              v += wt * g * other * (gam * phit - nsign * dphit);
            }
        }
    }
    a.b[cell * nloc + e] = v;
  }
}

}  // namespace tpss

using namespace tpss;

extern "C" tpss_status tpss_assemble_rhs(tpss_ctx* ctx, int level, int kind, double* b) {
  clear_error();
  TPSS_REQUIRE(ctx && b, "tpss_assemble_rhs: null argument");
  TPSS_REQUIRE(level >= 0 && level < ctx->nlevels, "tpss_assemble_rhs: level out of range");
  TPSS_REQUIRE(kind == 0 || kind == 1, "tpss_assemble_rhs: kind must be 0 or 1");
  if (ctx->mapped) return mapped_rhs(ctx, level, kind, b);
  const Level& L = ctx->levels[level];
  RhsArgs a{};
  a.B = ctx->d_basis;
  for (int t = 0; t < 3; ++t) {
    a.w[t] = L.d_widths[t];
    a.nc[t] = L.nc[t];
  }
  a.dim = ctx->dim;
  a.kind = kind;
  a.gpk = ctx->gamma_hat * (ctx->penalty_poly == TPSS_PENALTY_KP1SQ ? (double)(ctx->n1 * ctx->n1)
                                                                    : (double)(ctx->k * ctx->n1));
  a.b = b;
  const int nq = ctx->n1 + 1;
  const size_t smem = 3 * (size_t)(ctx->dim == 3 ? nq * nq * nq : nq * nq) * sizeof(double);
  static bool attr = false;   // up to 118 KB at k = 15 in 3D
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(rhs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
    attr = true;
  }
  rhs_kernel<<<(unsigned)L.ncells, 128, smem, ctx->stream>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

extern "C" tpss_status tpss_mg_setup(tpss_ctx* ctx, const tpss_mg_params* params) {
  clear_error();
  TPSS_REQUIRE(ctx && params, "tpss_mg_setup: null argument");
  TPSS_REQUIRE(params->smoother >= TPSS_ACS && params->smoother <= TPSS_MVS, "tpss_mg_setup: unknown smoother");
  TPSS_REQUIRE(params->precision >= TPSS_FP64 && params->precision <= TPSS_BF16, "tpss_mg_setup: unknown precision");
  TPSS_REQUIRE(params->omega > 0.0 && std::isfinite(params->omega), "tpss_mg_setup: omega must be positive");
  TPSS_REQUIRE(params->precision == TPSS_FP64 || ctx->k <= kMaxMixedDegree,
               "tpss_mg_setup: mixed-precision V-cycles support degrees up to 7");
  TPSS_REQUIRE(params->coarse_solver >= TPSS_COARSE_AUTO && params->coarse_solver <= TPSS_COARSE_CHEBYSHEV,
               "tpss_mg_setup: unknown coarse solver");
  TPSS_REQUIRE(params->mult_residual == TPSS_MULT_RESIDUAL_UPDATE || params->mult_residual == TPSS_MULT_RESIDUAL_FULL,
               "tpss_mg_setup: mult_residual must be 0 (update) or 1 (full)");
  TPSS_REQUIRE(params->smoothing_steps >= 0 && params->smoothing_steps <= 16,
               "tpss_mg_setup: smoothing_steps must be in 0..16");
  const bool vertex = params->smoother == TPSS_AVS || params->smoother == TPSS_MVS;
  TPSS_REQUIRE(!ctx->mapped || (!vertex && (params->precision == TPSS_FP64 || params->precision == TPSS_FP32) &&
                                params->coarse_solver != TPSS_COARSE_FD),
               "tpss_mg_setup: mapped meshes support FP64 and FP32 cell smoothers (ACS, MCS) with the dense or "
               "Chebyshev coarse solver");
  if (vertex)
    for (int l = 1; l < ctx->nlevels; ++l)
      for (int t = 0; t < ctx->dim; ++t)
        TPSS_REQUIRE(ctx->levels[l].nc[t] >= 2, "tpss_mg_setup: vertex patches need >= 2 cells per direction");
  destroy_mg(ctx);
  MGState* mg = new MGState();
  ctx->mg = mg;
  mg->params = *params;
  mg->mixed = params->precision != TPSS_FP64;
  const int L = ctx->nlevels;
  mg->patches.assign(L, nullptr);
  mg->b64.assign(L, nullptr);
  mg->x64.assign(L, nullptr);
  mg->b32.assign(L, nullptr);
  mg->x32.assign(L, nullptr);
  tpss_status st = TPSS_OK;
  auto fail = [&](tpss_status s) {
    destroy_mg(ctx);
    return s;
  };
  for (int l = 1; l < L; ++l) {
    if ((st = create_patches(ctx, l, vertex ? TPSS_VERTEX_PATCH : TPSS_CELL, params->precision,
                             &mg->patches[l])) != TPSS_OK)
      return fail(st);
    if (params->mult_colors != 0 && (params->smoother == TPSS_MVS || params->smoother == TPSS_MCS))
      if ((st = tpss_patches_set_mult_colors(mg->patches[l], params->mult_colors)) != TPSS_OK) return fail(st);
    // surrogate cell solvers (mapped meshes) always recompute the full residual
    if (!mg->patches[l]->per_sub)
      mg->patches[l]->mult_update = params->mult_residual == TPSS_MULT_RESIDUAL_FULL ? 0 : 1;
    if ((st = ensure_level_scratch(ctx, l, 1)) != TPSS_OK) return fail(st);
  }
  if ((st = ensure_level_scratch(ctx, 0, 1)) != TPSS_OK) return fail(st);
  for (int l = 0; l < L; ++l) {
    const size_t n = (size_t)ctx->levels[l].ndofs;
    if ((st = dalloc_t(&mg->b64[l], n)) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&mg->x64[l], n)) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&mg->b32[l], n)) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&mg->x32[l], n)) != TPSS_OK) return fail(st);
  }
  const size_t nf = (size_t)ctx->levels[L - 1].ndofs;
  if ((st = dalloc_t(&mg->r, nf)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&mg->z, nf)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&mg->p, nf)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&mg->q, nf)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&mg->zold, nf)) != TPSS_OK) return fail(st);
  if ((st = coarse_setup(ctx, mg)) != TPSS_OK) return fail(st);
  TPSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  return TPSS_OK;
}

extern "C" tpss_status tpss_vcycle(tpss_ctx* ctx, const double* b, double* x) {
  clear_error();
  TPSS_REQUIRE(ctx && b && x, "tpss_vcycle: null argument");
  TPSS_REQUIRE(ctx->mg, "tpss_vcycle: call tpss_mg_setup first");
  TPSS_REQUIRE(b != x, "tpss_vcycle: b and x must not alias");
  return precondition(ctx, ctx->mg, b, x);
}

extern "C" tpss_status tpss_coarse_solve(tpss_ctx* ctx, const double* b, double* x) {
  clear_error();
  TPSS_REQUIRE(ctx && b && x, "tpss_coarse_solve: null argument");
  TPSS_REQUIRE(ctx->mg, "tpss_coarse_solve: call tpss_mg_setup first");
  TPSS_REQUIRE(b != x, "tpss_coarse_solve: b and x must not alias");
  return coarse_apply<double, double>(ctx, ctx->mg, b, x);
}

extern "C" tpss_status tpss_coarse_chebyshev_info(const tpss_ctx* ctx, double* a, double* b, int* steps) {
  clear_error();
  TPSS_REQUIRE(ctx && a && b && steps, "tpss_coarse_chebyshev_info: null argument");
  TPSS_REQUIRE(ctx->mg && ctx->mg->coarse_acs, "tpss_coarse_chebyshev_info: no Chebyshev coarse solver set up");
  *a = ctx->mg->cheb_a;
  *b = ctx->mg->cheb_b;
  *steps = ctx->mg->cheb_m;
  return TPSS_OK;
}

// e = x - xs
__global__ void diff_kernel(double* __restrict__ e, const double* __restrict__ x, const double* __restrict__ xs,
                            int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    e[i] = x[i] - xs[i];
}

// PCG with the V-cycle from x = 0.  With xs (a device vector, the solution),
// the A-norms of the errors ||x_k - xs||_A are recorded in errs and the
// iteration stops at the first one <= rtol ||xs||_A instead of on the
// residual.
static tpss_status pcg_run(tpss_ctx* ctx, const double* b, double* x, double rtol, int maxit, int* iters,
                           double* rel_res, double* res_hist, const double* xs, double* errs) {
  MGState* mg = ctx->mg;
  const int L = ctx->nlevels - 1;
  const int64_t n = ctx->levels[L].ndofs;
  cudaStream_t s = ctx->stream;
  double* sc = ctx->d_scalars;
  const int g = grid_for(ctx, n);
  *iters = 0;
  *rel_res = 1.0;
  double e0 = 0.0;
  if (xs) {
    if (!mg->en_vec) TPSS_TRY(dalloc_t(&mg->en_vec, 2 * (size_t)n));
    TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    diff_kernel<<<g, 256, 0, s>>>(mg->en_vec, x, xs, n);
    TPSS_TRY(apply_operator_t<double>(ctx, L, 1, mg->en_vec, mg->en_vec + n, nullptr));
    TPSS_TRY(dot(ctx, mg->en_vec, mg->en_vec + n, n, sc + 6));
    double h0[8];
    TPSS_CHECK_CUDA(cudaMemcpyAsync(h0, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
    e0 = std::sqrt(std::max(h0[6], 0.0));
    errs[0] = e0;
    if (e0 == 0.0) return TPSS_OK;
  }
  TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(mg->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TPSS_TRY(dot(ctx, mg->r, mg->r, n, sc + 5));
  double h[8];
  TPSS_CHECK_CUDA(cudaMemcpyAsync(h, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
  const double rr0 = h[5];
  if (res_hist) res_hist[0] = std::sqrt(rr0);
  if (!std::isfinite(rr0)) {
    set_error("tpss_pcg_solve: right-hand side is not finite");
    return TPSS_EBREAKDOWN;
  }
  if (rr0 == 0.0) {
    *rel_res = 0.0;
    return TPSS_OK;
  }
  TPSS_TRY(precondition(ctx, mg, mg->r, mg->z));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(mg->p, mg->z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TPSS_TRY(dot(ctx, mg->r, mg->z, n, sc + 0));
  const bool flex = mg->params.flexible_cg != 0;
  for (int it = 1; it <= maxit; ++it) {
    TPSS_TRY(apply_operator_t<double>(ctx, L, 1, mg->p, mg->q, nullptr));
    TPSS_TRY(dot(ctx, mg->p, mg->q, n, sc + 1));
    cg_xr_kernel<double><<<g, 256, 0, s>>>(x, mg->r, mg->p, mg->q, n, sc);
    TPSS_TRY(dot(ctx, mg->r, mg->r, n, sc + 2));
    if (xs) {
      diff_kernel<<<g, 256, 0, s>>>(mg->en_vec, x, xs, n);
      TPSS_TRY(apply_operator_t<double>(ctx, L, 1, mg->en_vec, mg->en_vec + n, nullptr));
      TPSS_TRY(dot(ctx, mg->en_vec, mg->en_vec + n, n, sc + 6));
    }
    TPSS_CHECK_CUDA(cudaMemcpyAsync(h, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
    const double rel = std::sqrt(std::max(h[2], 0.0) / rr0);
    if (res_hist) res_hist[it] = std::sqrt(std::max(h[2], 0.0));
    *iters = it;
    *rel_res = rel;
    if (!std::isfinite(h[1]) || !(h[1] > 0.0) || !std::isfinite(h[2])) {
      set_error("tpss_pcg_solve: breakdown (p^T A p <= 0 or non-finite residual)");
      return TPSS_EBREAKDOWN;
    }
    if (xs) {
      errs[it] = std::sqrt(std::max(h[6], 0.0));
      if (errs[it] <= rtol * e0) return TPSS_OK;
    } else if (rel <= rtol) {
      return TPSS_OK;
    }
    if (flex) std::swap(mg->z, mg->zold);
    TPSS_TRY(precondition(ctx, mg, mg->r, mg->z));
    TPSS_TRY(dot(ctx, mg->r, mg->z, n, sc + 3));
    if (flex) TPSS_TRY(dot(ctx, mg->r, mg->zold, n, sc + 4));
    cg_p_kernel<double><<<g, 256, 0, s>>>(mg->p, mg->z, n, sc, flex ? 1 : 0);
    cg_shift_kernel<<<1, 1, 0, s>>>(sc);
    TPSS_CHECK_LAUNCH();
  }
  set_error("tpss_pcg_solve: not converged within maxit");
  return TPSS_ENOTCONV;
}

extern "C" tpss_status tpss_pcg_solve(tpss_ctx* ctx, const double* b, double* x, double rtol, int maxit,
                                      int* iters, double* rel_res, double* res_hist) {
  clear_error();
  TPSS_REQUIRE(ctx && b && x && iters && rel_res, "tpss_pcg_solve: null argument");
  TPSS_REQUIRE(ctx->mg, "tpss_pcg_solve: call tpss_mg_setup first");
  TPSS_REQUIRE(rtol > 0.0 && maxit >= 1, "tpss_pcg_solve: rtol must be > 0 and maxit >= 1");
  return pcg_run(ctx, b, x, rtol, maxit, iters, rel_res, res_hist, nullptr, nullptr);
}

extern "C" tpss_status tpss_pcg_energy_errors(tpss_ctx* ctx, const double* b, const double* xs, double* x,
                                              double rtol, int maxit, int* count, double* errs) {
  clear_error();
  TPSS_REQUIRE(ctx && b && xs && x && count && errs, "tpss_pcg_energy_errors: null argument");
  TPSS_REQUIRE(ctx->mg, "tpss_pcg_energy_errors: call tpss_mg_setup first");
  TPSS_REQUIRE(rtol > 0.0 && maxit >= 1, "tpss_pcg_energy_errors: rtol must be > 0 and maxit >= 1");
  TPSS_REQUIRE(x != xs && x != b, "tpss_pcg_energy_errors: x must not alias b or xs");
  int it = 0;
  double rel = 0.0;
  *count = 0;
  const tpss_status st = pcg_run(ctx, b, x, rtol, maxit, &it, &rel, nullptr, xs, errs);
  *count = it + 1;
  if (st == TPSS_ENOTCONV) set_error("tpss_pcg_energy_errors: error not reduced by rtol within maxit");
  return st;
}

// Mixed-precision iterative refinement: FP64 residual outside, an FP32 PCG
// with the FP32 V-cycle and the FP32 operator inside on the normalized
// residual, FP64 correction.  Flexible beta in the inner CG (the FP32
// V-cycle is not exactly symmetric).
extern "C" tpss_status tpss_ir_solve(tpss_ctx* ctx, const double* b, double* x, double rtol, int max_outer,
                                     double inner_rtol, int max_inner, int* outer_iters, int* inner_iters,
                                     double* rel_res) {
  clear_error();
  TPSS_REQUIRE(ctx && b && x && outer_iters && inner_iters && rel_res, "tpss_ir_solve: null argument");
  TPSS_REQUIRE(ctx->mg, "tpss_ir_solve: call tpss_mg_setup first");
  TPSS_REQUIRE(ctx->mg->mixed, "tpss_ir_solve: needs a mixed-precision (FP32 / TF32 / BF16) V-cycle");
  TPSS_REQUIRE(rtol > 0.0 && inner_rtol > 0.0 && inner_rtol < 1.0 && max_outer >= 1 && max_inner >= 1,
               "tpss_ir_solve: rtol > 0, 0 < inner_rtol < 1, max_outer >= 1 and max_inner >= 1 required");
  MGState* mg = ctx->mg;
  const int L = ctx->nlevels - 1;
  const int64_t n = ctx->levels[L].ndofs;
  cudaStream_t s = ctx->stream;
  if (mg->ir_vec == nullptr) TPSS_TRY(dalloc_t(&mg->ir_vec, (size_t)5 * n));
  float* r32 = mg->ir_vec;
  float* z32 = r32 + n;
  float* p32 = z32 + n;
  float* q32 = p32 + n;
  float* e32 = q32 + n;
  double* sc = ctx->d_scalars;
  const int g = grid_for(ctx, n);
  double h[8];
  auto fetch = [&]() -> tpss_status {
    TPSS_CHECK_CUDA(cudaMemcpyAsync(h, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
    return TPSS_OK;
  };
  *outer_iters = 0;
  *inner_iters = 0;
  *rel_res = 1.0;
  TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(mg->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TPSS_TRY(dot(ctx, mg->r, mg->r, n, sc + 5));
  TPSS_TRY(fetch());
  const double rr0 = h[5];
  if (!std::isfinite(rr0)) {
    set_error("tpss_ir_solve: right-hand side is not finite");
    return TPSS_EBREAKDOWN;
  }
  if (rr0 == 0.0) {
    *rel_res = 0.0;
    return TPSS_OK;
  }
  double rnorm = std::sqrt(rr0);
  for (int outer = 1; outer <= max_outer; ++outer) {
    // inner: A e = r / ||r|| in FP32 from e = 0
    scaled_convert_kernel<double, float><<<g, 256, 0, s>>>(mg->r, r32, 1.0 / rnorm, n);
    TPSS_CHECK_CUDA(cudaMemsetAsync(e32, 0, n * sizeof(float), s));
    TPSS_CHECK_LAUNCH();
    TPSS_TRY(dot(ctx, r32, r32, n, sc + 5));
    TPSS_TRY(vcycle_t<float>(ctx, mg, L, r32, z32));
    TPSS_CHECK_CUDA(cudaMemcpyAsync(p32, z32, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    TPSS_TRY(dot(ctx, r32, z32, n, sc + 0));
    TPSS_TRY(fetch());
    const double irr0 = h[5];
    for (int it = 1; it <= max_inner; ++it) {
      TPSS_TRY(apply_operator_t<float>(ctx, L, 1, p32, q32, nullptr));
      TPSS_TRY(dot(ctx, p32, q32, n, sc + 1));
      cg_xr_kernel<float><<<g, 256, 0, s>>>(e32, r32, p32, q32, n, sc);
      TPSS_TRY(dot(ctx, r32, r32, n, sc + 2));
      TPSS_TRY(fetch());
      ++*inner_iters;
      if (!std::isfinite(h[1]) || !(h[1] > 0.0) || !std::isfinite(h[2])) {
        set_error("tpss_ir_solve: inner breakdown (p^T A p <= 0 or non-finite residual)");
        return TPSS_EBREAKDOWN;
      }
      if (std::sqrt(std::max(h[2], 0.0) / irr0) <= inner_rtol) break;
      std::swap(z32, q32);   // q32 is free until the next operator application: keeps z_old
      TPSS_TRY(vcycle_t<float>(ctx, mg, L, r32, z32));
      TPSS_TRY(dot(ctx, r32, z32, n, sc + 3));
      TPSS_TRY(dot(ctx, r32, q32, n, sc + 4));
      cg_p_kernel<float><<<g, 256, 0, s>>>(p32, z32, n, sc, 1);
      cg_shift_kernel<<<1, 1, 0, s>>>(sc);
      TPSS_CHECK_LAUNCH();
    }
    // x += ||r|| e; r = b - A x in FP64
    add_scaled_f32_kernel<<<g, 256, 0, s>>>(x, e32, rnorm, n);
    TPSS_CHECK_LAUNCH();
    TPSS_TRY(apply_operator_t<double>(ctx, L, 1, x, mg->r, b));
    TPSS_TRY(dot(ctx, mg->r, mg->r, n, sc + 6));
    TPSS_TRY(fetch());
    rnorm = std::sqrt(std::max(h[6], 0.0));
    *outer_iters = outer;
    *rel_res = rnorm / std::sqrt(rr0);
    if (!std::isfinite(rnorm)) {
      set_error("tpss_ir_solve: non-finite residual");
      return TPSS_EBREAKDOWN;
    }
    if (*rel_res <= rtol) return TPSS_OK;
  }
  set_error("tpss_ir_solve: not converged within max_outer");
  return TPSS_ENOTCONV;
}

extern "C" tpss_status tpss_gmres_solve(tpss_ctx* ctx, const double* b, double* x, double rtol, int maxit,
                                        int restart, int left, int* iters, double* rel_res, double* res_hist) {
  clear_error();
  TPSS_REQUIRE(ctx && b && x && iters && rel_res, "tpss_gmres_solve: null argument");
  TPSS_REQUIRE(ctx->mg, "tpss_gmres_solve: call tpss_mg_setup first");
  TPSS_REQUIRE(rtol > 0.0 && maxit >= 1 && restart >= 1 && restart <= 200,
               "tpss_gmres_solve: rtol > 0, maxit >= 1, 1 <= restart <= 200 required");
  MGState* mg = ctx->mg;
  const int L = ctx->nlevels - 1;
  const int64_t n = ctx->levels[L].ndofs;
  cudaStream_t s = ctx->stream;
  if (mg->gm_restart < restart) {
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
    dfree(mg->gm_V); dfree(mg->gm_Z); dfree(mg->gm_h);
  dfree(mg->en_vec);
    mg->gm_V = mg->gm_Z = mg->gm_h = nullptr;
    mg->gm_restart = 0;
    TPSS_TRY(dalloc_t(&mg->gm_V, (size_t)(restart + 1) * n));
    TPSS_TRY(dalloc_t(&mg->gm_Z, (size_t)restart * n));
    TPSS_TRY(dalloc_t(&mg->gm_h, (size_t)2 * (restart + 1)));
    mg->gm_restart = restart;
  }
  // partial sums of the multi-dot live in ctx->d_partials (4096 doubles)
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(n / (kRedThreads * 8), 4096 / (restart + 1)));
  const int g = grid_for(ctx, n);
  double* V = mg->gm_V;
  double* Z = mg->gm_Z;
  double* dh = mg->gm_h;
  double* w = mg->q;   // finest-level scratch vectors
  double* av = mg->p;
  const bool left_pc = left != 0;
  auto vec = [&](double* base, int i) { return base + (int64_t)i * n; };
  // <V_i, w> for i < j into dh[0..j), copied to the host
  auto project = [&](int j, std::vector<double>& h) -> tpss_status {
    dim3 grid(chunks, j);
    multi_dot_kernel<<<grid, kRedThreads, 0, s>>>(V, w, n, ctx->d_partials, chunks);
    multi_final_kernel<<<j, kRedThreads, 0, s>>>(ctx->d_partials, chunks, dh);
    TPSS_CHECK_LAUNCH();
    h.resize(j);
    TPSS_CHECK_CUDA(cudaMemcpyAsync(h.data(), dh, j * sizeof(double), cudaMemcpyDeviceToHost, s));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
    multi_axpy_kernel<<<g, 256, 0, s>>>(w, V, dh, j, n, -1.0);
    TPSS_CHECK_LAUNCH();
    return TPSS_OK;
  };
  auto norm = [&](const double* v, double* out) -> tpss_status {
    TPSS_TRY(dot(ctx, v, v, n, ctx->d_scalars + 6));
    double hv = 0.0;
    TPSS_CHECK_CUDA(cudaMemcpyAsync(&hv, ctx->d_scalars + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
    *out = std::sqrt(std::max(hv, 0.0));
    return TPSS_OK;
  };
  TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  if (left_pc) {
    TPSS_TRY(precondition(ctx, mg, b, mg->r));   // r_0 = M b
  } else {
    TPSS_CHECK_CUDA(cudaMemcpyAsync(mg->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  double beta0 = 0.0;
  TPSS_TRY(norm(mg->r, &beta0));
  *iters = 0;
  *rel_res = beta0 > 0.0 ? 1.0 : 0.0;
  if (res_hist) res_hist[0] = beta0;
  if (!std::isfinite(beta0)) {
    set_error("tpss_gmres_solve: right-hand side is not finite");
    return TPSS_EBREAKDOWN;
  }
  if (beta0 == 0.0) return TPSS_OK;
  int it = 0;
  std::vector<double> H((size_t)(restart + 1) * restart), gv(restart + 1), cs(restart), sn(restart), h1, h2;
  double beta = beta0;
  while (it < maxit) {
    scale_copy_kernel<<<g, 256, 0, s>>>(vec(V, 0), mg->r, 1.0 / beta, n);
    TPSS_CHECK_LAUNCH();
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jdone = 0;
    bool done = false;
    for (int j = 0; j < restart && it < maxit; ++j) {
      ++it;
      if (left_pc) {   // w = M A v_j
        TPSS_TRY(apply_operator_t<double>(ctx, L, 1, vec(V, j), av, nullptr));
        TPSS_TRY(precondition(ctx, mg, av, w));
      } else {         // z_j = M v_j, w = A z_j
        TPSS_TRY(precondition(ctx, mg, vec(V, j), vec(Z, j)));
        TPSS_TRY(apply_operator_t<double>(ctx, L, 1, vec(Z, j), w, nullptr));
      }
      TPSS_TRY(project(j + 1, h1));   // classical Gram-Schmidt ...
      TPSS_TRY(project(j + 1, h2));   // ... with one reorthogonalization
      auto Hij = [&](int i, int jj) -> double& { return H[(size_t)i * restart + jj]; };
      for (int i = 0; i <= j; ++i) Hij(i, j) = h1[i] + h2[i];
      double hn = 0.0;
      TPSS_TRY(norm(w, &hn));
      Hij(j + 1, j) = hn;
      if (!std::isfinite(hn)) {
        set_error("tpss_gmres_solve: breakdown (non-finite Arnoldi vector)");
        return TPSS_EBREAKDOWN;
      }
      if (hn > 0.0) {
        scale_copy_kernel<<<g, 256, 0, s>>>(vec(V, j + 1), w, 1.0 / hn, n);
        TPSS_CHECK_LAUNCH();
      }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double d = std::hypot(Hij(j, j), Hij(j + 1, j));
      cs[j] = Hij(j, j) / d;
      sn[j] = Hij(j + 1, j) / d;
      Hij(j, j) = d;
      Hij(j + 1, j) = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      if (res_hist) res_hist[it] = std::fabs(gv[j + 1]);
      *iters = it;
      *rel_res = std::fabs(gv[j + 1]) / beta0;
      jdone = j + 1;
      if (std::fabs(gv[j + 1]) <= rtol * beta0 || hn == 0.0) {
        done = true;
        break;
      }
    }
    // x += Z y with H(1:j,1:j) y = g(1:j)
    std::vector<double> y(jdone);
    for (int i = jdone - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int k = i + 1; k < jdone; ++k) acc -= H[(size_t)i * restart + k] * y[k];
      y[i] = acc / H[(size_t)i * restart + i];
    }
    TPSS_CHECK_CUDA(cudaMemcpyAsync(dh, y.data(), jdone * sizeof(double), cudaMemcpyHostToDevice, s));
    multi_axpy_kernel<<<g, 256, 0, s>>>(x, left_pc ? V : Z, dh, jdone, n, 1.0);
    TPSS_CHECK_LAUNCH();
    if (done) return TPSS_OK;
    // restart from the true (left: preconditioned) residual
    if (left_pc) {
      TPSS_TRY(apply_operator_t<double>(ctx, L, 1, x, av, b));
      TPSS_TRY(precondition(ctx, mg, av, mg->r));
    } else {
      TPSS_TRY(apply_operator_t<double>(ctx, L, 1, x, mg->r, b));
    }
    TPSS_TRY(norm(mg->r, &beta));
    if (!(beta > 0.0)) return TPSS_OK;
  }
  set_error("tpss_gmres_solve: not converged within maxit");
  return TPSS_ENOTCONV;
}
