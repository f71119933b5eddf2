// Context creation and the fast-diagonalization setup (Sec. 3.2).
//
// Everything numeric runs on the device in FP64:
//   setup_basis_kernel   Gauss-Lobatto nodes (roots of P_k' by Newton), Gauss
//                        rules, Lagrange tables, reference mass/stiffness.
//   level_op1d_kernel    per direction and cell position: M_t(c) and A_t(c) of
//                        eq. 1Dstiffnessmass - eq. 1Dsipg plus the face
//                        coupling coefficients to the neighbouring cells.
//   patch_matrices_kernel  A^(t), M^(t) of eq. 1Dsipg (cells) or eq. 1DsipgVP
//                        (vertex patches) per direction and position.
//   gen_eig_kernel       the generalized eigenproblem of eq. generalizedEVP by
//                        Cholesky of M and cyclic Jacobi on L^{-1} A L^{-T}.
//   inv_table_kernel     1/(lambda_i + lambda_j + lambda_l) per subdomain
//                        (the diagonal of Lambda^{-1} in eq. fastinverse).
#include <cmath>
#include <cstring>

#include "tpss_internal.cuh"

namespace tpss {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }

tpss_status dalloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    return TPSS_ENOMEM;
  }
  return TPSS_OK;
}
void dfree(void* p) {
  if (p) cudaFree(p);
}

// ------------------------------------------------------------------ basis
__device__ void legendre_eval(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (x * p1 - p0) / (x * x - 1.0);
}

__device__ double lagrange_val(const double* nodes, int n, int j, double x) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) v *= (x - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

__device__ double lagrange_der(const double* nodes, int n, int j, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == j) continue;
    double t = 1.0 / (nodes[j] - nodes[m]);
    for (int l = 0; l < n; ++l)
      if (l != j && l != m) t *= (x - nodes[l]) / (nodes[j] - nodes[l]);
    s += t;
  }
  return s;
}

// Gauss rule with nq points on [0,1] (Newton on P_nq from Chebyshev-like guesses).
__device__ bool gauss_rule(int nq, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  bool ok = true;
  for (int i = 0; i < nq; ++i) {
    double t = -cos(pi * (i + 0.75) / (nq + 0.5));
    double P, dP;
    int it = 0;
    for (; it < 100; ++it) {
      legendre_eval(nq, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    if (it == 100) ok = false;
    legendre_eval(nq, t, &P, &dP);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dP * dP);  // 2/((1-t^2) P'^2) mapped to [0,1]
  }
  return ok;
}

// One block: thread 0 finds the nodes and Gauss rules (Newton), then the
// tables are filled in parallel; the reference mass and stiffness matrices
// come from tabulated basis values and derivatives at the Gauss points.
constexpr int kBasisThreads = 256;

__global__ void __launch_bounds__(kBasisThreads) setup_basis_kernel(Basis1D* B, int k) {
  __shared__ double Vq[kMaxN1 * kMaxN1], Dq[kMaxN1 * kMaxN1];   // phi_i(xq_q), phi_i'(xq_q) at [q*n1+i]
  const double pi = 3.14159265358979323846;
  const int n1 = k + 1, tid = threadIdx.x;
  if (tid == 0) {
    B->k = k;
    B->n1 = n1;
    B->nq_rhs = k + 2;
    B->status = 0;
    // Gauss-Lobatto nodes: end points and roots of P_k' (Newton, P_k'' from the
    // Legendre equation (1-t^2) P'' = 2 t P' - k(k+1) P).
    double t_nodes[kMaxN1];
    t_nodes[0] = -1.0;
    t_nodes[k] = 1.0;
    for (int j = 1; j < k; ++j) {
      double t = -cos(pi * j / k);
      int it = 0;
      for (; it < 100; ++it) {
        double P, dP;
        legendre_eval(k, t, &P, &dP);
        double d2P = (2.0 * t * dP - k * (k + 1.0) * P) / (1.0 - t * t);
        double dt = dP / d2P;
        t -= dt;
        if (fabs(dt) < 1e-16) break;
      }
      if (it == 100) B->status = 1;
      t_nodes[j] = t;
    }
    for (int j = 0; j <= k; ++j) B->nodes[j] = 0.5 * (t_nodes[j] + 1.0);
    if (!gauss_rule(n1, B->xq, B->wq)) B->status = 2;
    if (!gauss_rule(n1 + 1, B->xr, B->wr)) B->status = 3;
  }
  __syncthreads();
  const double* nd = B->nodes;
  for (int e = tid; e < n1 * n1; e += kBasisThreads) {
    const int q = e / n1, i = e % n1;
    Vq[e] = lagrange_val(nd, n1, i, B->xq[q]);
    Dq[e] = lagrange_der(nd, n1, i, B->xq[q]);
    for (int s2 = 0; s2 < 2; ++s2) B->Pc[s2][e] = lagrange_val(nd, n1, i, 0.5 * (nd[q] + s2));   // e = q*n1+i: row q, col i
    B->Vq[e] = Vq[e];
    B->Dq[e] = Dq[e];
  }
  for (int e = tid; e < (n1 + 1) * n1; e += kBasisThreads)
    B->Vr[e] = lagrange_val(nd, n1, e % n1, B->xr[e / n1]);
  for (int i = tid; i < n1; i += kBasisThreads) {
    B->d0[i] = lagrange_der(nd, n1, i, 0.0);
    B->d1[i] = lagrange_der(nd, n1, i, 1.0);
  }
  __syncthreads();
  for (int e = tid; e < n1 * n1; e += kBasisThreads) {
    const int i = e / n1, j = e % n1;
    double m = 0.0, l = 0.0;
    for (int q = 0; q < n1; ++q) {
      m += B->wq[q] * Vq[q * n1 + i] * Vq[q * n1 + j];
      l += B->wq[q] * Dq[q * n1 + i] * Dq[q * n1 + j];
    }
    B->Mhat[e] = m;
    B->Lhat[e] = l;
  }
}

// Per-level 1D data.  For cell c of direction t with width h = w[c]:
//   M_t(c) = h Mhat
//   A_t(c) = Lhat / h + N_0 + N_1 (eq. 1Dsipg), with the Nitsche terms of
//   eq. 1Dnitsche, N_p = eta gamma M_p - G_p - G_p^T, eta = 1/2 on interior
//   faces (applied to the penalty as well, following eq. bfsipg with its
//   1/sqrt(2) averages) and eta = 1 on boundary faces; gamma from eq. penalty.
//   Face couplings to the neighbours (rank-2 in the GL nodal basis):
//   (A u)_i += delta_{i,k} (cR0 u_R[0] + cR1 d0.u_R) + d1_i cRd u_R[0]
//            + delta_{i,0} (cL0 u_L[k] + cL1 d1.u_L) + d0_i cLd u_L[k]
//   where u_R / u_L are the right / left neighbour's values on the same line.
__global__ void level_op1d_kernel(const Basis1D* __restrict__ B, const double* __restrict__ w,
                                  int nc, double gpk, double* __restrict__ M, double* __restrict__ A,
                                  double* __restrict__ F) {
  const int n1 = B->n1;
  const int c = blockIdx.x;
  if (c >= nc) return;
  const double h = w[c];
  const bool has_l = c > 0, has_r = c + 1 < nc;
  const double hl = has_l ? w[c - 1] : h, hr = has_r ? w[c + 1] : h;
  const double gl = gpk * (1.0 / h + 1.0 / hl), gr = gpk * (1.0 / h + 1.0 / hr);
  for (int e = threadIdx.x; e < n1 * n1; e += blockDim.x)
    op1d_entry(B, h, hl, hr, has_l, has_r, gpk, e / n1, e % n1, &M[(size_t)c * n1 * n1 + e],
               &A[(size_t)c * n1 * n1 + e]);
  if (threadIdx.x == 0) {
    double* f = F + (size_t)c * kFaceCoef;
    f[0] = has_r ? -0.5 * gr : 0.0;
    f[1] = has_r ? -0.5 / hr : 0.0;
    f[2] = has_r ? 0.5 / h : 0.0;
    f[3] = has_l ? -0.5 * gl : 0.0;
    f[4] = has_l ? 0.5 / hl : 0.0;
    f[5] = has_l ? -0.5 / h : 0.0;
  }
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ a, D* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = static_cast<D>(a[i]);
}

template <typename S, typename D>
static tpss_status convert(const S* a, D* b, size_t n, cudaStream_t s) {
  if (n == 0) return TPSS_OK;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  convert_kernel<S, D><<<blocks, 256, 0, s>>>(a, b, n);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// ------------------------------------------------------ patch 1D matrices
// Cells: A^(t) = A_t(c), M^(t) = M_t(c).  Vertex patch at position p (cells p
// and p+1 along t, "+" = p = left, "-" = p+1 = right, eq. 1DsipgVP):
//   A^(t) = [[A_t(p), B_p], [B_p^T, A_t(p+1)]],  M^(t) = diag(M_t(p), M_t(p+1))
// with the interface block B_p[i][j] (test i in cell p, trial j in p+1) equal to
// the right-face coupling of cell p: delta_{i,k}(cR0 delta_{j,0} + cR1 d0_j)
// + d1_i cRd delta_{j,0}; the lower-left block is the left-face coupling of
// cell p+1, which is its transpose.
__global__ void patch_matrices_kernel(const Basis1D* __restrict__ B, const double* __restrict__ Mc,
                                      const double* __restrict__ Ac, const double* __restrict__ F,
                                      int npos, int vertex, double* __restrict__ Ap,
                                      double* __restrict__ Mp) {
  const int n1 = B->n1, k = B->k;
  const int p = blockIdx.x;
  if (p >= npos) return;
  const int n = vertex ? 2 * n1 : n1;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    const int ci = i / n1, cj = j / n1, ii = i % n1, jj = j % n1;
    double a = 0.0, m = 0.0;
    if (ci == cj) {
      const size_t off = (size_t)(p + ci) * n1 * n1 + ii * n1 + jj;
      a = Ac[off];
      m = Mc[off];
    } else if (ci == 0) {  // test in the left cell p, trial in the right cell p+1
      const double* f = F + (size_t)p * kFaceCoef;
      a = (ii == k ? (jj == 0 ? f[0] : 0.0) + f[1] * B->d0[jj] : 0.0) + (jj == 0 ? B->d1[ii] * f[2] : 0.0);
    } else {  // test in the right cell p+1, trial in the left cell p
      const double* f = F + (size_t)(p + 1) * kFaceCoef;
      a = (ii == 0 ? (jj == k ? f[3] : 0.0) + f[4] * B->d1[jj] : 0.0) + (jj == k ? B->d0[ii] * f[5] : 0.0);
    }
    Ap[(size_t)p * n * n + e] = a;
    Mp[(size_t)p * n * n + e] = m;
  }
}

// ---------------------------------------------- generalized eigenproblem
// One warp per problem A z = lambda M z (n <= 32), lanes own rows or columns.
// Cholesky M = L L^T; C = L^{-1} A L^{-T}; cyclic Jacobi C = V diag V^T;
// Z = L^{-T} V, so that Z^T M Z = V^T V = I and Z^T A Z = diag (eq. generalizedEVP).
constexpr int kEigMaxSweeps = 50;

__global__ void gen_eig_kernel(const double* __restrict__ Aall, const double* __restrict__ Mall,
                               int nprob, int n, double* __restrict__ Zall,
                               double* __restrict__ lamall, int* __restrict__ err) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int prob = blockIdx.x * (blockDim.x / 32) + warp;
  double* L = sm + (size_t)warp * 3 * n * n;
  double* C = L + n * n;
  double* V = C + n * n;
  if (prob >= nprob) return;  // whole warp exits together
  const double* A = Aall + (size_t)prob * n * n;
  const double* M = Mall + (size_t)prob * n * n;
  for (int e = lane; e < n * n; e += 32) {
    L[e] = M[e];
    C[e] = A[e];
    V[e] = (e / n == e % n) ? 1.0 : 0.0;
  }
  __syncwarp();
  // Cholesky (lower), in place in L
  bool bad = false;
  for (int j = 0; j < n; ++j) {
    if (lane == 0) {
      double s = L[j * n + j];
      for (int m = 0; m < j; ++m) s -= L[j * n + m] * L[j * n + m];
      L[j * n + j] = s > 0.0 ? sqrt(s) : -1.0;
    }
    __syncwarp();
    const double djj = L[j * n + j];
    if (djj <= 0.0) bad = true;
    if (!bad && lane > j && lane < n) {
      double s = L[lane * n + j];
      for (int m = 0; m < j; ++m) s -= L[lane * n + m] * L[j * n + m];
      L[lane * n + j] = s / djj;
    }
    __syncwarp();
  }
  if (bad) {
    if (lane == 0) atomicOr(err, 1);
    return;
  }
  // W = L^{-1} A (lane = column), stored in C
  if (lane < n) {
    for (int i = 0; i < n; ++i) {
      double s = C[i * n + lane];
      for (int m = 0; m < i; ++m) s -= L[i * n + m] * C[m * n + lane];
      C[i * n + lane] = s / L[i * n + i];
    }
  }
  __syncwarp();
  // C = W L^{-T}: row r of C solves L x = (row r of W)^T; lane = row
  if (lane < n) {
    double x[kMaxNP * 2];
    for (int i = 0; i < n; ++i) {
      double s = C[lane * n + i];
      for (int m = 0; m < i; ++m) s -= L[i * n + m] * x[m];
      x[i] = s / L[i * n + i];
    }
    for (int i = 0; i < n; ++i) C[lane * n + i] = x[i];
  }
  __syncwarp();
  // symmetrize
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e % n;
    if (i < j) {
      const double s = 0.5 * (C[i * n + j] + C[j * n + i]);
      C[i * n + j] = s;
      C[j * n + i] = s;
    }
  }
  __syncwarp();
  // cyclic Jacobi
  for (int sweep = 0; sweep < kEigMaxSweeps; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double c = C[i * n + j];
        if (i == j) diag += c * c; else off += c * c;
      }
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = C[p * n + q];
        if (fabs(apq) <= 1e-300) continue;
        const double theta = (C[q * n + q] - C[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        __syncwarp();
        if (lane < n) {  // columns p, q of C and V
          const double cp = C[lane * n + p], cq = C[lane * n + q];
          C[lane * n + p] = c * cp - s * cq;
          C[lane * n + q] = s * cp + c * cq;
          const double vp = V[lane * n + p], vq = V[lane * n + q];
          V[lane * n + p] = c * vp - s * vq;
          V[lane * n + q] = s * vp + c * vq;
        }
        __syncwarp();
        if (lane < n) {  // rows p, q of C
          const double rp = C[p * n + lane], rq = C[q * n + lane];
          C[p * n + lane] = c * rp - s * rq;
          C[q * n + lane] = s * rp + c * rq;
        }
        __syncwarp();
        if (lane == 0) {
          C[p * n + q] = 0.0;
          C[q * n + p] = 0.0;
        }
        __syncwarp();
      }
  }
  __syncwarp();
  // Z = L^{-T} V (lane = column), eigenvalues on the diagonal of C
  if (lane < n) {
    double* Z = Zall + (size_t)prob * n * n;
    double z[kMaxNP * 2];
    for (int i = n - 1; i >= 0; --i) {
      double s = V[i * n + lane];
      for (int m = i + 1; m < n; ++m) s -= L[m * n + i] * z[m];
      z[i] = s / L[i * n + i];
    }
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + lane] = z[i];
    const double lam = C[lane * n + lane];
    lamall[(size_t)prob * n + lane] = lam;
    if (!(lam > 0.0)) atomicOr(err, 2);
  }
}

// 1/(lambda^(1)_i + lambda^(2)_j [+ lambda^(3)_l]) for every subdomain, in the
// subdomain's patch-tensor order (first index fastest).
__global__ void inv_table_kernel(const double* __restrict__ l0, const double* __restrict__ l1,
                                 const double* __restrict__ l2, int dim, int n, int np0, int np1,
                                 int np2, double* __restrict__ inv) {
  const int64_t vol = dim == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const int64_t total = vol * np0 * np1 * (dim == 3 ? np2 : 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sub = e / vol;
    const int64_t loc = e % vol;
    const int px = (int)(sub % np0), py = (int)((sub / np0) % np1);
    const int i = (int)(loc % n), j = (int)((loc / n) % n);
    double s = l0[(size_t)px * n + i] + l1[(size_t)py * n + j];
    if (dim == 3) {
      const int pz = (int)(sub / ((int64_t)np0 * np1));
      const int l = (int)(loc / ((int64_t)n * n));
      s += l2[(size_t)pz * n + l];
    }
    inv[e] = 1.0 / s;
  }
}

// ------------------------------------------------------------ host helpers
static tpss_status build_level(tpss_ctx* ctx, int l) {
  Level& L = ctx->levels[l];
  const int n1 = ctx->n1;
  const double gpk = ctx->gamma_hat * (ctx->penalty_poly == TPSS_PENALTY_KP1SQ
                                           ? (double)(n1 * n1) : (double)(ctx->k * n1));
  L.ncells = 1;
  for (int t = 0; t < ctx->dim; ++t) L.ncells *= L.nc[t];
  L.ndofs = L.ncells * ctx->nloc;
  for (int t = 0; t < ctx->dim; ++t) {
    const int nc = L.nc[t];
    TPSS_TRY(dalloc_t(&L.d_widths[t], nc));
    TPSS_CHECK_CUDA(cudaMemcpyAsync(L.d_widths[t], L.widths[t].data(), nc * sizeof(double),
                                    cudaMemcpyHostToDevice, ctx->stream));
    TPSS_TRY(dalloc_t(&L.op64.M[t], (size_t)nc * n1 * n1));
    TPSS_TRY(dalloc_t(&L.op64.A[t], (size_t)nc * n1 * n1));
    TPSS_TRY(dalloc_t(&L.op64.F[t], (size_t)nc * kFaceCoef));
    level_op1d_kernel<<<nc, 64, 0, ctx->stream>>>(ctx->d_basis, L.d_widths[t], nc, gpk,
                                                  L.op64.M[t], L.op64.A[t], L.op64.F[t]);
    TPSS_CHECK_LAUNCH();
    TPSS_TRY(dalloc_t(&L.op32.M[t], (size_t)nc * n1 * n1));
    TPSS_TRY(dalloc_t(&L.op32.A[t], (size_t)nc * n1 * n1));
    TPSS_TRY(dalloc_t(&L.op32.F[t], (size_t)nc * kFaceCoef));
    TPSS_TRY(convert(L.op64.M[t], L.op32.M[t], (size_t)nc * n1 * n1, ctx->stream));
    TPSS_TRY(convert(L.op64.A[t], L.op32.A[t], (size_t)nc * n1 * n1, ctx->stream));
    TPSS_TRY(convert(L.op64.F[t], L.op32.F[t], (size_t)nc * kFaceCoef, ctx->stream));
  }
  // shared reference vectors (device copies per level keep kernels self-contained)
  const char* base = reinterpret_cast<const char*>(ctx->d_basis);
  const double* d0 = reinterpret_cast<const double*>(base + offsetof(Basis1D, d0));
  const double* d1 = reinterpret_cast<const double*>(base + offsetof(Basis1D, d1));
  const double* pc = reinterpret_cast<const double*>(base + offsetof(Basis1D, Pc));
  TPSS_TRY(dalloc_t(&L.op64.d0, n1));
  TPSS_TRY(dalloc_t(&L.op64.d1, n1));
  TPSS_TRY(dalloc_t(&L.op64.Pc, 2 * n1 * n1));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(L.op64.d0, d0, n1 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(L.op64.d1, d1, n1 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  // Pc is stored with stride kMaxN1*kMaxN1 per child in Basis1D; compact it
  for (int s = 0; s < 2; ++s)
    TPSS_CHECK_CUDA(cudaMemcpyAsync(L.op64.Pc + s * n1 * n1, pc + s * kMaxN1 * kMaxN1,
                                    n1 * n1 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  TPSS_TRY(dalloc_t(&L.op32.d0, n1));
  TPSS_TRY(dalloc_t(&L.op32.d1, n1));
  TPSS_TRY(dalloc_t(&L.op32.Pc, 2 * n1 * n1));
  TPSS_TRY(convert(L.op64.d0, L.op32.d0, n1, ctx->stream));
  TPSS_TRY(convert(L.op64.d1, L.op32.d1, n1, ctx->stream));
  TPSS_TRY(convert(L.op64.Pc, L.op32.Pc, 2 * n1 * n1, ctx->stream));
  return TPSS_OK;
}

static void free_level(Level& L) {
  dfree(L.d_verts);
  dfree(L.d_geo);
  dfree(L.d_geo32);
  for (int t = 0; t < 3; ++t) {
    dfree(L.d_widths[t]);
    dfree(L.op64.M[t]); dfree(L.op64.A[t]); dfree(L.op64.F[t]);
    dfree(L.op32.M[t]); dfree(L.op32.A[t]); dfree(L.op32.F[t]);
  }
  dfree(L.op64.d0); dfree(L.op64.d1); dfree(L.op64.Pc);
  dfree(L.op32.d0); dfree(L.op32.d1); dfree(L.op32.Pc);
  for (int i = 0; i < 5; ++i) {
    dfree(L.t64[i]);
    dfree(L.t32[i]);
  }
}

tpss_status ensure_level_scratch(tpss_ctx* ctx, int level, int nrhs) {
  Level& L = ctx->levels[level];
  if (L.nrhs_cap >= nrhs) return TPSS_OK;
  // scratch is only grown while no work that uses it is in flight
  TPSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < 5; ++i) {
    dfree(L.t64[i]);
    dfree(L.t32[i]);
    L.t64[i] = nullptr;
    L.t32[i] = nullptr;
  }
  L.nrhs_cap = 0;
  const size_t n = (size_t)L.ndofs * nrhs;
  for (int i = 0; i < 5; ++i) {
    TPSS_TRY(dalloc_t(&L.t64[i], n));
    TPSS_TRY(dalloc_t(&L.t32[i], n));
  }
  L.nrhs_cap = nrhs;
  return TPSS_OK;
}

static void free_patches(tpss_patches* P) {
  for (int t = 0; t < 3; ++t) {
    dfree(P->d_A[t]); dfree(P->d_M[t]); dfree(P->d_Z[t]); dfree(P->d_lam[t]);
    dfree(P->d_Z32[t]); dfree(P->d_lam32[t]);
  }
  dfree(P->d_inv);
  dfree(P->d_inv32);
  dfree(P->d_scratch);
  dfree(P->d_add_list);
  dfree(P->d_mul_list);
  dfree(P->d_mul8_list);
  dfree(P->d_flux_list);
  dfree(P->d_lex_list);
  dfree(P->d_plane_list);
  dfree(P->d_bop);
  if (P->h_fail_flag) cudaFreeHost(P->h_fail_flag);
  if (P->aux_stream) cudaStreamDestroy(P->aux_stream);
  if (P->fork_event) cudaEventDestroy(P->fork_event);
  if (P->join_event) cudaEventDestroy(P->join_event);
}

// Is cell m in a subdomain of multiplicative color `color`?  (The same rule
// as the colorings below: vertex v with parity bits and the extra bit
// (sum floor(v_t/2)) mod 2, interior vertices only; cells red-black.)
static bool host_in_color(const int* m, const int* nc, int dim, bool vertex, int color) {
  if (!vertex) {
    int s = 0;
    for (int t = 0; t < dim; ++t) s += m[t];
    return (s & 1) == color;
  }
  int extra = 0;
  for (int t = 0; t < dim; ++t) {
    const int bit = (color >> t) & 1;
    const int v = ((m[t] & 1) == bit) ? m[t] : m[t] + 1;
    if (v < 1 || v > nc[t] - 1) return false;
    extra += v / 2;
  }
  return (extra & 1) == ((color >> dim) & 1);
}

tpss_status create_patches(tpss_ctx* ctx, int level, int kind, int precision, tpss_patches** out);

}  // namespace tpss

using namespace tpss;

extern "C" const char* tpss_last_error(void) { return g_err.c_str(); }

extern "C" tpss_status tpss_create(const tpss_problem_desc* desc, void* cuda_stream, tpss_ctx** out) {
  clear_error();
  TPSS_REQUIRE(desc && out, "tpss_create: null argument");
  *out = nullptr;
  TPSS_REQUIRE(desc->dim == 2 || desc->dim == 3, "tpss_create: dim must be 2 or 3");
  TPSS_REQUIRE(desc->degree >= 1 && desc->degree <= kMaxDegree, "tpss_create: degree must be in 1..15");
  TPSS_REQUIRE(desc->nlevels >= 1 && desc->nlevels <= 12, "tpss_create: nlevels must be in 1..12");
  TPSS_REQUIRE(desc->gamma_hat > 0.0, "tpss_create: gamma_hat must be positive");
  TPSS_REQUIRE(desc->penalty_poly == TPSS_PENALTY_PAPER || desc->penalty_poly == TPSS_PENALTY_KP1SQ,
               "tpss_create: unknown penalty_poly");
  for (int t = 0; t < desc->dim; ++t) {
    TPSS_REQUIRE(desc->ncells[t] >= 1, "tpss_create: ncells must be >= 1");
    TPSS_REQUIRE(desc->widths[t] != nullptr, "tpss_create: widths must not be null");
    for (int c = 0; c < desc->ncells[t]; ++c)
      TPSS_REQUIRE(desc->widths[t][c] > 0.0 && std::isfinite(desc->widths[t][c]),
                   "tpss_create: widths must be positive and finite");
    const long long finest = (long long)desc->ncells[t] << (desc->nlevels - 1);
    TPSS_REQUIRE(finest <= 1024, "tpss_create: at most 1024 cells per direction on the finest level");
  }
  tpss_ctx* ctx = new tpss_ctx();
  ctx->dim = desc->dim;
  ctx->k = desc->degree;
  ctx->n1 = desc->degree + 1;
  ctx->nloc = ctx->dim == 3 ? ctx->n1 * ctx->n1 * ctx->n1 : ctx->n1 * ctx->n1;
  ctx->nlevels = desc->nlevels;
  ctx->gamma_hat = desc->gamma_hat;
  ctx->penalty_poly = desc->penalty_poly;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
  ctx->levels.resize(ctx->nlevels);
  for (int l = 0; l < ctx->nlevels; ++l) {
    Level& L = ctx->levels[l];
    for (int t = 0; t < ctx->dim; ++t) {
      L.nc[t] = desc->ncells[t] << l;
      if (l == 0) {
        L.widths[t].assign(desc->widths[t], desc->widths[t] + desc->ncells[t]);
      } else {
        const std::vector<double>& pw = ctx->levels[l - 1].widths[t];
        L.widths[t].resize(pw.size() * 2);
        for (size_t c = 0; c < pw.size(); ++c) L.widths[t][2 * c] = L.widths[t][2 * c + 1] = 0.5 * pw[c];
      }
    }
  }
  tpss_status st = TPSS_OK;
  auto fail = [&](tpss_status s) {
    tpss_destroy(ctx);
    return s;
  };
  if ((st = dalloc_t(&ctx->d_basis, 1)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&ctx->d_scalars, 64)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&ctx->d_partials, 4096)) != TPSS_OK) return fail(st);
  setup_basis_kernel<<<1, kBasisThreads, 0, ctx->stream>>>(ctx->d_basis, ctx->k);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("setup_basis_kernel launch failed");
    return fail(TPSS_ECUDA);
  }
  for (int l = 0; l < ctx->nlevels; ++l)
    if ((st = build_level(ctx, l)) != TPSS_OK) return fail(st);
  cudaError_t e = cudaMemcpyAsync(&ctx->h_basis, ctx->d_basis, sizeof(Basis1D), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    set_error(std::string("tpss_create: ") + cudaGetErrorString(e));
    return fail(TPSS_ECUDA);
  }
  if (ctx->h_basis.status != 0) {
    set_error("tpss_create: Newton iteration for the quadrature nodes did not converge");
    return fail(TPSS_ENUMERIC);
  }
  *out = ctx;
  return TPSS_OK;
}

extern "C" tpss_status tpss_destroy(tpss_ctx* ctx) {
  if (!ctx) return TPSS_OK;
  cudaStreamSynchronize(ctx->stream);
  destroy_mg(ctx);
  for (auto& L : ctx->levels) free_level(L);
  dfree(ctx->d_basis);
  dfree(ctx->d_scalars);
  dfree(ctx->d_partials);
  delete ctx;
  return TPSS_OK;
}

extern "C" tpss_status tpss_level_info(const tpss_ctx* ctx, int level, int64_t* ndofs, int ncells[3]) {
  clear_error();
  TPSS_REQUIRE(ctx, "tpss_level_info: null context");
  TPSS_REQUIRE(level >= 0 && level < ctx->nlevels, "tpss_level_info: level out of range");
  const Level& L = ctx->levels[level];
  if (ndofs) *ndofs = L.ndofs;
  if (ncells)
    for (int t = 0; t < 3; ++t) ncells[t] = t < ctx->dim ? L.nc[t] : 1;
  return TPSS_OK;
}

namespace tpss {

// Per multiplicative color, the cells outside the color that share a face
// with a cell of the color, with the mask of those faces.
static tpss_status build_flux_lists(tpss_patches* P, int dim, bool vertex) {
  const Level& L = P->ctx->levels[P->level];
  int nc[3] = {1, 1, 1};
  for (int t = 0; t < dim; ++t) nc[t] = L.nc[t];
  const int ncolors = vertex ? 1 << (dim + 1) : 2;
  std::vector<int2> flat;
  P->flux_offsets.assign(1, 0);
  for (int c = 0; c < ncolors; ++c) {
    for (int64_t cell = 0; cell < L.ncells; ++cell) {
      int m[3] = {(int)(cell % nc[0]), (int)((cell / nc[0]) % nc[1]), (int)(cell / ((int64_t)nc[0] * nc[1]))};
      if (host_in_color(m, nc, dim, vertex, c)) continue;
      int mask = 0;
      for (int t = 0; t < dim; ++t)
        for (int side = 0; side < 2; ++side) {
          int mn[3] = {m[0], m[1], m[2]};
          mn[t] += side ? 1 : -1;
          if (mn[t] < 0 || mn[t] >= nc[t]) continue;
          if (host_in_color(mn, nc, dim, vertex, c)) mask |= 1 << (2 * t + side);
        }
      if (mask) flat.push_back(make_int2((int)cell, mask));
    }
    P->flux_offsets.push_back((int)flat.size());
  }
  TPSS_TRY(dalloc_t(&P->d_flux_list, flat.size()));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(P->d_flux_list, flat.data(), flat.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                  P->ctx->stream));
  TPSS_CHECK_CUDA(cudaStreamSynchronize(P->ctx->stream));   // flat goes out of scope
  return TPSS_OK;
}

tpss_status create_patches(tpss_ctx* ctx, int level, int kind, int precision, tpss_patches** out) {
  const Level& L = ctx->levels[level];
  const int d = ctx->dim, n1 = ctx->n1;
  tpss_patches* P = new tpss_patches();
  P->ctx = ctx;
  P->level = level;
  P->kind = kind;
  P->precision = precision;
  P->n = kind == TPSS_VERTEX_PATCH ? 2 * n1 : n1;
  const int n = P->n;
  // BF16 / TF32 3D vertex patches: the tcgen05 column walk by default where
  // it is the fastest measured schedule (n >= 10, k >= 4); colored launches below
  if ((precision == TPSS_BF16 || precision == TPSS_TF32) && d == 3 && kind == TPSS_VERTEX_PATCH && !ctx->mapped &&
      n >= 10)
    P->additive_schedule = TPSS_ADDITIVE_TCGEN05;
  P->nsub = 1;
  for (int t = 0; t < d; ++t) {
    P->npos[t] = kind == TPSS_VERTEX_PATCH ? L.nc[t] - 1 : L.nc[t];
    P->nsub *= P->npos[t];
  }
  tpss_status st;
  auto fail = [&](tpss_status s) {
    free_patches(P);
    delete P;
    return s;
  };
  int* d_err = nullptr;
  if ((st = dalloc_t(&d_err, 1)) != TPSS_OK) return fail(st);
  cudaMemsetAsync(d_err, 0, sizeof(int), ctx->stream);
  if (ctx->mapped) {   // surrogate cell solvers, eigendata per cell (mapped.cu)
    P->per_sub = 1;
    P->mult_update = 0;
    if ((st = mapped_cell_eigendata(ctx, P, d_err)) != TPSS_OK) {
      dfree(d_err);
      return fail(st);
    }
    if (precision != TPSS_FP64) {   // FP32 copies: the SIMT patch kernel (x = 0) and the fused kernel
      const size_t nn = (size_t)P->nsub * n * n, vol = (size_t)P->nsub * (d == 3 ? n * n * n : n * n);
      for (int t = 0; t < d; ++t) {
        if ((st = dalloc_t(&P->d_Z32[t], nn)) != TPSS_OK) return fail(st);
        if ((st = dalloc_t(&P->d_lam32[t], (size_t)P->nsub * n)) != TPSS_OK) return fail(st);
        convert(P->d_Z[t], P->d_Z32[t], nn, ctx->stream);
        convert(P->d_lam[t], P->d_lam32[t], (size_t)P->nsub * n, ctx->stream);
      }
      if ((st = dalloc_t(&P->d_inv32, vol)) != TPSS_OK) return fail(st);
      convert(P->d_inv, P->d_inv32, vol, ctx->stream);
    }
  }
  for (int t = 0; t < d && !ctx->mapped; ++t) {
    const int np = P->npos[t];
    if ((st = dalloc_t(&P->d_A[t], (size_t)np * n * n)) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&P->d_M[t], (size_t)np * n * n)) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&P->d_Z[t], (size_t)np * n * n)) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&P->d_lam[t], (size_t)np * n)) != TPSS_OK) return fail(st);
    patch_matrices_kernel<<<np, 128, 0, ctx->stream>>>(ctx->d_basis, L.op64.M[t], L.op64.A[t], L.op64.F[t],
                                                       np, kind == TPSS_VERTEX_PATCH, P->d_A[t], P->d_M[t]);
    const int warps = n > 16 ? 1 : 4;
    const size_t smem = (size_t)warps * 3 * n * n * sizeof(double);
    gen_eig_kernel<<<(np + warps - 1) / warps, warps * 32, smem, ctx->stream>>>(
        P->d_A[t], P->d_M[t], np, n, P->d_Z[t], P->d_lam[t], d_err);
    if (cudaGetLastError() != cudaSuccess) {
      dfree(d_err);
      set_error("tpss_setup_patches: eigen kernel launch failed");
      return fail(TPSS_ECUDA);
    }
    if (precision != TPSS_FP64) {
      if ((st = dalloc_t(&P->d_Z32[t], (size_t)np * n * n)) != TPSS_OK) return fail(st);
      if ((st = dalloc_t(&P->d_lam32[t], (size_t)np * n)) != TPSS_OK) return fail(st);
      convert(P->d_Z[t], P->d_Z32[t], (size_t)np * n * n, ctx->stream);
      convert(P->d_lam[t], P->d_lam32[t], (size_t)np * n, ctx->stream);
    }
  }
  // operands of the tcgen05 smoother (every direction's FP32 eigenvectors are converted by now)
  if (!ctx->mapped && (precision == TPSS_BF16 || precision == TPSS_TF32) && (st = tc05_prepare(P)) != TPSS_OK)
    return fail(st);
  // second stream of the additive passes (second half of the right-hand sides)
  if (cudaStreamCreateWithFlags(&P->aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->fork_event, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->join_event, cudaEventDisableTiming) != cudaSuccess) {
    set_error("tpss_setup_patches: stream or event creation failed");
    return fail(TPSS_ECUDA);
  }
  const bool large = d == 3 && n > kMaxSharedPatchN;
  if (ctx->mapped) {
    // inverse table already built per cell
  } else if (large) {   // per-CTA tensor slabs of the large-patch kernel (no inverse table)
    if ((st = patch_large_ctas(n, ctx->num_sms, &P->scratch_ctas)) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&P->d_scratch, (size_t)P->scratch_ctas * n * n * n)) != TPSS_OK) return fail(st);
  } else if (precision == TPSS_FP64) {
    const size_t vol = d == 3 ? (size_t)n * n * n : (size_t)n * n;
    if ((st = dalloc_t(&P->d_inv, vol * P->nsub)) != TPSS_OK) return fail(st);
    inv_table_kernel<<<2048, 256, 0, ctx->stream>>>(P->d_lam[0], P->d_lam[1], d == 3 ? P->d_lam[2] : nullptr,
                                                    d, n, P->npos[0], P->npos[1], d == 3 ? P->npos[2] : 1,
                                                    P->d_inv);
  }
  // colorings (Sec. 2.3), built on the host as packed position lists
  const int nz = d == 3 ? P->npos[2] : 1;
  auto build = [&](auto colorf, int ncolors, int** dlist, std::vector<int>& offs) -> tpss_status {
    std::vector<std::vector<int>> by(ncolors);
    for (int pz = 0; pz < nz; ++pz)
      for (int py = 0; py < P->npos[1]; ++py)
        for (int px = 0; px < P->npos[0]; ++px) by[colorf(px, py, pz)].push_back(pack_pos(px, py, pz));
    std::vector<int> flat;
    offs.assign(1, 0);
    for (auto& v : by) {
      flat.insert(flat.end(), v.begin(), v.end());
      offs.push_back((int)flat.size());
    }
    TPSS_TRY(dalloc_t(dlist, flat.size()));
    TPSS_CHECK_CUDA(cudaMemcpyAsync(*dlist, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    ctx->stream));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));  // flat goes out of scope
    return TPSS_OK;
  };
  if (kind == TPSS_VERTEX_PATCH) {
    // vertex v_t = p_t + 1; additive: parity bits; multiplicative: + (sum floor(v_t/2)) mod 2
    auto add = [&](int px, int py, int pz) {
      return ((px + 1) & 1) | (((py + 1) & 1) << 1) | (d == 3 ? (((pz + 1) & 1) << 2) : 0);
    };
    auto mul = [&](int px, int py, int pz) {
      const int extra = ((px + 1) / 2 + (py + 1) / 2 + (d == 3 ? (pz + 1) / 2 : 0)) & 1;
      return add(px, py, pz) | (extra << d);
    };
    if ((st = build(add, 1 << d, &P->d_add_list, P->add_offsets)) != TPSS_OK) return fail(st);
    if ((st = build(mul, 1 << (d + 1), &P->d_mul_list, P->mul_offsets)) != TPSS_OK) return fail(st);
    if ((st = build(add, 1 << d, &P->d_mul8_list, P->mul8_offsets)) != TPSS_OK) return fail(st);
    P->mul_colors_default = 1 << (d + 1);
    if ((st = build_flux_lists(P, d, true)) != TPSS_OK) return fail(st);
  } else {
    auto one = [&](int, int, int) { return 0; };
    auto rb = [&](int px, int py, int pz) { return (px + py + pz) & 1; };
    if ((st = build(one, 1, &P->d_add_list, P->add_offsets)) != TPSS_OK) return fail(st);
    if ((st = build(rb, 2, &P->d_mul_list, P->mul_offsets)) != TPSS_OK) return fail(st);
    P->mul_colors_default = 2;
    if ((st = build_flux_lists(P, d, false)) != TPSS_OK) return fail(st);
  }
  P->mul_colors_active = P->mul_colors_default;
  {
    std::vector<int> lex_offsets;
    auto one = [&](int, int, int) { return 0; };
    if ((st = build(one, 1, &P->d_lex_list, lex_offsets)) != TPSS_OK) return fail(st);
  }
  if (kind == TPSS_VERTEX_PATCH && d == 3) {
    // plane by plane: the 4 additive colors of plane p_z, ((p_x+1)&1) | ((p_y+1)&1) << 1
    auto plane_color = [&](int px, int py, int pz) { return 4 * pz + (((px + 1) & 1) | (((py + 1) & 1) << 1)); };
    if ((st = build(plane_color, 4 * P->npos[2], &P->d_plane_list, P->plane_offsets)) != TPSS_OK) return fail(st);
  }
  int h_err = 0;
  cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  dfree(d_err);
  if (e != cudaSuccess) {
    set_error(std::string("tpss_setup_patches: ") + cudaGetErrorString(e));
    return fail(TPSS_ECUDA);
  }
  if (h_err) {
    set_error(h_err & 1 ? "tpss_setup_patches: 1D mass matrix not positive definite"
                        : "tpss_setup_patches: non-positive generalized eigenvalue (penalty too small?)");
    return fail(TPSS_ENUMERIC);
  }
  *out = P;
  return TPSS_OK;
}

}  // namespace tpss

extern "C" tpss_status tpss_setup_patches(tpss_ctx* ctx, int level, int kind, int precision,
                                          tpss_patches** out) {
  clear_error();
  TPSS_REQUIRE(ctx && out, "tpss_setup_patches: null argument");
  *out = nullptr;
  TPSS_REQUIRE(level >= 0 && level < ctx->nlevels, "tpss_setup_patches: level out of range");
  TPSS_REQUIRE(kind == TPSS_CELL || kind == TPSS_VERTEX_PATCH, "tpss_setup_patches: unknown kind");
  TPSS_REQUIRE(precision >= TPSS_FP64 && precision <= TPSS_BF16, "tpss_setup_patches: unknown precision");
  TPSS_REQUIRE(precision == TPSS_FP64 || ctx->k <= kMaxMixedDegree,
               "tpss_setup_patches: FP32/TF32/BF16 smoothers support degrees up to 7");
  TPSS_REQUIRE(!ctx->mapped || (kind == TPSS_CELL && (precision == TPSS_FP64 || precision == TPSS_FP32)),
               "tpss_setup_patches: mapped meshes support FP64 and FP32 cell patches (surrogate solvers) only");
  if (kind == TPSS_VERTEX_PATCH)
    for (int t = 0; t < ctx->dim; ++t)
      TPSS_REQUIRE(ctx->levels[level].nc[t] >= 2, "tpss_setup_patches: vertex patches need >= 2 cells per direction");
  return create_patches(ctx, level, kind, precision, out);
}

extern "C" tpss_status tpss_patches_destroy(tpss_patches* P) {
  if (!P) return TPSS_OK;
  cudaStreamSynchronize(P->ctx->stream);
  free_patches(P);
  delete P;
  return TPSS_OK;
}

extern "C" tpss_status tpss_patches_info(const tpss_patches* P, int* n, int npos[3], int64_t* nsub,
                                         int* ncolors_mult) {
  clear_error();
  TPSS_REQUIRE(P, "tpss_patches_info: null patches");
  if (n) *n = P->n;
  if (npos)
    for (int t = 0; t < 3; ++t) npos[t] = P->npos[t];
  if (nsub) *nsub = P->nsub;
  if (ncolors_mult) *ncolors_mult = P->mul_colors_active;
  return TPSS_OK;
}

extern "C" tpss_status tpss_patches_eigendata(const tpss_patches* P, int t, int pos, double* A, double* M,
                                              double* Z, double* lambda) {
  clear_error();
  TPSS_REQUIRE(P, "tpss_patches_eigendata: null patches");
  TPSS_REQUIRE(t >= 0 && t < P->ctx->dim, "tpss_patches_eigendata: direction out of range");
  TPSS_REQUIRE(pos >= 0 && pos < (P->per_sub ? P->nsub : P->npos[t]),
               "tpss_patches_eigendata: position out of range");
  const int n = P->n;
  const size_t off = (size_t)pos * n * n;
  cudaStream_t s = P->ctx->stream;
  if (A) TPSS_CHECK_CUDA(cudaMemcpyAsync(A, P->d_A[t] + off, n * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (M) TPSS_CHECK_CUDA(cudaMemcpyAsync(M, P->d_M[t] + off, n * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (Z) TPSS_CHECK_CUDA(cudaMemcpyAsync(Z, P->d_Z[t] + off, n * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (lambda)
    TPSS_CHECK_CUDA(cudaMemcpyAsync(lambda, P->d_lam[t] + (size_t)pos * n, n * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
  TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
  return TPSS_OK;
}

extern "C" tpss_status tpss_patches_set_mult_colors(tpss_patches* P, int ncolors) {
  clear_error();
  TPSS_REQUIRE(P, "tpss_patches_set_mult_colors: null patches");
  if (ncolors == 0) ncolors = P->mul_colors_default;
  const int d = P->ctx->dim;
  if (P->kind == TPSS_VERTEX_PATCH) {
    TPSS_REQUIRE(ncolors == (1 << (d + 1)) || ncolors == (1 << d),
                 "tpss_patches_set_mult_colors: vertex patches take 2^(d+1) or 2^d colors");
  } else {
    TPSS_REQUIRE(ncolors == 2, "tpss_patches_set_mult_colors: cells take 2 colors");
  }
  P->mul_colors_active = ncolors;
  return TPSS_OK;
}

extern "C" tpss_status tpss_patches_set_large_cluster(tpss_patches* P, int ctas) {
  clear_error();
  TPSS_REQUIRE(P, "tpss_patches_set_large_cluster: null patches");
  TPSS_REQUIRE(ctas == 0 || ctas == 1 || ctas == 2 || ctas == 4 || ctas == 8,
               "tpss_patches_set_large_cluster: ctas must be 0 (automatic), 1, 2, 4 or 8");
  P->large_cluster = ctas;
  return TPSS_OK;
}

extern "C" tpss_status tpss_patches_test_wait_expiry(tpss_patches* P) {
  clear_error();
  TPSS_REQUIRE(P, "tpss_patches_test_wait_expiry: null patches");
  TPSS_REQUIRE(P->d_bop != nullptr,
               "tpss_patches_test_wait_expiry: not a tcgen05 patch set (BF16 or TF32 3D vertex patches)");
  P->expire_test = 1;
  return TPSS_OK;
}

extern "C" tpss_status tpss_patches_set_additive_schedule(tpss_patches* P, int schedule) {
  clear_error();
  TPSS_REQUIRE(P, "tpss_patches_set_additive_schedule: null patches");
  TPSS_REQUIRE(schedule == TPSS_ADDITIVE_COLORS || schedule == TPSS_ADDITIVE_PLANES ||
                   schedule == TPSS_ADDITIVE_ATOMIC || schedule == TPSS_ADDITIVE_COLUMNS ||
                   schedule == TPSS_ADDITIVE_TCGEN05,
               "tpss_patches_set_additive_schedule: unknown schedule");
  P->additive_schedule = schedule;
  return TPSS_OK;
}

extern "C" tpss_status tpss_patches_set_mult_residual(tpss_patches* P, int mode) {
  clear_error();
  TPSS_REQUIRE(P, "tpss_patches_set_mult_residual: null patches");
  TPSS_REQUIRE(mode == TPSS_MULT_RESIDUAL_UPDATE || mode == TPSS_MULT_RESIDUAL_FULL,
               "tpss_patches_set_mult_residual: mode must be 0 (update) or 1 (full)");
  TPSS_REQUIRE(!P->per_sub || mode == TPSS_MULT_RESIDUAL_FULL,
               "tpss_patches_set_mult_residual: surrogate cell solvers recompute the full residual");
  P->mult_update = mode == TPSS_MULT_RESIDUAL_UPDATE ? 1 : 0;
  return TPSS_OK;
}
