// SIPG on 3D meshes of trilinear hexahedra and their Cartesian-surrogate cell
// solvers (Sec. 4, eq. schwarzproj, eq. avglength); the 2D counterpart and
// the common entry points are in mapped.cu.
//
// Mesh: a structured vertex array [(nz+1)][(ny+1)][(nx+1)] of (x, y, z),
// x index fastest; cell (i, j, l) has the corners c = a0 + 2 a1 + 4 a2 at
// vertex (i + a0, j + a1, l + a2) and the trilinear map
//   x(xi) = sum_c v_c prod_t (a_t xi_t + (1 - a_t)(1 - xi_t)).
// Refinement: a new vertex between old vertices along the directions of a
// set of m directions is the mean of the 2^m old vertices around it, summed
// in corner order (first direction fastest).
//
// Operator (eq. bfsipg on the mapped cells, matrix-free): one CTA slot per
// cell with (k+1)^3 threads.  Per cell, precomputed once per level
// (Geo3Layout):
//   C  [6][n1^3]     w |det J| J^{-1} J^{-T} at the Gauss points (c00 c01 c02 c11 c12 c22)
//   A  [6][3][n1^2]  J^{-1} n at the Gauss points of face f = 2 t + side, n
//                    the outward unit normal J^{-T} e_t / |J^{-T} e_t| (+-)
//   W  [6][n1^2]     w_u w_v |det J| |J^{-T} e_t| (Nanson's surface element)
//   S  [6]           the penalty of the face, gamma_hat P(k)(|e|/|K| + |e|/|N|)
//                    (h = |K| / |e|, boundary: 2 |e| / |K|)
// Cell term: reference gradients at the Gauss points by three sum-
// factorization stages (x: D, V; y: V, D, V; z: V, V, D), the metric, and
// the transposed stages.  Face terms (both sides of each of the 6 faces):
// traces and reference normal-derivative planes of the cell and of its
// neighbour, interpolated to the face's Gauss points in two stages (along
// u, then v; u < v the face's directions), the coefficients
//   v:       W (gamma/2 [u] - (d_n u^K + d_n u^N)/2)     (interior)
//   d_n v:   -W [u] / 2                                    (interior)
//   boundary: W (gamma u - d_n u) and -W u,  d_n u = (J^{-1} n) . g_ref u,
// and the transposed two stages onto the cell's face-adjacent test functions.
#include <algorithm>
#include <cmath>

#include "tpss_internal.cuh"

namespace tpss {

namespace {

struct Hex {
  double3 v[8];
};

// J[r][s] = d x_r / d xi_s at xi; returns det J and writes J^{-1} (row-major)
__device__ __forceinline__ double hex_inverse_jacobian(const Hex& H, double x0, double x1, double x2, double Ji[9]) {
  double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const double xi[3] = {x0, x1, x2};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    double f[3], df[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int a = (c >> t) & 1;
      f[t] = a ? xi[t] : 1.0 - xi[t];
      df[t] = a ? 1.0 : -1.0;
    }
    const double g0 = df[0] * f[1] * f[2], g1 = f[0] * df[1] * f[2], g2 = f[0] * f[1] * df[2];
    const double vr[3] = {H.v[c].x, H.v[c].y, H.v[c].z};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      J[3 * r + 0] += vr[r] * g0;
      J[3 * r + 1] += vr[r] * g1;
      J[3 * r + 2] += vr[r] * g2;
    }
  }
  const double m00 = J[4] * J[8] - J[5] * J[7], m01 = J[5] * J[6] - J[3] * J[8], m02 = J[3] * J[7] - J[4] * J[6];
  const double det = J[0] * m00 + J[1] * m01 + J[2] * m02;
  const double inv = 1.0 / det;
  Ji[0] = m00 * inv;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) * inv;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) * inv;
  Ji[3] = m01 * inv;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) * inv;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) * inv;
  Ji[6] = m02 * inv;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) * inv;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) * inv;
  return det;
}

__device__ __forceinline__ Hex load_hex(const double3* __restrict__ V, int nx, int ny, int i, int j, int l) {
  Hex H;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    H.v[c] = V[((int64_t)(l + (c >> 2)) * (ny + 1) + (j + ((c >> 1) & 1))) * (nx + 1) + i + (c & 1)];
  return H;
}

__device__ __forceinline__ double dist3(double3 a, double3 b) {
  const double dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
  return sqrt(dx * dx + dy * dy + dz * dz);
}

}  // namespace

struct Geo3Layout {
  int n1, nv, nf, C, A, W, S, G;
  __host__ __device__ explicit Geo3Layout(int n)
      : n1(n), nv(n * n * n), nf(n * n), C(0), A(6 * n * n * n), W(6 * n * n * n + 18 * n * n),
        S(6 * n * n * n + 24 * n * n), G(6 * n * n * n + 24 * n * n + 6) {}
};

// ---------------------------------------------------------------- meshes
__global__ void refine_vertices3_kernel(const double3* __restrict__ V, int nx, int ny, int nz,
                                        double3* __restrict__ F) {
  const int fx = 2 * nx + 1, fy = 2 * ny + 1, fz = 2 * nz + 1;
  const int64_t total = (int64_t)fx * fy * fz;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int f[3] = {(int)(e % fx), (int)((e / fx) % fy), (int)(e / ((int64_t)fx * fy))};
    int m = 0;
    double3 acc = make_double3(0.0, 0.0, 0.0);
    bool first = true;
    for (int c = 0; c < 8; ++c) {
      int a[3];
      bool skip = false;
      for (int t = 0; t < 3; ++t) {
        a[t] = (c >> t) & 1;
        if (a[t] && !(f[t] & 1)) skip = true;
      }
      if (skip) continue;
      const double3 v = V[((int64_t)((f[2] >> 1) + a[2]) * (ny + 1) + (f[1] >> 1) + a[1]) * (nx + 1) + (f[0] >> 1) + a[0]];
      if (first) {
        acc = v;
        first = false;
      } else {
        acc.x = acc.x + v.x;
        acc.y = acc.y + v.y;
        acc.z = acc.z + v.z;
      }
    }
    for (int t = 0; t < 3; ++t) m += f[t] & 1;
    const double s = m == 0 ? 1.0 : m == 1 ? 0.5 : m == 2 ? 0.25 : 0.125;
    F[e] = make_double3(s * acc.x, s * acc.y, s * acc.z);
  }
}

tpss_status mapped3_refine(const double* coarse, int nx, int ny, int nz, double* fine, cudaStream_t s) {
  const int64_t n = (int64_t)(2 * nx + 1) * (2 * ny + 1) * (2 * nz + 1);
  refine_vertices3_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
      reinterpret_cast<const double3*>(coarse), nx, ny, nz, reinterpret_cast<double3*>(fine));
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// -------------------------------------------------------------- geometry
// |K| by the (k+1)^3 Gauss rule (exact for a trilinear det J)
__global__ void hex_volume_kernel(const Basis1D* __restrict__ B, const double3* __restrict__ V, int nx, int ny, int nz,
                                  double* __restrict__ vol) {
  const int n1 = B->n1;
  const int64_t nc = (int64_t)nx * ny * nz;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const Hex H = load_hex(V, nx, ny, (int)(c % nx), (int)((c / nx) % ny), (int)(c / ((int64_t)nx * ny)));
    double s = 0.0;
    for (int q = 0; q < n1 * n1 * n1; ++q) {
      const int q0 = q % n1, q1 = (q / n1) % n1, q2 = q / (n1 * n1);
      double Ji[9];
      s += B->wq[q0] * B->wq[q1] * B->wq[q2] * fabs(hex_inverse_jacobian(H, B->xq[q0], B->xq[q1], B->xq[q2], Ji));
    }
    vol[c] = s;
  }
}

__global__ void mapped3_geometry_kernel(const Basis1D* __restrict__ B, const double3* __restrict__ V, int nx, int ny,
                                        int nz, double gpk, const double* __restrict__ vol, double* __restrict__ geo) {
  const int n1 = B->n1;
  const Geo3Layout g(n1);
  const int64_t c = blockIdx.x;
  const int ci[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((int64_t)nx * ny))};
  const int nc[3] = {nx, ny, nz};
  const Hex H = load_hex(V, nx, ny, ci[0], ci[1], ci[2]);
  double* out = geo + c * g.G;
  for (int e = threadIdx.x; e < g.nv; e += blockDim.x) {
    const int q0 = e % n1, q1 = (e / n1) % n1, q2 = e / (n1 * n1);
    double Ji[9];
    const double det = hex_inverse_jacobian(H, B->xq[q0], B->xq[q1], B->xq[q2], Ji);
    const double w = B->wq[q0] * B->wq[q1] * B->wq[q2] * fabs(det);
    // (J^{-1} J^{-T})_{rs} = sum_m Ji[r][m] Ji[s][m]
    auto m = [&](int r, int s) { return Ji[3 * r] * Ji[3 * s] + Ji[3 * r + 1] * Ji[3 * s + 1] + Ji[3 * r + 2] * Ji[3 * s + 2]; };
    out[g.C + 0 * g.nv + e] = w * m(0, 0);
    out[g.C + 1 * g.nv + e] = w * m(0, 1);
    out[g.C + 2 * g.nv + e] = w * m(0, 2);
    out[g.C + 3 * g.nv + e] = w * m(1, 1);
    out[g.C + 4 * g.nv + e] = w * m(1, 2);
    out[g.C + 5 * g.nv + e] = w * m(2, 2);
  }
  for (int e = threadIdx.x; e < 6 * g.nf; e += blockDim.x) {
    const int f = e / g.nf, p = e % g.nf, t = f >> 1, side = f & 1;
    const int u = t == 0 ? 1 : 0, v = t == 2 ? 1 : 2;
    double xi[3];
    xi[t] = (double)side;
    xi[u] = B->xq[p % n1];
    xi[v] = B->xq[p / n1];
    double Ji[9];
    const double det = hex_inverse_jacobian(H, xi[0], xi[1], xi[2], Ji);
    // J^{-T} e_t = row t of J^{-1}
    const double gx = Ji[3 * t], gy = Ji[3 * t + 1], gz = Ji[3 * t + 2];
    const double gn = sqrt(gx * gx + gy * gy + gz * gz);
    const double sg = side ? 1.0 : -1.0;
    const double nxv = sg * gx / gn, nyv = sg * gy / gn, nzv = sg * gz / gn;
    for (int r = 0; r < 3; ++r)
      out[g.A + (f * 3 + r) * g.nf + p] = Ji[3 * r] * nxv + Ji[3 * r + 1] * nyv + Ji[3 * r + 2] * nzv;
    out[g.W + f * g.nf + p] = B->wq[p % n1] * B->wq[p / n1] * fabs(det) * gn;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int f = threadIdx.x, t = f >> 1, side = f & 1;
    double a = 0.0;
    for (int p = 0; p < g.nf; ++p) a += out[g.W + f * g.nf + p];
    int nb[3] = {ci[0], ci[1], ci[2]};
    nb[t] += side ? 1 : -1;
    const bool interior = nb[t] >= 0 && nb[t] < nc[t];
    const double vk = vol[c];
    out[g.S + f] = interior ? gpk * (a / vk + a / vol[((int64_t)nb[2] * ny + nb[1]) * nx + nb[0]]) : gpk * (2.0 * a / vk);
  }
}

tpss_status mapped3_setup_level(tpss_ctx* ctx, int level, double gpk) {
  Level& L = ctx->levels[level];
  const int nx = L.nc[0], ny = L.nc[1], nz = L.nc[2];
  const double3* V = reinterpret_cast<const double3*>(L.d_verts);
  double* vol = nullptr;
  TPSS_TRY(dalloc_t(&vol, (size_t)L.ncells));
  tpss_status st = dalloc_t(&L.d_geo, (size_t)L.ncells * Geo3Layout(ctx->n1).G);
  if (st == TPSS_OK) {
    hex_volume_kernel<<<(unsigned)std::min<int64_t>((L.ncells + 127) / 128, 8192), 128, 0, ctx->stream>>>(
        ctx->d_basis, V, nx, ny, nz, vol);
    mapped3_geometry_kernel<<<(unsigned)L.ncells, 128, 0, ctx->stream>>>(ctx->d_basis, V, nx, ny, nz, gpk, vol,
                                                                           L.d_geo);
  }
  const cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(ctx->stream);   // vol is freed below
  dfree(vol);
  if (st != TPSS_OK) return st;
  if (e != cudaSuccess) {
    set_error(std::string("mapped geometry: ") + cudaGetErrorString(e));
    return TPSS_ECUDA;
  }
  return TPSS_OK;
}

// -------------------------------------------------------------- operator
template <int N1>
struct Mapped3Shape {
  static constexpr int NV = N1 * N1 * N1, NF = N1 * N1;
  static constexpr int CPB = 256 / NV > 0 ? 256 / NV : 1;
  static constexpr int THREADS = CPB * NV;
  static constexpr int G = 6 * NV + 24 * NF + 6;    // Geo3Layout(N1).G
  // per-cell slot (Ts): U (own + 6 neighbours), 6 cell scratch arrays,
  // face arrays: set A (6 x [6][NF]) and set B (4 x [6][NF])
  static constexpr int U = 0, SC = 7 * NV, FA = 13 * NV, FB = 13 * NV + 36 * NF;
  static constexpr int SLOT = 13 * NV + 60 * NF;
  static constexpr int TABLES = 2 * NF + 4 * N1;
};

template <typename T>
struct Mapped3ArgsT {
  const T* u;
  T* out;
  const T* rhs;        // not null: out = rhs - A u
  const T* geo;        // [ncells][G]
  const Basis1D* B;
  int nx, ny, nz;
  int64_t ncells, ndofs;
};

// tables in shared memory: Vq, Dq (n1^2), d0, d1 (n1)
template <int N1, typename T>
__device__ __forceinline__ void mapped3_tables(const Basis1D* __restrict__ B, T* sm) {
  constexpr int NF = N1 * N1;
  for (int e = threadIdx.x; e < NF; e += blockDim.x) {
    sm[e] = (T)B->Vq[e];
    sm[NF + e] = (T)B->Dq[e];
  }
  for (int e = threadIdx.x; e < N1; e += blockDim.x) {
    sm[2 * NF + e] = (T)B->d0[e];
    sm[2 * NF + N1 + e] = (T)B->d1[e];
  }
}

// (A u)_K at the local DoF tid of cell `cell`; every thread of the CTA calls
// it (it synchronizes the CTA), Wk is the cell's slot (Wk + S::U keeps u_K)
template <int N1, typename T>
__device__ __forceinline__ T mapped3_cell_apply(const Mapped3ArgsT<T>& a, T* sm, T* Wk, int64_t cell, bool active,
                                                int tid) {
  using S = Mapped3Shape<N1>;
  constexpr int NV = S::NV, NF = S::NF, K = N1 - 1, G = S::G;
  constexpr int GA = 6 * NV, GW = 6 * NV + 18 * NF, GS = 6 * NV + 24 * NF;   // Geo3Layout offsets
  T* Vq = sm;
  T* Dq = Vq + NF;
  T* dd = Dq + NF;   // d0 then d1
  T* U = Wk + S::U;
  T* sc = Wk + S::SC;       // 6 x NV
  T* fa = Wk + S::FA;       // 6 x 6 NF
  T* fb = Wk + S::FB;       // 4 x 6 NF
  const int ci0 = active ? (int)(cell % a.nx) : 0, ci1 = active ? (int)((cell / a.nx) % a.ny) : 0;
  const int ci2 = active ? (int)(cell / ((int64_t)a.nx * a.ny)) : 0;
  const int hasm = (ci0 > 0 ? 1 : 0) | (ci0 + 1 < a.nx ? 2 : 0) | (ci1 > 0 ? 4 : 0) | (ci1 + 1 < a.ny ? 8 : 0) |
                   (ci2 > 0 ? 16 : 0) | (ci2 + 1 < a.nz ? 32 : 0);
  auto has = [&](int f) { return ((hasm >> f) & 1) != 0; };
  const int64_t sxy = (int64_t)a.nx * a.ny;
  auto nbr = [&](int f) -> int64_t {
    const int64_t step = (f >> 1) == 0 ? 1 : (f >> 1) == 1 ? a.nx : sxy;
    return cell + ((f & 1) ? step : -step);
  };
  // local index with i_t = it and (j, l) along the face's directions (u < v)
  auto lidx = [](int t, int it, int j, int l) {
    return t == 0 ? it + N1 * (j + N1 * l) : t == 1 ? j + N1 * (it + N1 * l) : j + N1 * (l + N1 * it);
  };
  const int64_t vbase = (int64_t)blockIdx.y * a.ndofs;
  const T* gc = a.geo + cell * G;
  const int i0 = tid % N1, i1 = (tid / N1) % N1, i2 = tid / NF;

  // ---- P0: DoF values of the cell and its 6 neighbours
  if (active) {
    U[tid] = a.u[vbase + cell * NV + tid];
#pragma unroll
    for (int f = 0; f < 6; ++f)
      if (has(f)) U[(1 + f) * NV + tid] = a.u[vbase + nbr(f) * NV + tid];
  }
  __syncthreads();

  // ---- P1: x stage (D, V); traces and normal-derivative planes of both sides
  if (active) {
    T sd = T(0), sv = T(0);   // thread = (q0, i1, i2)
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const T v = U[m + N1 * (i1 + N1 * i2)];
      sd = fma(Dq[i0 * N1 + m], v, sd);
      sv = fma(Vq[i0 * N1 + m], v, sv);
    }
    sc[0 * NV + tid] = sd;
    sc[1 * NV + tid] = sv;
    for (int e = tid; e < 6 * NF; e += NV) {
      const int f = e / NF, p = e % NF, t = f >> 1, side = f & 1, j = p % N1, l = p / N1;
      const T* ds = dd + side * N1;
      T s = T(0);
#pragma unroll
      for (int m = 0; m < N1; ++m) s = fma(ds[m], U[lidx(t, m, j, l)], s);
      fb[0 * 6 * NF + e] = U[lidx(t, side * K, j, l)];
      fb[1 * 6 * NF + e] = s;
      if (has(f)) {
        const T* UN = U + (1 + f) * NV;
        const T* dn = dd + (1 - side) * N1;
        T sn = T(0);
#pragma unroll
        for (int m = 0; m < N1; ++m) sn = fma(dn[m], UN[lidx(t, m, j, l)], sn);
        fb[2 * 6 * NF + e] = UN[lidx(t, (1 - side) * K, j, l)];
        fb[3 * 6 * NF + e] = sn;
      }
    }
  }
  __syncthreads();

  // ---- P2: y stage (V, D, V); face stage along u (both sides)
  if (active) {
    T dv = T(0), vd = T(0), vv = T(0);   // thread = (q0, q1, i2)
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const T xd = sc[0 * NV + i0 + N1 * (m + N1 * i2)], xv = sc[1 * NV + i0 + N1 * (m + N1 * i2)];
      dv = fma(Vq[i1 * N1 + m], xd, dv);
      vd = fma(Dq[i1 * N1 + m], xv, vd);
      vv = fma(Vq[i1 * N1 + m], xv, vv);
    }
    sc[2 * NV + tid] = dv;
    sc[3 * NV + tid] = vd;
    sc[4 * NV + tid] = vv;
    for (int e = tid; e < 6 * NF; e += NV) {
      const int f = e / NF, p = e % NF, pu = p % N1, l = p / N1;
      const T* tr = fb + f * NF;
      const T* dl = fb + 6 * NF + f * NF;
      T t1 = T(0), t2 = T(0), t3 = T(0);
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        t1 = fma(Vq[pu * N1 + j], tr[j + N1 * l], t1);
        t2 = fma(Dq[pu * N1 + j], tr[j + N1 * l], t2);
        t3 = fma(Vq[pu * N1 + j], dl[j + N1 * l], t3);
      }
      fa[0 * 6 * NF + e] = t1;
      fa[1 * 6 * NF + e] = t2;
      fa[2 * 6 * NF + e] = t3;
      if (has(f)) {
        const T* trn = fb + 12 * NF + f * NF;
        const T* dln = fb + 18 * NF + f * NF;
        T n1v = T(0), n2v = T(0), n3v = T(0);
#pragma unroll
        for (int j = 0; j < N1; ++j) {
          n1v = fma(Vq[pu * N1 + j], trn[j + N1 * l], n1v);
          n2v = fma(Dq[pu * N1 + j], trn[j + N1 * l], n2v);
          n3v = fma(Vq[pu * N1 + j], dln[j + N1 * l], n3v);
        }
        fa[3 * 6 * NF + e] = n1v;
        fa[4 * 6 * NF + e] = n2v;
        fa[5 * 6 * NF + e] = n3v;
      }
    }
  }
  __syncthreads();

  // ---- P3: z stage (V, V, D) and the metric; face stage along v and the edge coefficients
  if (active) {
    T g0 = T(0), g1 = T(0), g2 = T(0);   // thread = (q0, q1, q2)
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const int o = i0 + N1 * (i1 + N1 * m);
      g0 = fma(Vq[i2 * N1 + m], sc[2 * NV + o], g0);
      g1 = fma(Vq[i2 * N1 + m], sc[3 * NV + o], g1);
      g2 = fma(Dq[i2 * N1 + m], sc[4 * NV + o], g2);
    }
    const T c00 = gc[0 * NV + tid], c01 = gc[1 * NV + tid], c02 = gc[2 * NV + tid];
    const T c11 = gc[3 * NV + tid], c12 = gc[4 * NV + tid], c22 = gc[5 * NV + tid];
    sc[0 * NV + tid] = fma(c00, g0, fma(c01, g1, c02 * g2));
    sc[1 * NV + tid] = fma(c01, g0, fma(c11, g1, c12 * g2));
    sc[5 * NV + tid] = fma(c02, g0, fma(c12, g1, c22 * g2));
    for (int e = tid; e < 6 * NF; e += NV) {
      const int f = e / NF, p = e % NF, pu = p % N1, pv = p / N1, t = f >> 1;
      const int u = t == 0 ? 1 : 0, v = t == 2 ? 1 : 2;
      const T* T1 = fa + f * NF;
      const T* T2 = fa + 6 * NF + f * NF;
      const T* T3 = fa + 12 * NF + f * NF;
      T uK = T(0), duK = T(0), dtK = T(0), dvK = T(0);
#pragma unroll
      for (int l = 0; l < N1; ++l) {
        const T vq = Vq[pv * N1 + l];
        uK = fma(vq, T1[pu + N1 * l], uK);
        duK = fma(vq, T2[pu + N1 * l], duK);
        dtK = fma(vq, T3[pu + N1 * l], dtK);
        dvK = fma(Dq[pv * N1 + l], T1[pu + N1 * l], dvK);
      }
      T gK[3];
      gK[t] = dtK;
      gK[u] = duK;
      gK[v] = dvK;
      const T aK0 = gc[GA + (f * 3 + 0) * NF + p], aK1 = gc[GA + (f * 3 + 1) * NF + p];
      const T aK2 = gc[GA + (f * 3 + 2) * NF + p];
      const T dnK = fma(aK0, gK[0], fma(aK1, gK[1], aK2 * gK[2]));
      const T Wq = gc[GW + f * NF + p], gam = gc[GS + f];
      T alpha, c1;
      if (has(f)) {
        const T* N1p = fa + 18 * NF + f * NF;
        const T* N2p = fa + 24 * NF + f * NF;
        const T* N3p = fa + 30 * NF + f * NF;
        T uN = T(0), duN = T(0), dtN = T(0), dvN = T(0);
#pragma unroll
        for (int l = 0; l < N1; ++l) {
          const T vq = Vq[pv * N1 + l];
          uN = fma(vq, N1p[pu + N1 * l], uN);
          duN = fma(vq, N2p[pu + N1 * l], duN);
          dtN = fma(vq, N3p[pu + N1 * l], dtN);
          dvN = fma(Dq[pv * N1 + l], N1p[pu + N1 * l], dvN);
        }
        T gN[3];
        gN[t] = dtN;
        gN[u] = duN;
        gN[v] = dvN;
        // the neighbour's J^{-1} n_N on its face f ^ 1, n_N = -n
        const T* gnb = a.geo + nbr(f) * G + GA + ((f ^ 1) * 3) * NF + p;
        const T dnN = -fma(gnb[0], gN[0], fma(gnb[NF], gN[1], gnb[2 * NF] * gN[2]));
        const T jump = uK - uN;
        alpha = Wq * (T(0.5) * gam * jump - T(0.5) * (dnK + dnN));
        c1 = -T(0.5) * Wq * jump;
      } else {
        alpha = Wq * (gam * uK - dnK);
        c1 = -Wq * uK;
      }
      const T aK[3] = {aK0, aK1, aK2};
      fb[0 * 6 * NF + e] = alpha;
      fb[1 * 6 * NF + e] = c1 * aK[t];
      fb[2 * 6 * NF + e] = c1 * aK[u];
      fb[3 * 6 * NF + e] = c1 * aK[v];
    }
  }
  __syncthreads();

  // ---- P4: transposed z stage; test stage along v
  if (active) {
    T bdv = T(0), bvd = T(0), bvv = T(0);   // thread = (q0, q1, i2)
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const int o = i0 + N1 * (i1 + N1 * m);
      bdv = fma(Vq[m * N1 + i2], sc[0 * NV + o], bdv);
      bvd = fma(Vq[m * N1 + i2], sc[1 * NV + o], bvd);
      bvv = fma(Dq[m * N1 + i2], sc[5 * NV + o], bvv);
    }
    sc[2 * NV + tid] = bdv;
    sc[3 * NV + tid] = bvd;
    sc[4 * NV + tid] = bvv;
    for (int e = tid; e < 6 * NF; e += NV) {
      const int f = e / NF, p = e % NF, pu = p % N1, l = p / N1;
      const T* al = fb + f * NF;
      const T* bt = fb + 6 * NF + f * NF;
      const T* bu = fb + 12 * NF + f * NF;
      const T* bv = fb + 18 * NF + f * NF;
      T qt = T(0), qa = T(0), qu = T(0);
#pragma unroll
      for (int pv = 0; pv < N1; ++pv) {
        const T vq = Vq[pv * N1 + l];
        qt = fma(vq, bt[pu + N1 * pv], qt);
        qu = fma(vq, bu[pu + N1 * pv], qu);
        qa = fma(vq, al[pu + N1 * pv], qa);
        qa = fma(Dq[pv * N1 + l], bv[pu + N1 * pv], qa);
      }
      fa[0 * 6 * NF + e] = qt;
      fa[1 * 6 * NF + e] = qa;
      fa[2 * 6 * NF + e] = qu;
    }
  }
  __syncthreads();

  // ---- P5: transposed y stage; test stage along u
  if (active) {
    T yd = T(0), yv = T(0);   // thread = (q0, i1, i2)
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const int o = i0 + N1 * (m + N1 * i2);
      yd = fma(Vq[m * N1 + i1], sc[2 * NV + o], yd);
      yv = fma(Dq[m * N1 + i1], sc[3 * NV + o], yv);
      yv = fma(Vq[m * N1 + i1], sc[4 * NV + o], yv);
    }
    sc[0 * NV + tid] = yd;
    sc[1 * NV + tid] = yv;
    for (int e = tid; e < 6 * NF; e += NV) {
      const int f = e / NF, p = e % NF, j = p % N1, l = p / N1;
      const T* qt = fa + f * NF;
      const T* qa = fa + 6 * NF + f * NF;
      const T* qu = fa + 12 * NF + f * NF;
      T bt = T(0), as = T(0);
#pragma unroll
      for (int pu = 0; pu < N1; ++pu) {
        bt = fma(Vq[pu * N1 + j], qt[pu + N1 * l], bt);
        as = fma(Vq[pu * N1 + j], qa[pu + N1 * l], as);
        as = fma(Dq[pu * N1 + j], qu[pu + N1 * l], as);
      }
      fb[0 * 6 * NF + e] = bt;
      fb[1 * 6 * NF + e] = as;
    }
  }
  __syncthreads();

  // ---- P6: transposed x stage and the face contributions; write
  if (active) {
    T v = T(0);   // thread = (i0, i1, i2)
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const int o = m + N1 * (i1 + N1 * i2);
      v = fma(Dq[m * N1 + i0], sc[0 * NV + o], v);
      v = fma(Vq[m * N1 + i0], sc[1 * NV + o], v);
    }
    const int ii[3] = {i0, i1, i2};
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int t = f >> 1, side = f & 1;
      const int u = t == 0 ? 1 : 0, w = t == 2 ? 1 : 2;
      const int p = ii[u] + N1 * ii[w];
      v = fma(dd[side * N1 + ii[t]], fb[f * NF + p], v);
      if (ii[t] == side * K) v += fb[6 * NF + f * NF + p];
    }
    return v;
  }
  return T(0);
}

template <int N1, typename T>
__global__ void __launch_bounds__(Mapped3Shape<N1>::THREADS) mapped3_op_kernel(Mapped3ArgsT<T> a) {
  using S = Mapped3Shape<N1>;
  constexpr int NV = S::NV;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  mapped3_tables<N1, T>(a.B, sm);
  const int slot = threadIdx.x / NV, tid = threadIdx.x % NV;
  const int64_t cell = (int64_t)blockIdx.x * S::CPB + slot;
  const bool active = cell < a.ncells;
  const T v = mapped3_cell_apply<N1, T>(a, sm, sm + S::TABLES + slot * S::SLOT, cell, active, tid);
  if (active) {
    const int64_t gi = (int64_t)blockIdx.y * a.ndofs + cell * NV + tid;
    a.out[gi] = a.rhs ? a.rhs[gi] - v : v;
  }
}

// Residual, surrogate cell solve and update fused (see mapped.cu, 2D):
//   r = b - (A x)_K, z = (Z_2 x Z_1 x Z_0) Lambda^{-1} (Z_2 x Z_1 x Z_0)^T r,
//   mode 0: out_K = x_K + omega z;  mode 1: d_K = c1 d_K + c2 z, out_K = x_K + d_K
template <typename T>
struct Mapped3FusedArgsT {
  Mapped3ArgsT<T> op;
  const T* b;
  T* out;
  T* d;
  const int* list;
  int64_t count;
  const T* Z[3];
  const T* inv;
  int mode;
  T omega, c1, c2;
};

// CPB: cells per CTA (the shape's default, or fewer on small levels so that
// the work of a launch spreads over more SMs)
template <int N1, typename T, int CPB>
__global__ void __launch_bounds__(CPB * Mapped3Shape<N1>::NV) mapped3_fused_kernel(Mapped3FusedArgsT<T> f) {
  using S = Mapped3Shape<N1>;
  constexpr int NV = S::NV, NF = S::NF, SL = S::SLOT + 3 * NF;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  mapped3_tables<N1, T>(f.op.B, sm);
  const int slot = threadIdx.x / NV, tid = threadIdx.x % NV;
  const int64_t idx = (int64_t)blockIdx.x * CPB + slot;
  const bool active = idx < f.count;
  int64_t cell = 0;
  if (active) {
    if (f.list) {
      const int p = f.list[idx];
      cell = unpack_x(p) + (int64_t)f.op.nx * (unpack_y(p) + (int64_t)f.op.ny * unpack_z(p));
    } else {
      cell = idx;
    }
  }
  T* Wk = sm + S::TABLES + slot * SL;
  T* Zs = Wk + S::SLOT;   // Z_0, Z_1, Z_2 of the cell
  if (active)
    for (int e = tid; e < 3 * NF; e += NV) Zs[e] = f.Z[e / NF][cell * NF + e % NF];
  const T v = mapped3_cell_apply<N1, T>(f.op, sm, Wk, cell, active, tid);
  const int64_t gi = (int64_t)blockIdx.y * f.op.ndofs + cell * NV + tid;
  const T xo = active ? Wk[S::U + tid] : T(0);
  T* sc = Wk + S::SC;
  const int i0 = tid % N1, i1 = (tid / N1) % N1, i2 = tid / NF;
  const T* Z0 = Zs;
  const T* Z1 = Zs + NF;
  const T* Z2 = Zs + 2 * NF;
  __syncthreads();   // the operator's last stage read sc
  if (active) sc[tid] = f.b[gi] - v;
  __syncthreads();
  if (active) {   // Z_0^T along x
    T s = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s = fma(Z0[m * N1 + i0], sc[m + N1 * i1 + NF * i2], s);
    sc[NV + tid] = s;
  }
  __syncthreads();
  if (active) {   // Z_1^T along y
    T s = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s = fma(Z1[m * N1 + i1], sc[NV + i0 + N1 * m + NF * i2], s);
    sc[2 * NV + tid] = s;
  }
  __syncthreads();
  if (active) {   // Z_2^T along z, then 1 / (lambda_i + lambda_j + lambda_l)
    T s = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s = fma(Z2[m * N1 + i2], sc[2 * NV + i0 + N1 * i1 + NF * m], s);
    sc[3 * NV + tid] = s * f.inv[cell * NV + tid];
  }
  __syncthreads();
  if (active) {   // Z_2 along z
    T s = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s = fma(Z2[i2 * N1 + m], sc[3 * NV + i0 + N1 * i1 + NF * m], s);
    sc[4 * NV + tid] = s;
  }
  __syncthreads();
  if (active) {   // Z_1 along y
    T s = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s = fma(Z1[i1 * N1 + m], sc[4 * NV + i0 + N1 * m + NF * i2], s);
    sc[5 * NV + tid] = s;
  }
  __syncthreads();
  if (active) {   // Z_0 along x, update
    T z = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) z = fma(Z0[i0 * N1 + m], sc[5 * NV + m + N1 * i1 + NF * i2], z);
    if (f.mode == 0) {
      f.out[gi] = fma(f.omega, z, xo);
    } else {
      const T dn = fma(f.c1, f.d[gi], f.c2 * z);
      f.d[gi] = dn;
      f.out[gi] = xo + dn;
    }
  }
}

template <int N1, typename T, int CPB>
static tpss_status launch_fused3_cpb(tpss_ctx* ctx, const Mapped3FusedArgsT<T>& a, int nrhs) {
  using S = Mapped3Shape<N1>;
  const size_t smem = (size_t)(S::TABLES + CPB * (S::SLOT + 3 * S::NF)) * sizeof(T);
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(mapped3_fused_kernel<N1, T, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr = true;
  }
  const dim3 grid((unsigned)((a.count + CPB - 1) / CPB), (unsigned)nrhs);
  mapped3_fused_kernel<N1, T, CPB><<<grid, CPB * S::NV, smem, ctx->stream>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// launches of fewer than two CTAs per SM (the coarse levels) take CTAs of
// about 64 threads
template <int N1, typename T>
static tpss_status launch_fused3(tpss_ctx* ctx, const Mapped3FusedArgsT<T>& a, int nrhs) {
  using S = Mapped3Shape<N1>;
  constexpr int SMALL = S::NV >= 64 ? 1 : 64 / (S::NV);
  if (SMALL < S::CPB && (a.count + S::CPB - 1) / S::CPB * nrhs < 2 * (int64_t)ctx->num_sms)
    return launch_fused3_cpb<N1, T, SMALL>(ctx, a, nrhs);
  return launch_fused3_cpb<N1, T, S::CPB>(ctx, a, nrhs);
}

template <typename T>
tpss_status mapped3_fused_t(tpss_patches* P, const int* list, int64_t count, int nrhs, const T* x, const T* b, T* out,
                            T* d, int mode, T omega, T c1, T c2) {
  tpss_ctx* ctx = P->ctx;
  const Level& L = ctx->levels[P->level];
  Mapped3FusedArgsT<T> a{};
  a.op.u = x;
  a.op.geo = geo_of<T>(L);
  a.op.B = ctx->d_basis;
  a.op.nx = L.nc[0];
  a.op.ny = L.nc[1];
  a.op.nz = L.nc[2];
  a.op.ncells = L.ncells;
  a.op.ndofs = L.ndofs;
  a.b = b;
  a.out = out;
  a.d = d;
  a.list = list;
  a.count = count;
  for (int t = 0; t < 3; ++t) a.Z[t] = patch_Z<T>(P, t);
  a.inv = patch_inv<T>(P);
  a.mode = mode;
  a.omega = omega;
  a.c1 = c1;
  a.c2 = c2;
  if (!a.op.geo || !a.Z[0] || !a.inv) {
    set_error("smoother: surrogate cell data missing for this precision");
    return TPSS_EINVAL;
  }
  switch (ctx->n1) {
    case 2: return launch_fused3<2, T>(ctx, a, nrhs);
    case 3: return launch_fused3<3, T>(ctx, a, nrhs);
    case 4: return launch_fused3<4, T>(ctx, a, nrhs);
    case 5: return launch_fused3<5, T>(ctx, a, nrhs);
    case 6: return launch_fused3<6, T>(ctx, a, nrhs);
    case 7: return launch_fused3<7, T>(ctx, a, nrhs);
    case 8: return launch_fused3<8, T>(ctx, a, nrhs);
    default: break;
  }
  set_error("smoother: meshes of hexahedra support degrees 1..7");
  return TPSS_EINVAL;
}
template tpss_status mapped3_fused_t<double>(tpss_patches*, const int*, int64_t, int, const double*, const double*,
                                             double*, double*, int, double, double, double);
template tpss_status mapped3_fused_t<float>(tpss_patches*, const int*, int64_t, int, const float*, const float*,
                                            float*, float*, int, float, float, float);

template <int N1, typename T>
static tpss_status launch_mapped3(tpss_ctx* ctx, const Mapped3ArgsT<T>& a, int nrhs) {
  using S = Mapped3Shape<N1>;
  const size_t smem = (size_t)(S::TABLES + S::CPB * S::SLOT) * sizeof(T);
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(mapped3_op_kernel<N1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr = true;
  }
  const dim3 grid((unsigned)((a.ncells + S::CPB - 1) / S::CPB), (unsigned)nrhs);
  mapped3_op_kernel<N1, T><<<grid, S::THREADS, smem, ctx->stream>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

template <typename T>
tpss_status mapped3_apply_t(tpss_ctx* ctx, int level, int nrhs, const T* u, T* out, const T* rhs) {
  const Level& L = ctx->levels[level];
  Mapped3ArgsT<T> a{};
  a.u = u;
  a.out = out;
  a.rhs = rhs;
  a.geo = geo_of<T>(L);
  a.B = ctx->d_basis;
  a.nx = L.nc[0];
  a.ny = L.nc[1];
  a.nz = L.nc[2];
  a.ncells = L.ncells;
  a.ndofs = L.ndofs;
  switch (ctx->n1) {
    case 2: return launch_mapped3<2, T>(ctx, a, nrhs);
    case 3: return launch_mapped3<3, T>(ctx, a, nrhs);
    case 4: return launch_mapped3<4, T>(ctx, a, nrhs);
    case 5: return launch_mapped3<5, T>(ctx, a, nrhs);
    case 6: return launch_mapped3<6, T>(ctx, a, nrhs);
    case 7: return launch_mapped3<7, T>(ctx, a, nrhs);
    case 8: return launch_mapped3<8, T>(ctx, a, nrhs);
    default: break;
  }
  set_error("operator: meshes of hexahedra support degrees 1..7");
  return TPSS_EINVAL;
}
template tpss_status mapped3_apply_t<double>(tpss_ctx*, int, int, const double*, double*, const double*);
template tpss_status mapped3_apply_t<float>(tpss_ctx*, int, int, const float*, float*, const float*);

// ------------------------------------------------- surrogate cell solvers
// hbar[t][c]: the mean length of the cell's 4 edges along t (eq. avglength)
__global__ void surrogate_widths3_kernel(const double3* __restrict__ V, int nx, int ny, int nz, double* __restrict__ h) {
  const int64_t nc = (int64_t)nx * ny * nz;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const Hex H = load_hex(V, nx, ny, (int)(c % nx), (int)((c / nx) % ny), (int)(c / ((int64_t)nx * ny)));
    for (int t = 0; t < 3; ++t) {
      double s = 0.0;
      bool first = true;
      for (int k = 0; k < 8; ++k) {
        if ((k >> t) & 1) continue;
        const double l = dist3(H.v[k], H.v[k + (1 << t)]);
        s = first ? l : s + l;
        first = false;
      }
      h[t * nc + c] = s / 4.0;
    }
  }
}

// inv[c][i + n j + n^2 l] = 1 / (lambda^(0)_i(c) + lambda^(1)_j(c) + lambda^(2)_l(c))
__global__ void inv_table_cells3_kernel(const double* __restrict__ l0, const double* __restrict__ l1,
                                        const double* __restrict__ l2, int n, int64_t ncells, double* __restrict__ inv) {
  const int64_t vol = (int64_t)n * n * n, total = ncells * vol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / vol;
    const int loc = (int)(e % vol);
    inv[e] = 1.0 / (l0[c * n + loc % n] + l1[c * n + (loc / n) % n] + l2[c * n + loc / (n * n)]);
  }
}

tpss_status mapped3_surrogate_widths(tpss_ctx* ctx, int level, double* h) {
  const Level& L = ctx->levels[level];
  surrogate_widths3_kernel<<<(unsigned)std::min<int64_t>((L.ncells + 255) / 256, 4096), 256, 0, ctx->stream>>>(
      reinterpret_cast<const double3*>(L.d_verts), L.nc[0], L.nc[1], L.nc[2], h);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

tpss_status mapped3_inv_table(tpss_ctx* ctx, tpss_patches* P) {
  inv_table_cells3_kernel<<<2048, 256, 0, ctx->stream>>>(P->d_lam[0], P->d_lam[1], P->d_lam[2], P->n, P->nsub,
                                                         P->d_inv);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// ------------------------------------------------------- right-hand side
// kind 0: f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), g = 0, (k+2)-point rule per direction
__global__ void mapped3_rhs_kernel(const Basis1D* __restrict__ B, const double3* __restrict__ V, int nx, int ny,
                                   double* __restrict__ b) {
  extern __shared__ double sm[];
  const int n1 = B->n1, nq = B->nq_rhs;
  const int64_t c = blockIdx.x;
  const int64_t sxy = (int64_t)nx * ny;
  const Hex H = load_hex(V, nx, ny, (int)(c % nx), (int)((c / nx) % ny), (int)(c / sxy));
  double* F = sm;                   // nq^3
  double* G1 = F + nq * nq * nq;    // n1 nq nq
  double* G2 = G1 + n1 * nq * nq;   // n1 n1 nq
  const double pi = 3.14159265358979323846;
  for (int e = threadIdx.x; e < nq * nq * nq; e += blockDim.x) {
    const int q0 = e % nq, q1 = (e / nq) % nq, q2 = e / (nq * nq);
    const double xi[3] = {B->xr[q0], B->xr[q1], B->xr[q2]};
    double Ji[9];
    const double det = hex_inverse_jacobian(H, xi[0], xi[1], xi[2], Ji);
    double x[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 8; ++k) {
      double w = 1.0;
      for (int t = 0; t < 3; ++t) w *= ((k >> t) & 1) ? xi[t] : 1.0 - xi[t];
      x[0] += w * H.v[k].x;
      x[1] += w * H.v[k].y;
      x[2] += w * H.v[k].z;
    }
    F[e] = B->wr[q0] * B->wr[q1] * B->wr[q2] * fabs(det) * 3.0 * pi * pi * sin(pi * x[0]) * sin(pi * x[1]) *
           sin(pi * x[2]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n1 * nq * nq; e += blockDim.x) {
    const int i0 = e % n1, q12 = e / n1;
    double s = 0.0;
    for (int q0 = 0; q0 < nq; ++q0) s += B->Vr[q0 * n1 + i0] * F[q0 + nq * q12];
    G1[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n1 * n1 * nq; e += blockDim.x) {
    const int i0 = e % n1, i1 = (e / n1) % n1, q2 = e / (n1 * n1);
    double s = 0.0;
    for (int q1 = 0; q1 < nq; ++q1) s += B->Vr[q1 * n1 + i1] * G1[i0 + n1 * (q1 + nq * q2)];
    G2[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n1 * n1 * n1; e += blockDim.x) {
    const int i01 = e % (n1 * n1), i2 = e / (n1 * n1);
    double s = 0.0;
    for (int q2 = 0; q2 < nq; ++q2) s += B->Vr[q2 * n1 + i2] * G2[i01 + n1 * n1 * q2];
    b[c * n1 * n1 * n1 + e] = s;
  }
}

tpss_status mapped3_rhs(tpss_ctx* ctx, int level, double* b) {
  const Level& L = ctx->levels[level];
  const int nq = ctx->n1 + 1, n1 = ctx->n1;
  const size_t smem = (size_t)(nq * nq * nq + n1 * nq * nq + n1 * n1 * nq) * sizeof(double);
  mapped3_rhs_kernel<<<(unsigned)L.ncells, 128, smem, ctx->stream>>>(
      ctx->d_basis, reinterpret_cast<const double3*>(L.d_verts), L.nc[0], L.nc[1], b);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

}  // namespace tpss
