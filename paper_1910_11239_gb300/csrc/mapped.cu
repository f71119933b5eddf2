// SIPG on 2D meshes of bilinear quadrilaterals and the inexact cell solvers
// on Cartesian surrogate cells of Sec. 4 (eq. schwarzproj, eq. avglength).
//
// Mesh: a structured (nx+1) x (ny+1) vertex array per level (x index
// fastest); cell (i, j) has the corners v0 = V[j][i], v1 = V[j][i+1],
// v2 = V[j+1][i], v3 = V[j+1][i+1] at the reference corners (0,0), (1,0),
// (0,1), (1,1) and the bilinear map
//   x(a, b) = v0 (1-a)(1-b) + v1 a (1-b) + v2 (1-a) b + v3 a b.
// Finer levels split every cell at its reference midpoints, so the child
// maps are the parent map on quarters of the reference square, the spaces
// are nested and the transfers are the Cartesian ones (transfer.cu).
//
// Operator (eq. bfsipg on mapped cells, matrix-free): one CTA handles CPB
// cells, (k+1)^2 threads per cell.  The geometry (metric at the Gauss
// points, J^{-1} n at the edge points, |e| and the penalty per edge) is
// computed once per level; the kernel is bound by the FP64 pipe, and these
// 3 (k+1)^2 + 8 (k+1) + 8 doubles per cell cost less HBM time than
// recomputing them (two Jacobian inversions per edge point) costs FP64 time.
//   cell term   sum_q w_q |det J| (J^{-1} J^{-T} g_u) . g_v with reference
//               gradients g from sum factorization (Gauss points xq, k+1 per
//               direction; Vq, Dq the basis values and derivatives there)
//   face terms  per edge point: jump [u] = u^K - u^N, normal derivatives
//               d_n u = (J^{-1} n) . g_ref u on both sides (each with its own
//               Jacobian), and, with the paper's 1/sqrt(2) averages,
//                 v^K:          W (gamma/2 [u] - (d_n u^K + d_n u^N)/2)
//                 d_n v^K:      -W [u] / 2
//               boundary edges: W (gamma u - d_n u) and -W u; W = w_q |e|.
// The penalty is gamma_hat P(k) (1/h^+ + 1/h^-) (eq. penalty) with h^+- =
// |K^+-| / |e|, the mean extent of the cell normal to the edge; h^+ = h^- on
// boundary edges.
//
// Surrogate cell solvers (eq. avglength): cell K is replaced by the
// rectangle with hbar_0 = (l_01 + l_23)/2, hbar_1 = (l_02 + l_13)/2 (vertex
// distances); its local matrix is the Cartesian cell block of that
// rectangle, M_1 x A_0 + A_1 x M_0, whose 1D matrices take the neighbours'
// surrogate widths normal to the shared faces for the penalty.  The 1D
// generalized eigenproblems are solved per cell and direction by the same
// kernel as on Cartesian meshes; the smoother reads them per cell.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tpss_internal.cuh"

namespace tpss {

namespace {

struct Quad {
  double2 v0, v1, v2, v3;
};

// J = [dx/da dx/db; dy/da dy/db] at (a, b); returns det J, writes J^{-1}
// (row-major: Ji[0] Ji[1] / Ji[2] Ji[3]).
__device__ __forceinline__ double inverse_jacobian(const Quad& Q, double a, double b, double Ji[4]) {
  const double j00 = (Q.v1.x - Q.v0.x) * (1.0 - b) + (Q.v3.x - Q.v2.x) * b;
  const double j10 = (Q.v1.y - Q.v0.y) * (1.0 - b) + (Q.v3.y - Q.v2.y) * b;
  const double j01 = (Q.v2.x - Q.v0.x) * (1.0 - a) + (Q.v3.x - Q.v1.x) * a;
  const double j11 = (Q.v2.y - Q.v0.y) * (1.0 - a) + (Q.v3.y - Q.v1.y) * a;
  const double det = j00 * j11 - j01 * j10;
  const double inv = 1.0 / det;
  Ji[0] = j11 * inv;
  Ji[1] = -j01 * inv;
  Ji[2] = -j10 * inv;
  Ji[3] = j00 * inv;
  return det;
}

__device__ __forceinline__ double quad_area(const Quad& Q) {
  // shoelace over v0, v1, v3, v2 (counter-clockwise for a positively oriented map)
  const double s = (Q.v0.x * Q.v1.y - Q.v1.x * Q.v0.y) + (Q.v1.x * Q.v3.y - Q.v3.x * Q.v1.y) +
                   (Q.v3.x * Q.v2.y - Q.v2.x * Q.v3.y) + (Q.v2.x * Q.v0.y - Q.v0.x * Q.v2.y);
  return 0.5 * fabs(s);
}

__device__ __forceinline__ double dist(double2 a, double2 b) {
  const double dx = b.x - a.x, dy = b.y - a.y;
  return sqrt(dx * dx + dy * dy);
}

}  // namespace

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// ---------------------------------------------------------------- meshes
// F = refinement of V (nx x ny cells): edge midpoints 0.5 (a + b), cell
// centres 0.25 (((a + b) + c) + d) -- the images of the reference midpoints.
__global__ void refine_vertices_kernel(const double2* __restrict__ V, int nx, int ny, double2* __restrict__ F) {
  const int fx = 2 * nx + 1, fy = 2 * ny + 1, sx = nx + 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < fx * fy; e += gridDim.x * blockDim.x) {
    const int i = e % fx, j = e / fx;
    const int i0 = i / 2, j0 = j / 2;
    const double2 a = V[j0 * sx + i0];
    double2 p;
    if (!(i & 1) && !(j & 1)) {
      p = a;
    } else if (!(j & 1)) {
      const double2 b = V[j0 * sx + i0 + 1];
      p = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y + b.y));
    } else if (!(i & 1)) {
      const double2 c = V[(j0 + 1) * sx + i0];
      p = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y + c.y));
    } else {
      const double2 b = V[j0 * sx + i0 + 1], c = V[(j0 + 1) * sx + i0], d = V[(j0 + 1) * sx + i0 + 1];
      p = make_double2(0.25 * (((a.x + b.x) + c.x) + d.x), 0.25 * (((a.y + b.y) + c.y) + d.y));
    }
    F[e] = p;
  }
}

// -------------------------------------------------------------- geometry
// Per level and cell, computed once when the context is created (G doubles
// per cell, GeoLayout):
//   C[3][n1^2]   w_q0 w_q1 |det J| J^{-1} J^{-T} at the Gauss points (c00, c01, c11)
//   A[4][2][n1]  J^{-1} n at the n1 Gauss points of edge f = 2 t + side, n the
//                cell's outward unit normal (straight edges: one n per edge)
//   S[4][2]      |e| and the penalty gamma_e of the edge (eq. penalty with
//                h = |K| / |e|; interior: both cells, boundary: h^+ = h^-)
struct GeoLayout {
  int n1, nl, C, A, S, G;
  __host__ __device__ explicit GeoLayout(int n) : n1(n), nl(n * n), C(0), A(3 * n * n), S(3 * n * n + 8 * n),
                                                 G(3 * n * n + 8 * n + 8) {}
};

__global__ void mapped_geometry_kernel(const Basis1D* __restrict__ B, const double2* __restrict__ V, int nx, int ny,
                                       double gpk, double* __restrict__ geo) {
  const int n1 = B->n1;
  const GeoLayout g(n1);
  const int64_t c = blockIdx.x;
  const int cx = (int)(c % nx), cy = (int)(c / nx);
  auto quad = [&](int i, int j) {
    Quad Q;
    Q.v0 = V[(int64_t)j * (nx + 1) + i];
    Q.v1 = V[(int64_t)j * (nx + 1) + i + 1];
    Q.v2 = V[(int64_t)(j + 1) * (nx + 1) + i];
    Q.v3 = V[(int64_t)(j + 1) * (nx + 1) + i + 1];
    return Q;
  };
  const Quad Q = quad(cx, cy);
  double* out = geo + c * g.G;
  for (int e = threadIdx.x; e < g.nl; e += blockDim.x) {
    const int q0 = e % n1, q1 = e / n1;
    double Ji[4];
    const double det = inverse_jacobian(Q, B->xq[q0], B->xq[q1], Ji);
    const double w = B->wq[q0] * B->wq[q1] * fabs(det);
    out[g.C + e] = w * (Ji[0] * Ji[0] + Ji[1] * Ji[1]);
    out[g.C + g.nl + e] = w * (Ji[0] * Ji[2] + Ji[1] * Ji[3]);
    out[g.C + 2 * g.nl + e] = w * (Ji[2] * Ji[2] + Ji[3] * Ji[3]);
  }
  for (int e = threadIdx.x; e < 4 * n1 + 4; e += blockDim.x) {
    const int f = e < 4 * n1 ? e / n1 : e - 4 * n1, t = f >> 1, side = f & 1;
    // edge of face f: t = 0 from v0 (side 0) / v1 to v2 / v3; t = 1 from v0 / v2 to v1 / v3
    const double2 pa = t == 0 ? (side ? Q.v1 : Q.v0) : (side ? Q.v2 : Q.v0);
    const double2 pb = t == 0 ? (side ? Q.v3 : Q.v2) : (side ? Q.v3 : Q.v1);
    const double tx = pb.x - pa.x, ty = pb.y - pa.y;
    const double le = sqrt(tx * tx + ty * ty);
    double nxv = t == 0 ? ty / le : -ty / le, nyv = t == 0 ? -tx / le : tx / le;
    if (side == 0) {
      nxv = -nxv;
      nyv = -nyv;
    }
    if (e < 4 * n1) {
      const double s = B->xq[e % n1];
      double Ji[4];
      inverse_jacobian(Q, t == 0 ? (double)side : s, t == 0 ? s : (double)side, Ji);
      out[g.A + f * 2 * n1 + e % n1] = Ji[0] * nxv + Ji[1] * nyv;
      out[g.A + f * 2 * n1 + n1 + e % n1] = Ji[2] * nxv + Ji[3] * nyv;
    } else {
      const int ni = cx + (t == 0 ? (side ? 1 : -1) : 0), nj = cy + (t == 1 ? (side ? 1 : -1) : 0);
      const double hK = quad_area(Q) / le;
      double gam;
      if (ni >= 0 && ni < nx && nj >= 0 && nj < ny) gam = gpk * (1.0 / hK + 1.0 / (quad_area(quad(ni, nj)) / le));
      else gam = gpk * (2.0 / hK);
      out[g.S + 2 * f] = le;
      out[g.S + 2 * f + 1] = gam;
    }
  }
}

// -------------------------------------------------------------- operator
template <int N1>
struct MappedShape {
  static constexpr int NL = N1 * N1;
  static constexpr int CPB_RAW = 256 / NL;
  static constexpr int CPB = CPB_RAW > 32 ? 32 : (CPB_RAW < 1 ? 1 : CPB_RAW);
  static constexpr int THREADS = CPB * NL;
  static constexpr int G = 3 * NL + 8 * N1 + 8;   // GeoLayout(N1).G
  // per-cell slot (doubles): own geometry, the neighbours' J^{-1} n on the
  // shared edges [4][2][N1], U (own + 4 neighbours), tA, tB, F0, F1 and 9
  // edge arrays [4][N1]
  static constexpr int GEO = 0, NA = G, U = NA + 8 * N1, TA = U + 5 * NL, TB = TA + NL, F0 = TB + NL, F1 = F0 + NL;
  static constexpr int FACE = F1 + NL;
  static constexpr int SLOT = FACE + 9 * 4 * N1;
  static constexpr int TABLES = 2 * NL + 4 * N1;
};

template <typename T>
struct MappedOpArgsT {
  const T* u;
  T* out;
  const T* rhs;        // not null: out = rhs - A u
  const T* geo;        // [ncells][G]
  const Basis1D* B;
  int nx, ny;
  int64_t ncells, ndofs;
};

// tables of the 2D kernels in shared memory: Vq, Dq (n1^2), d0, d1, wq (n1)
template <int N1, typename T>
__device__ __forceinline__ void mapped_tables(const Basis1D* __restrict__ B, T* sm) {
  constexpr int NL = N1 * N1;
  for (int e = threadIdx.x; e < NL; e += blockDim.x) {
    sm[e] = (T)B->Vq[e];
    sm[NL + e] = (T)B->Dq[e];
  }
  for (int e = threadIdx.x; e < N1; e += blockDim.x) {
    sm[2 * NL + e] = (T)B->d0[e];
    sm[2 * NL + N1 + e] = (T)B->d1[e];
    sm[2 * NL + 2 * N1 + e] = (T)B->wq[e];
  }
}

// (A u)_K at the local DoF tid of cell `cell` (a.u read, nothing written to
// global memory).  Every thread of the CTA calls it (it synchronizes the
// CTA); the tables must have been written (they become visible at its first
// barrier); W is the cell's slot, and W + S::U keeps u_K afterwards.
template <int N1, typename T>
__device__ __forceinline__ T mapped_cell_apply(const MappedOpArgsT<T>& a, T* sm, T* W, int64_t cell, bool active,
                                               int tid) {
  using S = MappedShape<N1>;
  constexpr int NL = N1 * N1, K = N1 - 1, G = S::G;
  constexpr int GA = 3 * NL, GS = 3 * NL + 8 * N1;   // GeoLayout offsets
  T* Vq = sm;
  T* Dq = Vq + NL;
  T* dd = Dq + NL;        // d0 then d1: phi_i'(0), phi_i'(1)
  T* wq = dd + 2 * N1;
  T* geo = W + S::GEO;
  T* na = W + S::NA;
  T* U = W + S::U;
  T* tA = W + S::TA;
  T* tB = W + S::TB;
  T* F0 = W + S::F0;
  T* F1 = W + S::F1;
  T* trK = W + S::FACE;
  T* dlK = trK + 4 * N1;
  T* trN = dlK + 4 * N1;
  T* dlN = trN + 4 * N1;
  T* al = dlN + 4 * N1;
  T* be = al + 4 * N1;
  T* de = be + 4 * N1;
  T* As = de + 4 * N1;
  T* Bs = As + 4 * N1;
  const int cx = active ? (int)(cell % a.nx) : 0, cy = active ? (int)(cell / a.nx) : 0;
  const int64_t vbase = (int64_t)blockIdx.y * a.ndofs;
  // face f = 2 t + side: neighbour along t at -1 (side 0) / +1 (side 1)
  const int hasm = (cx > 0 ? 1 : 0) | (cx + 1 < a.nx ? 2 : 0) | (cy > 0 ? 4 : 0) | (cy + 1 < a.ny ? 8 : 0);
  auto has = [&](int f) { return ((hasm >> f) & 1) != 0; };
  auto nbr = [&](int f) -> int64_t {
    return cell + (f == 0 ? -1 : f == 1 ? 1 : f == 2 ? -a.nx : a.nx);
  };
  // local index of (i_t = it, the other index = j) for direction t
  auto lidx = [](int t, int it, int j) { return t == 0 ? it + N1 * j : j + N1 * it; };

  // ---- P0: DoF values of the cell and its neighbours; geometry
  if (active) {
    U[tid] = a.u[vbase + cell * NL + tid];
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (has(f)) U[(1 + f) * NL + tid] = a.u[vbase + nbr(f) * NL + tid];
    const T* gc = a.geo + cell * G;
    for (int e = tid; e < G; e += NL) geo[e] = gc[e];
    // the neighbour across edge f sees it as its edge f ^ 1
    for (int e = tid; e < 8 * N1; e += NL) {
      const int f = e / (2 * N1);
      if (has(f)) na[e] = a.geo[nbr(f) * G + GA + (f ^ 1) * 2 * N1 + e % (2 * N1)];
    }
  }
  __syncthreads();

  // ---- P1: cell stage A; edge traces and reference normal-derivative lines
  if (active) {
    const int q0 = tid % N1, i1 = tid / N1;
    T sa = T(0), sb = T(0);
#pragma unroll
    for (int i0 = 0; i0 < N1; ++i0) {
      const T v = U[i0 + N1 * i1];
      sa = fma(Dq[q0 * N1 + i0], v, sa);
      sb = fma(Vq[q0 * N1 + i0], v, sb);
    }
    tA[tid] = sa;
    tB[tid] = sb;
    for (int e = tid; e < 4 * N1; e += NL) {
      const int f = e / N1, j = e % N1, t = f >> 1, side = f & 1;
      const T* ds = dd + side * N1;
      T s = T(0);
#pragma unroll
      for (int m = 0; m < N1; ++m) s = fma(ds[m], U[lidx(t, m, j)], s);
      trK[e] = U[lidx(t, side * K, j)];
      dlK[e] = s;
      if (has(f)) {
        const T* UN = U + (1 + f) * NL;
        const T* dn = dd + (1 - side) * N1;
        T sn = T(0);
#pragma unroll
        for (int m = 0; m < N1; ++m) sn = fma(dn[m], UN[lidx(t, m, j)], sn);
        trN[e] = UN[lidx(t, (1 - side) * K, j)];
        dlN[e] = sn;
      }
    }
  }
  __syncthreads();

  // ---- P2: reference gradients at the Gauss points times the metric; edge-point coefficients
  if (active) {
    const int q0 = tid % N1, q1 = tid / N1;
    T g0 = T(0), g1 = T(0);
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) {
      g0 = fma(Vq[q1 * N1 + i1], tA[q0 + N1 * i1], g0);
      g1 = fma(Dq[q1 * N1 + i1], tB[q0 + N1 * i1], g1);
    }
    const T c00 = geo[tid], c01 = geo[NL + tid], c11 = geo[2 * NL + tid];
    F0[tid] = fma(c00, g0, c01 * g1);
    F1[tid] = fma(c01, g0, c11 * g1);
    for (int e = tid; e < 4 * N1; e += NL) {
      const int f = e / N1, q = e % N1, t = f >> 1;
      const T* fl = trK + f * N1;
      const T* dl = dlK + f * N1;
      T uK = T(0), dtK = T(0), dtanK = T(0);
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        uK = fma(Vq[q * N1 + j], fl[j], uK);
        dtK = fma(Vq[q * N1 + j], dl[j], dtK);
        dtanK = fma(Dq[q * N1 + j], fl[j], dtanK);
      }
      const T aK0 = geo[GA + f * 2 * N1 + q], aK1 = geo[GA + f * 2 * N1 + N1 + q];   // J^{-1} n
      const T dnK = t == 0 ? fma(aK0, dtK, aK1 * dtanK) : fma(aK0, dtanK, aK1 * dtK);
      const T Wq = wq[q] * geo[GS + 2 * f], gam = geo[GS + 2 * f + 1];
      T alpha, c1;
      if (has(f)) {
        const T* gl = trN + f * N1;
        const T* gd = dlN + f * N1;
        T uN = T(0), dtN = T(0), dtanN = T(0);
#pragma unroll
        for (int j = 0; j < N1; ++j) {
          uN = fma(Vq[q * N1 + j], gl[j], uN);
          dtN = fma(Vq[q * N1 + j], gd[j], dtN);
          dtanN = fma(Dq[q * N1 + j], gl[j], dtanN);
        }
        // the neighbour's J^{-1} n_N with n_N = -n
        const T aN0 = -na[f * 2 * N1 + q], aN1 = -na[f * 2 * N1 + N1 + q];
        const T dnN = t == 0 ? fma(aN0, dtN, aN1 * dtanN) : fma(aN0, dtanN, aN1 * dtN);
        const T jump = uK - uN;
        alpha = Wq * (T(0.5) * gam * jump - T(0.5) * (dnK + dnN));
        c1 = -T(0.5) * Wq * jump;
      } else {
        alpha = Wq * (gam * uK - dnK);
        c1 = -Wq * uK;
      }
      al[e] = alpha;
      be[e] = c1 * (t == 0 ? aK0 : aK1);    // times d_t v
      de[e] = c1 * (t == 0 ? aK1 : aK0);    // times d_tan v
    }
  }
  __syncthreads();

  // ---- P3: cell stage C (test gradients, first direction); edge sums per test line
  if (active) {
    const int i0 = tid % N1, q1 = tid / N1;
    T sa = T(0), sb = T(0);
#pragma unroll
    for (int q0 = 0; q0 < N1; ++q0) {
      sa = fma(Dq[q0 * N1 + i0], F0[q0 + N1 * q1], sa);
      sb = fma(Vq[q0 * N1 + i0], F1[q0 + N1 * q1], sb);
    }
    tA[tid] = sa;
    tB[tid] = sb;
    for (int e = tid; e < 4 * N1; e += NL) {
      const int f = e / N1, j = e % N1;
      T sbv = T(0), sav = T(0);
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        sbv = fma(Vq[q * N1 + j], be[f * N1 + q], sbv);
        sav = fma(Vq[q * N1 + j], al[f * N1 + q], sav);
        sav = fma(Dq[q * N1 + j], de[f * N1 + q], sav);
      }
      Bs[e] = sbv;
      As[e] = sav;
    }
  }
  __syncthreads();

  // ---- P4: cell stage D and the edge contributions; write
  if (active) {
    const int i0 = tid % N1, i1 = tid / N1;
    T v = T(0);
#pragma unroll
    for (int q1 = 0; q1 < N1; ++q1) {
      v = fma(Vq[q1 * N1 + i1], tA[i0 + N1 * q1], v);
      v = fma(Dq[q1 * N1 + i1], tB[i0 + N1 * q1], v);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int t = f >> 1, side = f & 1;
      const int it = t == 0 ? i0 : i1, j = t == 0 ? i1 : i0;
      v = fma(dd[side * N1 + it], Bs[f * N1 + j], v);
      if (it == side * K) v += As[f * N1 + j];
    }
    return v;
  }
  return T(0);
}

template <int N1, typename T>
__global__ void __launch_bounds__(MappedShape<N1>::THREADS) mapped_op_kernel(MappedOpArgsT<T> a) {
  using S = MappedShape<N1>;
  constexpr int NL = N1 * N1;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  mapped_tables<N1, T>(a.B, sm);
  const int slot = threadIdx.x / NL, tid = threadIdx.x % NL;
  const int64_t cell = (int64_t)blockIdx.x * S::CPB + slot;
  const bool active = cell < a.ncells;
  const T v = mapped_cell_apply<N1, T>(a, sm, sm + S::TABLES + slot * S::SLOT, cell, active, tid);
  if (active) {
    const int64_t gi = (int64_t)blockIdx.y * a.ndofs + cell * NL + tid;
    a.out[gi] = a.rhs ? a.rhs[gi] - v : v;
  }
}

// Residual, surrogate cell solve and update fused, for the cells of `list`
// (packed positions; null: all cells):
//   r = b - (A x)_K,  z = Z_1 x Z_0 diag(1/(lambda_i + lambda_j)) (Z_1 x Z_0)^T r,
//   mode 0:  out_K = x_K + omega z
//   mode 1:  d_K = c1 d_K + c2 z,  out_K = x_K + d_K   (a Chebyshev step)
// out may equal x when no listed cell is a face neighbour of another (one
// color of the red-black sweep); otherwise out is a different vector.
template <typename T>
struct MappedFusedArgsT {
  MappedOpArgsT<T> op;  // op.u = x
  const T* b;
  T* out;
  T* d;
  const int* list;
  int64_t count;
  const T* Z[3];       // per cell and direction [N1 * N1], column j = eigenvector j
  const T* inv;        // per cell [N1^dim]
  int mode;
  T omega, c1, c2;
};

// CPB: cells per CTA (the shape's default, or fewer on small levels so that
// the work of a launch spreads over more SMs)
template <int N1, typename T, int CPB>
__global__ void __launch_bounds__(CPB * MappedShape<N1>::NL) mapped_fused_kernel(MappedFusedArgsT<T> f) {
  using S = MappedShape<N1>;
  constexpr int NL = N1 * N1, SL = S::SLOT + 2 * NL;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  mapped_tables<N1, T>(f.op.B, sm);
  const int slot = threadIdx.x / NL, tid = threadIdx.x % NL;
  const int64_t idx = (int64_t)blockIdx.x * CPB + slot;
  const bool active = idx < f.count;
  int64_t cell = 0;
  if (active) {
    if (f.list) {
      const int p = f.list[idx];
      cell = unpack_x(p) + (int64_t)f.op.nx * unpack_y(p);
    } else {
      cell = idx;
    }
  }
  T* W = sm + S::TABLES + slot * SL;
  T* Zs = W + S::SLOT;   // Z_0, Z_1 of the cell
  if (active) {
    Zs[tid] = f.Z[0][cell * NL + tid];
    Zs[NL + tid] = f.Z[1][cell * NL + tid];
  }
  const T v = mapped_cell_apply<N1, T>(f.op, sm, W, cell, active, tid);
  const int64_t gi = (int64_t)blockIdx.y * f.op.ndofs + cell * NL + tid;
  const T xo = active ? W[S::U + tid] : T(0);
  T* R = W + S::TA;
  T* T1 = W + S::TB;
  T* T2 = W + S::F0;
  T* T3 = W + S::F1;
  const int i0 = tid % N1, i1 = tid / N1;
  __syncthreads();   // the operator's last stage read these arrays
  if (active) R[tid] = f.b[gi] - v;
  __syncthreads();
  if (active) {   // Z_0^T along x
    T s = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s = fma(Zs[m * N1 + i0], R[m + N1 * i1], s);
    T1[tid] = s;
  }
  __syncthreads();
  if (active) {   // Z_1^T along y, then 1 / (lambda_i + lambda_j)
    T s = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s = fma(Zs[NL + m * N1 + i1], T1[i0 + N1 * m], s);
    T2[tid] = s * f.inv[cell * NL + tid];
  }
  __syncthreads();
  if (active) {   // Z_1 along y
    T s = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s = fma(Zs[NL + i1 * N1 + m], T2[i0 + N1 * m], s);
    T3[tid] = s;
  }
  __syncthreads();
  if (active) {   // Z_0 along x, update
    T z = T(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) z = fma(Zs[i0 * N1 + m], T3[m + N1 * i1], z);
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
static tpss_status launch_fused_cpb(tpss_ctx* ctx, const MappedFusedArgsT<T>& a, int nrhs) {
  using S = MappedShape<N1>;
  const size_t smem = (size_t)(S::TABLES + CPB * (S::SLOT + 2 * N1 * N1)) * sizeof(T);
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(mapped_fused_kernel<N1, T, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr = true;
  }
  const dim3 grid((unsigned)((a.count + CPB - 1) / CPB), (unsigned)nrhs);
  mapped_fused_kernel<N1, T, CPB><<<grid, CPB * N1 * N1, smem, ctx->stream>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// launches of fewer than two CTAs per SM (the coarse levels) take CTAs of
// about 64 threads
template <int N1, typename T>
static tpss_status launch_fused(tpss_ctx* ctx, const MappedFusedArgsT<T>& a, int nrhs) {
  using S = MappedShape<N1>;
  constexpr int SMALL = N1 * N1 >= 64 ? 1 : 64 / (N1 * N1);
  if (SMALL < S::CPB && (a.count + S::CPB - 1) / S::CPB * nrhs < 2 * (int64_t)ctx->num_sms)
    return launch_fused_cpb<N1, T, SMALL>(ctx, a, nrhs);
  return launch_fused_cpb<N1, T, S::CPB>(ctx, a, nrhs);
}

template <int N1, typename T>
static tpss_status launch_mapped(tpss_ctx* ctx, const MappedOpArgsT<T>& a, int nrhs) {
  using S = MappedShape<N1>;
  const size_t smem = (size_t)(S::TABLES + S::CPB * S::SLOT) * sizeof(T);
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(mapped_op_kernel<N1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr = true;
  }
  const dim3 grid((unsigned)((a.ncells + S::CPB - 1) / S::CPB), (unsigned)nrhs);
  mapped_op_kernel<N1, T><<<grid, S::THREADS, smem, ctx->stream>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

template <typename T>
tpss_status mapped_fused_t(tpss_patches* P, const int* list, int64_t count, int nrhs, const T* x, const T* b, T* out,
                           T* d, int mode, T omega, T c1, T c2) {
  tpss_ctx* ctx = P->ctx;
  if (ctx->dim == 3) return mapped3_fused_t<T>(P, list, count, nrhs, x, b, out, d, mode, omega, c1, c2);
  const Level& L = ctx->levels[P->level];
  MappedFusedArgsT<T> a{};
  a.op.u = x;
  a.op.geo = geo_of<T>(L);
  a.op.B = ctx->d_basis;
  a.op.nx = L.nc[0];
  a.op.ny = L.nc[1];
  a.op.ncells = L.ncells;
  a.op.ndofs = L.ndofs;
  a.b = b;
  a.out = out;
  a.d = d;
  a.list = list;
  a.count = count;
  for (int t = 0; t < 2; ++t) a.Z[t] = patch_Z<T>(P, t);
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
    case 2: return launch_fused<2, T>(ctx, a, nrhs);
    case 3: return launch_fused<3, T>(ctx, a, nrhs);
    case 4: return launch_fused<4, T>(ctx, a, nrhs);
    case 5: return launch_fused<5, T>(ctx, a, nrhs);
    case 6: return launch_fused<6, T>(ctx, a, nrhs);
    case 7: return launch_fused<7, T>(ctx, a, nrhs);
    case 8: return launch_fused<8, T>(ctx, a, nrhs);
    default: break;
  }
  if constexpr (sizeof(T) == sizeof(double)) {   // degrees 8..15: FP64 only
    switch (ctx->n1) {
      case 9: return launch_fused<9, T>(ctx, a, nrhs);
      case 10: return launch_fused<10, T>(ctx, a, nrhs);
      case 11: return launch_fused<11, T>(ctx, a, nrhs);
      case 12: return launch_fused<12, T>(ctx, a, nrhs);
      case 13: return launch_fused<13, T>(ctx, a, nrhs);
      case 14: return launch_fused<14, T>(ctx, a, nrhs);
      case 15: return launch_fused<15, T>(ctx, a, nrhs);
      case 16: return launch_fused<16, T>(ctx, a, nrhs);
      default: break;
    }
  }
  set_error("smoother: meshes of quadrilaterals support degrees 1..15 in FP64, 1..7 in FP32");
  return TPSS_EINVAL;
}
template tpss_status mapped_fused_t<double>(tpss_patches*, const int*, int64_t, int, const double*, const double*,
                                            double*, double*, int, double, double, double);
template tpss_status mapped_fused_t<float>(tpss_patches*, const int*, int64_t, int, const float*, const float*, float*,
                                           float*, int, float, float, float);

static double penalty_prefactor(const tpss_ctx* ctx) {
  return ctx->gamma_hat * (ctx->penalty_poly == TPSS_PENALTY_KP1SQ ? (double)(ctx->n1 * ctx->n1)
                                                                   : (double)(ctx->k * ctx->n1));
}

template <typename T>
tpss_status mapped_apply_t(tpss_ctx* ctx, int level, int nrhs, const T* u, T* out, const T* rhs) {
  if (ctx->dim == 3) return mapped3_apply_t<T>(ctx, level, nrhs, u, out, rhs);
  const Level& L = ctx->levels[level];
  MappedOpArgsT<T> a{};
  a.u = u;
  a.out = out;
  a.rhs = rhs;
  a.geo = geo_of<T>(L);
  a.B = ctx->d_basis;
  a.nx = L.nc[0];
  a.ny = L.nc[1];
  a.ncells = L.ncells;
  a.ndofs = L.ndofs;
  switch (ctx->n1) {
    case 2: return launch_mapped<2, T>(ctx, a, nrhs);
    case 3: return launch_mapped<3, T>(ctx, a, nrhs);
    case 4: return launch_mapped<4, T>(ctx, a, nrhs);
    case 5: return launch_mapped<5, T>(ctx, a, nrhs);
    case 6: return launch_mapped<6, T>(ctx, a, nrhs);
    case 7: return launch_mapped<7, T>(ctx, a, nrhs);
    case 8: return launch_mapped<8, T>(ctx, a, nrhs);
    default: break;
  }
  if constexpr (sizeof(T) == sizeof(double)) {   // degrees 8..15: FP64 only
    switch (ctx->n1) {
      case 9: return launch_mapped<9, T>(ctx, a, nrhs);
      case 10: return launch_mapped<10, T>(ctx, a, nrhs);
      case 11: return launch_mapped<11, T>(ctx, a, nrhs);
      case 12: return launch_mapped<12, T>(ctx, a, nrhs);
      case 13: return launch_mapped<13, T>(ctx, a, nrhs);
      case 14: return launch_mapped<14, T>(ctx, a, nrhs);
      case 15: return launch_mapped<15, T>(ctx, a, nrhs);
      case 16: return launch_mapped<16, T>(ctx, a, nrhs);
      default: break;
    }
  }
  set_error("operator: meshes of quadrilaterals support degrees 1..15 in FP64, 1..7 in FP32");
  return TPSS_EINVAL;
}
template tpss_status mapped_apply_t<double>(tpss_ctx*, int, int, const double*, double*, const double*);
template tpss_status mapped_apply_t<float>(tpss_ctx*, int, int, const float*, float*, const float*);

// ------------------------------------------------- surrogate cell solvers
// hbar[t][c] of eq. avglength (vertex distances)
__global__ void surrogate_widths_kernel(const double2* __restrict__ V, int nx, int ny, double* __restrict__ h0,
                                        double* __restrict__ h1) {
  const int64_t nc = (int64_t)nx * ny;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)(c / nx);
    const double2 v0 = V[(int64_t)j * (nx + 1) + i], v1 = V[(int64_t)j * (nx + 1) + i + 1];
    const double2 v2 = V[(int64_t)(j + 1) * (nx + 1) + i], v3 = V[(int64_t)(j + 1) * (nx + 1) + i + 1];
    h0[c] = 0.5 * (dist(v0, v1) + dist(v2, v3));
    h1[c] = 0.5 * (dist(v0, v2) + dist(v1, v3));
  }
}

// 1D matrices of cell c's surrogate along t: width hbar_t(c), neighbours'
// hbar_t across the faces normal to t
__global__ void surrogate_op1d_kernel(const Basis1D* __restrict__ B, const double* __restrict__ w, int nx, int ny,
                                      int nz, int t, double gpk, double* __restrict__ M, double* __restrict__ A) {
  const int n1 = B->n1;
  const int64_t c = blockIdx.x;
  const int ci[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((int64_t)nx * ny))};
  const int nc[3] = {nx, ny, nz};
  const bool has_l = ci[t] > 0, has_r = ci[t] + 1 < nc[t];
  const int64_t step = t == 0 ? 1 : t == 1 ? nx : (int64_t)nx * ny;
  const double h = w[c];
  const double hl = has_l ? w[c - step] : h, hr = has_r ? w[c + step] : h;
  for (int e = threadIdx.x; e < n1 * n1; e += blockDim.x)
    op1d_entry(B, h, hl, hr, has_l, has_r, gpk, e / n1, e % n1, &M[c * n1 * n1 + e], &A[c * n1 * n1 + e]);
}

// inv[c][i + n j] = 1 / (lambda^(0)_i(c) + lambda^(1)_j(c))
__global__ void inv_table_cells_kernel(const double* __restrict__ l0, const double* __restrict__ l1, int n,
                                       int64_t ncells, double* __restrict__ inv) {
  const int64_t total = ncells * n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / (n * n);
    const int loc = (int)(e % (n * n));
    inv[e] = 1.0 / (l0[c * n + loc % n] + l1[c * n + loc / n]);
  }
}

tpss_status mapped_cell_eigendata(tpss_ctx* ctx, tpss_patches* P, int* d_err) {
  const Level& L = ctx->levels[P->level];
  const int n = ctx->n1, nx = L.nc[0], ny = L.nc[1], d = ctx->dim;
  const int64_t nc = L.ncells;
  double* hb = nullptr;
  TPSS_TRY(dalloc_t(&hb, (size_t)d * nc));
  tpss_status st = TPSS_OK;
  if (d == 3) {
    st = mapped3_surrogate_widths(ctx, P->level, hb);
  } else {
    const int gb = (int)std::min<int64_t>((nc + 255) / 256, 4096);
    surrogate_widths_kernel<<<gb, 256, 0, ctx->stream>>>(reinterpret_cast<const double2*>(L.d_verts), nx, ny, hb,
                                                         hb + nc);
  }
  for (int t = 0; t < d && st == TPSS_OK; ++t) {
    if ((st = dalloc_t(&P->d_A[t], (size_t)nc * n * n)) != TPSS_OK) break;
    if ((st = dalloc_t(&P->d_M[t], (size_t)nc * n * n)) != TPSS_OK) break;
    if ((st = dalloc_t(&P->d_Z[t], (size_t)nc * n * n)) != TPSS_OK) break;
    if ((st = dalloc_t(&P->d_lam[t], (size_t)nc * n)) != TPSS_OK) break;
    surrogate_op1d_kernel<<<(unsigned)nc, 64, 0, ctx->stream>>>(ctx->d_basis, hb + t * nc, nx, ny, L.nc[2], t,
                                                                penalty_prefactor(ctx), P->d_M[t], P->d_A[t]);
    const int warps = 4;
    const size_t smem = (size_t)warps * 3 * n * n * sizeof(double);
    gen_eig_kernel<<<(unsigned)((nc + warps - 1) / warps), warps * 32, smem, ctx->stream>>>(
        P->d_A[t], P->d_M[t], (int)nc, n, P->d_Z[t], P->d_lam[t], d_err);
  }
  if (st == TPSS_OK) st = dalloc_t(&P->d_inv, (size_t)nc * (d == 3 ? n * n * n : n * n));
  if (st == TPSS_OK) {
    if (d == 3) st = mapped3_inv_table(ctx, P);
    else inv_table_cells_kernel<<<2048, 256, 0, ctx->stream>>>(P->d_lam[0], P->d_lam[1], n, nc, P->d_inv);
  }
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(ctx->stream);   // hb is freed below
  dfree(hb);
  if (st != TPSS_OK) return st;
  if (e != cudaSuccess) {
    set_error(std::string("surrogate cell solvers: ") + cudaGetErrorString(e));
    return TPSS_ECUDA;
  }
  return TPSS_OK;
}

// ------------------------------------------------------- right-hand side
// kind 0: f = 2 pi^2 sin(pi x) sin(pi y), g = 0 on the mesh's boundary
// (exact solution sin(pi x) sin(pi y) when the mesh covers the unit square),
// integrated with the (k+2)-point Gauss rule per direction on the mapped cell.
__global__ void mapped_rhs_kernel(const Basis1D* __restrict__ B, const double2* __restrict__ V, int nx,
                                  double* __restrict__ b) {
  extern __shared__ double sm[];
  const int n1 = B->n1, nq = B->nq_rhs;
  const int64_t c = blockIdx.x;
  const int i = (int)(c % nx), j = (int)(c / nx);
  Quad Q;
  Q.v0 = V[(int64_t)j * (nx + 1) + i];
  Q.v1 = V[(int64_t)j * (nx + 1) + i + 1];
  Q.v2 = V[(int64_t)(j + 1) * (nx + 1) + i];
  Q.v3 = V[(int64_t)(j + 1) * (nx + 1) + i + 1];
  double* F = sm;            // nq^2
  double* G = F + nq * nq;   // n1 nq
  const double pi = 3.14159265358979323846;
  for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
    const double xa = B->xr[e % nq], xb = B->xr[e / nq];
    double Ji[4];
    const double det = inverse_jacobian(Q, xa, xb, Ji);
    const double px = Q.v0.x * (1 - xa) * (1 - xb) + Q.v1.x * xa * (1 - xb) + Q.v2.x * (1 - xa) * xb + Q.v3.x * xa * xb;
    const double py = Q.v0.y * (1 - xa) * (1 - xb) + Q.v1.y * xa * (1 - xb) + Q.v2.y * (1 - xa) * xb + Q.v3.y * xa * xb;
    F[e] = B->wr[e % nq] * B->wr[e / nq] * fabs(det) * 2.0 * pi * pi * sin(pi * px) * sin(pi * py);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n1 * nq; e += blockDim.x) {
    const int i0 = e % n1, q1 = e / n1;
    double s = 0.0;
    for (int q0 = 0; q0 < nq; ++q0) s += B->Vr[q0 * n1 + i0] * F[q0 + nq * q1];
    G[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n1 * n1; e += blockDim.x) {
    const int i0 = e % n1, i1 = e / n1;
    double s = 0.0;
    for (int q1 = 0; q1 < nq; ++q1) s += B->Vr[q1 * n1 + i1] * G[i0 + n1 * q1];
    b[c * n1 * n1 + e] = s;
  }
}

tpss_status mapped_rhs(tpss_ctx* ctx, int level, int kind, double* b) {
  TPSS_REQUIRE(kind == 0, "tpss_assemble_rhs: mapped meshes support kind 0 only");
  if (ctx->dim == 3) return mapped3_rhs(ctx, level, b);
  const Level& L = ctx->levels[level];
  const int nq = ctx->n1 + 1;
  const size_t smem = (size_t)(nq * nq + ctx->n1 * nq) * sizeof(double);
  mapped_rhs_kernel<<<(unsigned)L.ncells, 128, smem, ctx->stream>>>(
      ctx->d_basis, reinterpret_cast<const double2*>(L.d_verts), L.nc[0], b);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

}  // namespace tpss

using namespace tpss;

// J of the d-linear map at reference point xi (host, for the validity check)
static double host_det(int d, const double* const* c, const double* xi) {
  double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < (1 << d); ++k)
    for (int s2 = 0; s2 < d; ++s2) {
      double g = 1.0;
      for (int t = 0; t < d; ++t) {
        const int a = (k >> t) & 1;
        g *= t == s2 ? (a ? 1.0 : -1.0) : (a ? xi[t] : 1.0 - xi[t]);
      }
      for (int r = 0; r < d; ++r) J[d * r + s2] += c[k][r] * g;
    }
  if (d == 2) return J[0] * J[3] - J[1] * J[2];
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
}

extern "C" tpss_status tpss_create_mapped(int dim, int degree, const int ncells[3], const double* vertices,
                                          int nlevels, double gamma_hat, int penalty_poly, void* cuda_stream,
                                          tpss_ctx** out) {
  clear_error();
  TPSS_REQUIRE(vertices && out && ncells, "tpss_create_mapped: null argument");
  *out = nullptr;
  TPSS_REQUIRE(dim == 2 || dim == 3, "tpss_create_mapped: dim must be 2 or 3");
  TPSS_REQUIRE(degree >= 1 && degree <= (dim == 2 ? kMaxDegree : kMaxMappedDegree3),
               "tpss_create_mapped: degree must be in 1..15 (dim 2) or 1..7 (dim 3)");
  TPSS_REQUIRE(nlevels >= 1 && nlevels <= 12, "tpss_create_mapped: nlevels must be in 1..12");
  int nc[3] = {1, 1, 1};
  size_t nverts = 1;
  for (int t = 0; t < dim; ++t) {
    nc[t] = ncells[t];
    TPSS_REQUIRE(nc[t] >= 1, "tpss_create_mapped: ncells must be >= 1");
    TPSS_REQUIRE(((long long)nc[t] << (nlevels - 1)) <= 1024,
                 "tpss_create_mapped: at most 1024 cells per direction on the finest level");
    nverts *= (size_t)(nc[t] + 1);
  }
  for (size_t i = 0; i < (size_t)dim * nverts; ++i)
    TPSS_REQUIRE(std::isfinite(vertices[i]), "tpss_create_mapped: vertices must be finite");
  // every cell positively oriented: det J > 0 at its 2^d corners (for d = 2
  // this is convexity with the corners v0, v1, v3, v2 counter-clockwise)
  const int sx = nc[0] + 1, sy = nc[1] + 1;
  for (int l = 0; l < nc[2]; ++l)
    for (int j = 0; j < nc[1]; ++j)
      for (int i = 0; i < nc[0]; ++i) {
        const double* c[8];
        for (int k = 0; k < (1 << dim); ++k)
          c[k] = &vertices[(size_t)dim * (((size_t)(l + (k >> 2)) * sy + (j + ((k >> 1) & 1))) * sx + i + (k & 1))];
        for (int k = 0; k < (1 << dim); ++k) {
          const double xi[3] = {(double)(k & 1), (double)((k >> 1) & 1), (double)((k >> 2) & 1)};
          TPSS_REQUIRE(host_det(dim, c, xi) > 0.0,
                       "tpss_create_mapped: cells must be convex and positively oriented (det J > 0 at the corners)");
        }
      }
  std::vector<double> w[3];
  tpss_problem_desc desc{};
  desc.dim = dim;
  desc.degree = degree;
  for (int t = 0; t < 3; ++t) {
    desc.ncells[t] = nc[t];
    w[t].assign(nc[t], 1.0 / nc[t]);
    desc.widths[t] = w[t].data();
  }
  desc.nlevels = nlevels;
  desc.gamma_hat = gamma_hat;
  desc.penalty_poly = penalty_poly;
  tpss_ctx* ctx = nullptr;
  TPSS_TRY(tpss_create(&desc, cuda_stream, &ctx));
  ctx->mapped = 1;
  auto fail = [&](tpss_status s) {
    tpss_destroy(ctx);
    return s;
  };
  tpss_status st;
  for (int l = 0; l < nlevels; ++l) {
    Level& L = ctx->levels[l];
    size_t nv = 1;
    for (int t = 0; t < dim; ++t) nv *= (size_t)(L.nc[t] + 1);
    if ((st = dalloc_t(&L.d_verts, dim * nv)) != TPSS_OK) return fail(st);
    if (l == 0) {
      if (cudaMemcpyAsync(L.d_verts, vertices, dim * nv * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) !=
          cudaSuccess) {
        set_error("tpss_create_mapped: vertex upload failed");
        return fail(TPSS_ECUDA);
      }
    } else {
      const Level& C = ctx->levels[l - 1];
      if (dim == 3) {
        if ((st = mapped3_refine(C.d_verts, C.nc[0], C.nc[1], C.nc[2], L.d_verts, ctx->stream)) != TPSS_OK)
          return fail(st);
      } else {
        refine_vertices_kernel<<<(unsigned)std::min<size_t>((nv + 255) / 256, 4096), 256, 0, ctx->stream>>>(
            reinterpret_cast<const double2*>(C.d_verts), C.nc[0], C.nc[1], reinterpret_cast<double2*>(L.d_verts));
      }
    }
  }
  for (int l = 0; l < nlevels; ++l) {
    Level& L = ctx->levels[l];
    if (dim == 3) {
      if ((st = mapped3_setup_level(ctx, l, penalty_prefactor(ctx))) != TPSS_OK) return fail(st);
      continue;
    }
    if ((st = dalloc_t(&L.d_geo, (size_t)L.ncells * GeoLayout(ctx->n1).G)) != TPSS_OK) return fail(st);
    mapped_geometry_kernel<<<(unsigned)L.ncells, 64, 0, ctx->stream>>>(
        ctx->d_basis, reinterpret_cast<const double2*>(L.d_verts), L.nc[0], L.nc[1], penalty_prefactor(ctx),
        L.d_geo);
  }
  for (int l = 0; l < nlevels; ++l) {   // FP32 copy for the mixed-precision V-cycle
    Level& L = ctx->levels[l];
    const size_t g = (size_t)L.ncells * (dim == 3 ? (size_t)(6 * ctx->n1 + 24) * ctx->n1 * ctx->n1 + 6
                                                   : (size_t)GeoLayout(ctx->n1).G);
    if ((st = dalloc_t(&L.d_geo32, g)) != TPSS_OK) return fail(st);
    to_float_kernel<<<(unsigned)std::min<size_t>((g + 255) / 256, 4096), 256, 0, ctx->stream>>>(L.d_geo, L.d_geo32, g);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    set_error("tpss_create_mapped: vertex refinement or geometry setup failed");
    return fail(TPSS_ECUDA);
  }
  *out = ctx;
  return TPSS_OK;
}

extern "C" tpss_status tpss_mapped_vertices(const tpss_ctx* ctx, int level, double* vertices) {
  clear_error();
  TPSS_REQUIRE(ctx && vertices, "tpss_mapped_vertices: null argument");
  TPSS_REQUIRE(ctx->mapped, "tpss_mapped_vertices: not a mapped mesh");
  TPSS_REQUIRE(level >= 0 && level < ctx->nlevels, "tpss_mapped_vertices: level out of range");
  const Level& L = ctx->levels[level];
  size_t nv = 1;
  for (int t = 0; t < ctx->dim; ++t) nv *= (size_t)(L.nc[t] + 1);
  TPSS_CHECK_CUDA(cudaMemcpyAsync(vertices, L.d_verts, ctx->dim * nv * sizeof(double), cudaMemcpyDeviceToHost,
                                  ctx->stream));
  TPSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  return TPSS_OK;
}
