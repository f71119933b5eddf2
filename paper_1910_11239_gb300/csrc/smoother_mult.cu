// Residual updates between the colors of the multiplicative smoother.
//
// Alg. 3 / eq. coloredschwarz recompute r = b - A x before every color.  On a
// Cartesian mesh this is avoidable: the colorings used here (red-black
// cells; the 2^(d+1)-color vertex-patch coloring of Sec. 2.3) never put two
// face-adjacent cells into different subdomains of one color, and the local
// solvers are exact (A_j^{-1} by fast diagonalization, Sec. 3.2).  After the
// color's local solves x += d, d = omega sum_j R_j^T A_j^{-1} R_j r, so
//   * on every cell of a subdomain j of the color:  R_j (A d) = A_j d_j
//     = omega R_j r, hence r_new = (1 - omega) r there;
//   * on a cell K outside the color, A d collects only the face couplings of
//     eq. bfsipg across K's faces to cells N of the color.  In the Kronecker
//     form of the operator the coupling across a face normal to t is
//     M_(t2) x M_(t1) x F_t, with F_t the rank-2 1D coupling of eq. 1DsipgVP
//     (end value and end derivative of the neighbour's line) and the
//     tangential factors K's own cell mass matrices, so
//       r_K -= (M x M x F_t) d_N   over those faces,
//     which costs O((k+1)^3) per face instead of an operator application.
// One CTA per (cell, right-hand side), one thread per line normal to the
// face being processed; the correction is accumulated in shared memory and
// applied to r_K once.  Exact up to rounding (parity with the full-residual
// sweep is tested); not valid for the face-conflicting 2^d-color vertex
// coloring, which keeps the full residual.
#include "tpss_internal.cuh"

namespace tpss {

template <typename T>
struct MultUpdateArgsT {
  const T* M[3];
  const T* F[3];
  const T* d0;
  const T* d1;
  int nc[3];
  int64_t ndofs;
  int vertex;
  int color;
  const T* dx;          // the color's update d (valid on the color's cells)
  T* r;                 // residual, updated in place
  T one_minus_omega;
};

// Is cell m (multi-index) in a subdomain of color `color`?
template <int DIM>
__device__ __forceinline__ bool in_color(const int* m, const int* nc, int vertex, int color) {
  if (!vertex) {
    int s = 0;
    for (int t = 0; t < DIM; ++t) s += m[t];
    return (s & 1) == color;
  }
  // vertex v_t in {m_t, m_t + 1} with the color's parity bit; interior only
  int extra = 0;
  for (int t = 0; t < DIM; ++t) {
    const int bit = (color >> t) & 1;
    const int v = ((m[t] & 1) == bit) ? m[t] : m[t] + 1;
    if (v < 1 || v > nc[t] - 1) return false;
    extra += v / 2;
  }
  return (extra & 1) == ((color >> DIM) & 1);
}

// index of (i0, i1, i2) in a cell tensor, first index fastest
template <int N1>
__device__ __forceinline__ int cidx(int i0, int i1, int i2) { return i0 + N1 * (i1 + N1 * i2); }

template <int DIM, int N1, typename T>
__global__ void __launch_bounds__(DIM == 3 ? N1 * N1 : N1) mult_update_kernel(MultUpdateArgsT<T> a) {
  constexpr int NLOC = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
  constexpr int NT = DIM == 3 ? N1 * N1 : N1;   // lines normal to a face
  extern __shared__ unsigned char smu_raw[];
  T* dn = reinterpret_cast<T*>(smu_raw);   // neighbour's d, NLOC
  T* acc = dn + NLOC;                      // correction of r_K, NLOC
  T* s0 = acc + NLOC;                      // face arrays, NT each
  T* s1 = s0 + NT;
  T* tmp0 = s1 + NT;
  T* tmp1 = tmp0 + NT;
  const int tid = threadIdx.x;
  const int64_t cell = blockIdx.x;
  const int64_t vbase = (int64_t)blockIdx.y * a.ndofs;
  int m[3] = {0, 0, 0};
  {
    int64_t rest = cell;
    for (int t = 0; t < DIM; ++t) {
      m[t] = (int)(rest % a.nc[t]);
      rest /= a.nc[t];
    }
  }
  T* rK = a.r + vbase + cell * NLOC;
  if (in_color<DIM>(m, a.nc, a.vertex, a.color)) {
    for (int e = tid; e < NLOC; e += NT) rK[e] *= a.one_minus_omega;
    return;
  }
  // faces to cells of the color
  int faces = 0;
  for (int t = 0; t < DIM; ++t)
    for (int side = 0; side < 2; ++side) {
      int mn[3] = {m[0], m[1], m[2]};
      mn[t] += side ? 1 : -1;
      if (mn[t] < 0 || mn[t] >= a.nc[t]) continue;
      if (in_color<DIM>(mn, a.nc, a.vertex, a.color)) faces |= 1 << (2 * t + side);
    }
  if (faces == 0) return;
  for (int e = tid; e < NLOC; e += NT) acc[e] = T(0);
  int64_t cstride[3] = {1, a.nc[0], (int64_t)a.nc[0] * a.nc[1]};
  for (int t = 0; t < DIM; ++t)
    for (int side = 0; side < 2; ++side) {
      if (!(faces & (1 << (2 * t + side)))) continue;
      const int64_t nb = cell + (side ? cstride[t] : -cstride[t]);
      __syncthreads();   // dn and the face arrays are free
      const T* dN = a.dx + vbase + nb * NLOC;
      for (int e = tid; e < NLOC; e += NT) dn[e] = dN[e];
      __syncthreads();
      // tangential directions u < w (w unused in 2D); this thread's line
      const int u = t == 0 ? 1 : 0;
      const int w = t == 2 ? 1 : 2;
      const int iu = tid % N1, iw = DIM == 3 ? tid / N1 : 0;
      auto at = [&](int it, int uu, int ww) {   // cell index with normal index it
        int ii[3] = {0, 0, 0};
        ii[t] = it;
        ii[u] = uu;
        if (DIM == 3) ii[w] = ww;
        return DIM == 3 ? cidx<N1>(ii[0], ii[1], ii[2]) : ii[0] + N1 * ii[1];
      };
      // end value and end derivative of the neighbour's line (right
      // neighbour: value at 0, derivative d0; left neighbour: at k, d1)
      const T* dv = side ? a.d0 : a.d1;
      T v0 = dn[at(side ? 0 : N1 - 1, iu, iw)], v1 = T(0);
#pragma unroll
      for (int j = 0; j < N1; ++j) v1 = fma(dv[j], dn[at(j, iu, iw)], v1);
      s0[tid] = v0;
      s1[tid] = v1;
      __syncthreads();
      // tangential mass matrices of K: along u, then along w (3D)
      const T* Mu = a.M[u] + (size_t)m[u] * N1 * N1;
      T q0 = T(0), q1 = T(0);
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        const T mm = Mu[iu * N1 + j];
        q0 = fma(mm, s0[j + N1 * iw], q0);
        q1 = fma(mm, s1[j + N1 * iw], q1);
      }
      if (DIM == 3) {
        tmp0[tid] = q0;
        tmp1[tid] = q1;
        __syncthreads();
        const T* Mw = a.M[w] + (size_t)m[w] * N1 * N1;
        q0 = T(0);
        q1 = T(0);
#pragma unroll
        for (int j = 0; j < N1; ++j) {
          const T mm = Mw[iw * N1 + j];
          q0 = fma(mm, tmp0[iu + N1 * j], q0);
          q1 = fma(mm, tmp1[iu + N1 * j], q1);
        }
      }
      // rank-2 coupling F_t of K's position along t into K's normal line
      const T* f = a.F[t] + (size_t)m[t] * kFaceCoef;
      if (side) {   // neighbour on the right: row k gets f0 v + f1 d0.v, all rows d1_i f2 v
        const T c = f[2] * q0;
#pragma unroll
        for (int i = 0; i < N1; ++i) acc[at(i, iu, iw)] += a.d1[i] * c;
        acc[at(N1 - 1, iu, iw)] += f[0] * q0 + f[1] * q1;
      } else {      // neighbour on the left: row 0 gets f3 v + f4 d1.v, all rows d0_i f5 v
        const T c = f[5] * q0;
#pragma unroll
        for (int i = 0; i < N1; ++i) acc[at(i, iu, iw)] += a.d0[i] * c;
        acc[at(0, iu, iw)] += f[3] * q0 + f[4] * q1;
      }
    }
  __syncthreads();
  for (int e = tid; e < NLOC; e += NT) rK[e] -= acc[e];
}

template <int DIM, int N1, typename T>
static tpss_status launch_update(const MultUpdateArgsT<T>& a, int64_t ncells, int nrhs, cudaStream_t s) {
  constexpr int NLOC = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
  constexpr int NT = DIM == 3 ? N1 * N1 : N1;
  constexpr size_t smem = (size_t)(2 * NLOC + 4 * NT) * sizeof(T);
  static bool attr = false;
  if (smem > 48 * 1024 && !attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(mult_update_kernel<DIM, N1, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  dim3 grid((unsigned)ncells, (unsigned)nrhs);
  mult_update_kernel<DIM, N1, T><<<grid, NT, smem, s>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

template <typename T>
tpss_status mult_residual_update(tpss_patches* P, int color, T omega, int nrhs, const T* dx, T* r, cudaStream_t s) {
  const tpss_ctx* ctx = P->ctx;
  const Level& L = ctx->levels[P->level];
  MultUpdateArgsT<T> a{};
  for (int t = 0; t < 3; ++t) {
    if constexpr (sizeof(T) == sizeof(double)) {
      a.M[t] = L.op64.M[t];
      a.F[t] = L.op64.F[t];
    } else {
      a.M[t] = L.op32.M[t];
      a.F[t] = L.op32.F[t];
    }
    a.nc[t] = t < ctx->dim ? L.nc[t] : 1;
  }
  if constexpr (sizeof(T) == sizeof(double)) {
    a.d0 = L.op64.d0;
    a.d1 = L.op64.d1;
  } else {
    a.d0 = L.op32.d0;
    a.d1 = L.op32.d1;
  }
  a.ndofs = L.ndofs;
  a.vertex = P->kind == TPSS_VERTEX_PATCH;
  a.color = color;
  a.dx = dx;
  a.r = r;
  a.one_minus_omega = T(1) - omega;
  const int n1 = ctx->n1;
#define TPSS_MU_CASE(D, N)                                                     \
  if (ctx->dim == D && n1 == N) return launch_update<D, N, T>(a, L.ncells, nrhs, s);
  TPSS_MU_CASE(3, 2) TPSS_MU_CASE(3, 3) TPSS_MU_CASE(3, 4) TPSS_MU_CASE(3, 5)
  TPSS_MU_CASE(3, 6) TPSS_MU_CASE(3, 7) TPSS_MU_CASE(3, 8)
  TPSS_MU_CASE(2, 2) TPSS_MU_CASE(2, 3) TPSS_MU_CASE(2, 4) TPSS_MU_CASE(2, 5)
  TPSS_MU_CASE(2, 6) TPSS_MU_CASE(2, 7) TPSS_MU_CASE(2, 8)
  if constexpr (sizeof(T) == sizeof(double)) {
    TPSS_MU_CASE(3, 9) TPSS_MU_CASE(3, 10) TPSS_MU_CASE(3, 11) TPSS_MU_CASE(3, 12)
    TPSS_MU_CASE(3, 13) TPSS_MU_CASE(3, 14) TPSS_MU_CASE(3, 15) TPSS_MU_CASE(3, 16)
    TPSS_MU_CASE(2, 9) TPSS_MU_CASE(2, 10) TPSS_MU_CASE(2, 11) TPSS_MU_CASE(2, 12)
    TPSS_MU_CASE(2, 13) TPSS_MU_CASE(2, 14) TPSS_MU_CASE(2, 15) TPSS_MU_CASE(2, 16)
  }
#undef TPSS_MU_CASE
  set_error("multiplicative smoother: unsupported degree for the residual update");
  return TPSS_EINVAL;
}

template tpss_status mult_residual_update<double>(tpss_patches*, int, double, int, const double*, double*,
                                                  cudaStream_t);
template tpss_status mult_residual_update<float>(tpss_patches*, int, float, int, const float*, float*,
                                                 cudaStream_t);

}  // namespace tpss
