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
// The scaling on the color's own cells is done by the patch kernels as they
// scatter.  The cells next to the color come from per-color lists built at
// setup ({cell, mask of its faces to the color}); a CTA takes several of
// them, one thread per line normal to the face being processed, accumulates
// the correction in shared memory and applies it to r_K once.  Exact up to
// rounding (parity with the full-residual sweep is tested); not valid for the
// face-conflicting 2^d-color vertex coloring, which keeps the full residual.
#include "tpss_internal.cuh"

namespace tpss {

template <typename T>
struct MultUpdateArgsT {
  const T* M[3];        // level cell mass matrices per direction and position
  const T* F[3];        // face coefficients per direction and position
  const T* d0;
  const T* d1;
  int nc[3];
  int64_t ndofs;
  const int2* list;     // {cell, face mask} of the cells next to the color
  int count;
  const T* dx;          // the color's update d (valid on the color's cells)
  T* r;                 // residual, updated in place
};

// Cells per CTA: about 256 threads with one thread per line normal to a face.
template <int DIM, int N1>
struct FluxShape {
  static constexpr int NT = DIM == 3 ? N1 * N1 : N1;
  static constexpr int NLOC = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
  static constexpr int CPB = NT >= 256 ? 1 : 256 / NT;
  static constexpr int SLOT = 2 * NLOC + 4 * NT;   // per cell: d_N, correction, 4 face arrays
};

// index in a cell tensor (first index fastest) with index `it` along the
// face normal t and (iu, iw) along the tangential directions u < w
template <int DIM, int N1>
__device__ __forceinline__ int face_idx(int t, int it, int iu, int iw) {
  int ii[3] = {0, 0, 0};
  const int u = t == 0 ? 1 : 0, w = t == 2 ? 1 : 2;
  ii[t] = it;
  ii[u] = iu;
  if (DIM == 3) ii[w] = iw;
  return DIM == 3 ? ii[0] + N1 * (ii[1] + N1 * ii[2]) : ii[0] + N1 * ii[1];
}

template <int DIM, int N1, typename T>
__global__ void __launch_bounds__(FluxShape<DIM, N1>::CPB * FluxShape<DIM, N1>::NT)
mult_update_kernel(MultUpdateArgsT<T> a) {
  using S = FluxShape<DIM, N1>;
  constexpr int NT = S::NT, NLOC = S::NLOC;
  extern __shared__ unsigned char smu_raw[];
  const int slot = threadIdx.x / NT, lt = threadIdx.x % NT;
  const int q = blockIdx.x * S::CPB + slot;
  const bool valid = q < a.count;
  T* dn = reinterpret_cast<T*>(smu_raw) + slot * S::SLOT;   // neighbour's d
  T* acc = dn + NLOC;                                       // correction of r_K
  T* s0 = acc + NLOC;
  T* s1 = s0 + NT;
  T* tmp0 = s1 + NT;
  T* tmp1 = tmp0 + NT;
  const int64_t vbase = (int64_t)blockIdx.y * a.ndofs;
  int2 ent = make_int2(0, 0);
  int m[3] = {0, 0, 0};
  if (valid) {
    ent = a.list[q];
    int64_t rest = ent.x;
    for (int t = 0; t < DIM; ++t) {
      m[t] = (int)(rest % a.nc[t]);
      rest /= a.nc[t];
    }
    for (int e = lt; e < NLOC; e += NT) acc[e] = T(0);
  }
  const int64_t cstride[3] = {1, a.nc[0], (int64_t)a.nc[0] * a.nc[1]};
  const int iu = lt % N1, iw = DIM == 3 ? lt / N1 : 0;
  // face slots in a fixed order for every cell of the CTA (uniform barriers);
  // unrolled so that the direction t is a constant in the index arithmetic
#pragma unroll
  for (int fs = 0; fs < 2 * DIM; ++fs) {
    const int t = fs / 2, side = fs % 2;
    const bool on = valid && ((ent.y >> fs) & 1);
    __syncthreads();   // dn and the face arrays are free
    if (on) {
      const T* dN = a.dx + vbase + ((int64_t)ent.x + (side ? cstride[t] : -cstride[t])) * NLOC;
      for (int e = lt; e < NLOC; e += NT) dn[e] = dN[e];
    }
    __syncthreads();
    if (on) {
      // end value and end derivative of the neighbour's line (right
      // neighbour: value at 0, derivative d0; left neighbour: at k, d1)
      const T* dv = side ? a.d0 : a.d1;
      T v1 = T(0);
#pragma unroll
      for (int j = 0; j < N1; ++j) v1 = fma(dv[j], dn[face_idx<DIM, N1>(t, j, iu, iw)], v1);
      s0[lt] = dn[face_idx<DIM, N1>(t, side ? 0 : N1 - 1, iu, iw)];
      s1[lt] = v1;
    }
    __syncthreads();
    T q0 = T(0), q1 = T(0);
    if (on) {   // K's tangential mass along u
      const int u = t == 0 ? 1 : 0;
      const T* Mu = a.M[u] + (size_t)m[u] * N1 * N1;
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        const T mm = Mu[iu * N1 + j];
        q0 = fma(mm, s0[j + N1 * iw], q0);
        q1 = fma(mm, s1[j + N1 * iw], q1);
      }
      if (DIM == 3) {
        tmp0[lt] = q0;
        tmp1[lt] = q1;
      }
    }
    if (DIM == 3) {
      __syncthreads();
      if (on) {   // ... and along w
        const int w = t == 2 ? 1 : 2;
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
    }
    if (on) {   // rank-2 coupling F_t at K's position along t, into K's normal line
      const T* f = a.F[t] + (size_t)m[t] * kFaceCoef;
      if (side) {   // right neighbour: row k gets f0 v + f1 d0.v, every row d1_i f2 v
        const T c = f[2] * q0;
#pragma unroll
        for (int i = 0; i < N1; ++i) acc[face_idx<DIM, N1>(t, i, iu, iw)] += a.d1[i] * c;
        acc[face_idx<DIM, N1>(t, N1 - 1, iu, iw)] += f[0] * q0 + f[1] * q1;
      } else {      // left neighbour: row 0 gets f3 v + f4 d1.v, every row d0_i f5 v
        const T c = f[5] * q0;
#pragma unroll
        for (int i = 0; i < N1; ++i) acc[face_idx<DIM, N1>(t, i, iu, iw)] += a.d0[i] * c;
        acc[face_idx<DIM, N1>(t, 0, iu, iw)] += f[3] * q0 + f[4] * q1;
      }
    }
  }
  __syncthreads();
  if (valid) {
    T* rK = a.r + vbase + (int64_t)ent.x * NLOC;
    for (int e = lt; e < NLOC; e += NT) rK[e] -= acc[e];
  }
}

template <int DIM, int N1, typename T>
static tpss_status launch_update(const MultUpdateArgsT<T>& a, int nrhs, cudaStream_t s) {
  using S = FluxShape<DIM, N1>;
  constexpr size_t smem = (size_t)S::CPB * S::SLOT * sizeof(T);
  static bool attr = false;
  if (smem > 48 * 1024 && !attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(mult_update_kernel<DIM, N1, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  if (a.count <= 0) return TPSS_OK;
  dim3 grid((unsigned)((a.count + S::CPB - 1) / S::CPB), (unsigned)nrhs);
  mult_update_kernel<DIM, N1, T><<<grid, S::CPB * S::NT, smem, s>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

template <typename T>
tpss_status mult_residual_update(tpss_patches* P, int color, int nrhs, const T* dx, T* r, cudaStream_t s) {
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
  a.list = P->d_flux_list + P->flux_offsets[color];
  a.count = P->flux_offsets[color + 1] - P->flux_offsets[color];
  a.dx = dx;
  a.r = r;
  const int n1 = ctx->n1;
#define TPSS_MU_CASE(D, N)                                                     \
  if (ctx->dim == D && n1 == N) return launch_update<D, N, T>(a, nrhs, s);
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

template tpss_status mult_residual_update<double>(tpss_patches*, int, int, const double*, double*, cudaStream_t);
template tpss_status mult_residual_update<float>(tpss_patches*, int, int, const float*, float*, cudaStream_t);

}  // namespace tpss
