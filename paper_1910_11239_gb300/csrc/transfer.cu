// Level transfers (Sec. 2.2): prolongation is the embedding V_{l-1} -> V_l,
// restriction its transpose.
//
// A parent cell and its 2^d children form a "patch" of 2(k+1) points per
// direction (child c_t in {0,1}, p_t = c_t (k+1) + i_t).  Along one direction
// the embedding maps the parent's k+1 values to the 2(k+1) child values with
// the 1D matrix [P_0; P_1], (P_s)_{ij} = phi_j((x_i + s)/2) (the parent basis
// evaluated at the child's Gauss-Lobatto points).  The d-dimensional embedding
// is the Kronecker product of these 1D maps and is applied by sum
// factorization, one direction after another (14 (k+1)^4 FMAs per parent in
// 3D); restriction applies the transposed 1D maps in the reverse order.
// One CTA per (right-hand side, parent cell); the tensors live in shared memory.
#include "tpss_internal.cuh"

namespace tpss {

// out = R in along direction t of an (e0, e1, e2) tensor (first index fastest).
// R is rows x cols (row-major) and replaces extent e_t = cols by rows.
template <typename T>
__device__ void contract_dir(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ R,
                             int rows, int cols, int t, int e0, int e1, int e2) {
  int oe[3] = {e0, e1, e2};
  oe[t] = rows;
  const int is[3] = {1, e0, e0 * e1};
  const int os[3] = {1, oe[0], oe[0] * oe[1]};
  const int u = t == 0 ? 1 : 0, v = t == 2 ? 1 : 2;  // the two other directions
  const int nlines = oe[u] * oe[v];
  for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
    const int a = l % oe[u], b = l / oe[u];
    const int ib = a * is[u] + b * is[v], ob = a * os[u] + b * os[v];
    for (int i = 0; i < rows; ++i) {
      T s = 0;
      for (int j = 0; j < cols; ++j) s = fma(R[i * cols + j], in[ib + j * is[t]], s);
      out[ob + i * os[t]] = s;
    }
  }
}

// PROLONG = true: fine += I^up coarse; false: coarse = I^down fine.
template <int DIM, bool PROLONG, typename T>
__global__ void transfer_kernel(const T* __restrict__ src, T* __restrict__ dst, const T* __restrict__ Pc,
                                int n1, int cnc0, int cnc1, int cnc2, int64_t cdofs, int64_t fdofs) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int np = 2 * n1;
  const int big = DIM == 3 ? np * np * np : np * np;
  T* R = sm;                        // [2 n1][n1] = [P_0; P_1]
  T* RT = R + np * n1;              // [n1][2 n1] = transpose
  T* b0 = RT + np * n1;             // big
  T* b1 = b0 + big;                 // big
  const int64_t parent = blockIdx.x;
  const int rhs = blockIdx.y;
  const int cx = (int)(parent % cnc0), cy = (int)((parent / cnc0) % cnc1);
  const int cz = DIM == 3 ? (int)(parent / ((int64_t)cnc0 * cnc1)) : 0;
  const int fnc0 = 2 * cnc0, fnc1 = 2 * cnc1;
  const int nloc = DIM == 3 ? n1 * n1 * n1 : n1 * n1;
  for (int e = threadIdx.x; e < np * n1; e += blockDim.x) {
    const int i = e / n1, j = e % n1;  // R[i][j] = P_{i/n1}[i%n1][j]
    const T v = Pc[(i / n1) * n1 * n1 + (i % n1) * n1 + j];
    R[i * n1 + j] = v;
    RT[j * np + i] = v;
  }
  const int nchild = DIM == 3 ? 8 : 4;
  auto child_base = [&](int c) -> int64_t {
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const int64_t fc = (2 * cx + sx) + (int64_t)fnc0 * ((2 * cy + sy) + (int64_t)fnc1 * (DIM == 3 ? (2 * cz + sz) : 0));
    return (int64_t)rhs * fdofs + fc * nloc;
  };
  auto patch_index = [&](int c, int loc) -> int {
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const int ix = loc % n1, iy = (loc / n1) % n1, iz = loc / (n1 * n1);
    const int px = sx * n1 + ix, py = sy * n1 + iy;
    if (DIM == 3) return px + np * (py + np * (sz * n1 + iz));
    return px + np * py;
  };
  if (PROLONG) {
    const int64_t pbase = (int64_t)rhs * cdofs + parent * nloc;
    for (int e = threadIdx.x; e < nloc; e += blockDim.x) b0[e] = src[pbase + e];
    __syncthreads();
    // x: (n1,n1,n1) -> (2n1,n1,n1); y: -> (2n1,2n1,n1); z: -> (2n1,2n1,2n1)
    contract_dir<T>(b0, b1, R, np, n1, 0, n1, n1, DIM == 3 ? n1 : 1);
    __syncthreads();
    contract_dir<T>(b1, b0, R, np, n1, 1, np, n1, DIM == 3 ? n1 : 1);
    __syncthreads();
    T* res = b0;
    if (DIM == 3) {
      contract_dir<T>(b0, b1, R, np, n1, 2, np, np, n1);
      __syncthreads();
      res = b1;
    }
    for (int e = threadIdx.x; e < nchild * nloc; e += blockDim.x) {
      const int c = e / nloc, loc = e % nloc;
      dst[child_base(c) + loc] += res[patch_index(c, loc)];
    }
  } else {
    for (int e = threadIdx.x; e < nchild * nloc; e += blockDim.x) {
      const int c = e / nloc, loc = e % nloc;
      b0[patch_index(c, loc)] = src[child_base(c) + loc];
    }
    __syncthreads();
    T* res;
    if (DIM == 3) {
      contract_dir<T>(b0, b1, RT, n1, np, 2, np, np, np);   // -> (2n1,2n1,n1)
      __syncthreads();
      contract_dir<T>(b1, b0, RT, n1, np, 1, np, np, n1);   // -> (2n1,n1,n1)
      __syncthreads();
      contract_dir<T>(b0, b1, RT, n1, np, 0, np, n1, n1);   // -> (n1,n1,n1)
      __syncthreads();
      res = b1;
    } else {
      contract_dir<T>(b0, b1, RT, n1, np, 1, np, np, 1);
      __syncthreads();
      contract_dir<T>(b1, b0, RT, n1, np, 0, np, n1, 1);
      __syncthreads();
      res = b0;
    }
    const int64_t pbase = (int64_t)rhs * cdofs + parent * nloc;
    for (int e = threadIdx.x; e < nloc; e += blockDim.x) dst[pbase + e] = res[e];
  }
}

// 3D FP64 transfers for n1 > 8 (k = 8..15), where the two (2 n1)^3 patch
// tensors above no longer fit in shared memory: every child is mapped on its
// own with the n1 x n1 blocks P_{s_x}, P_{s_y}, P_{s_z} of the 1D embedding
// (24 n1^4 FMAs per parent instead of 14 n1^4), so shared memory holds three
// n1^3 tensors.  Restriction accumulates P_{s_x}^T P_{s_y}^T P_{s_z}^T applied
// to each child into the parent tensor.
template <bool PROLONG>
__global__ void transfer_child_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                      const double* __restrict__ Pc, int n1, int cnc0, int cnc1, int64_t cdofs,
                                      int64_t fdofs) {
  extern __shared__ double smc[];
  const int nn = n1 * n1, nloc = nn * n1;
  double* R = smc;            // [2][n1*n1]: P_0, P_1 (prolongation) or their transposes
  double* b0 = R + 2 * nn;    // n1^3
  double* b1 = b0 + nloc;     // n1^3
  double* par = b1 + nloc;    // n1^3: the parent tensor
  const int64_t parent = blockIdx.x;
  const int64_t rhs = blockIdx.y;
  const int cx = (int)(parent % cnc0), cy = (int)((parent / cnc0) % cnc1);
  const int cz = (int)(parent / ((int64_t)cnc0 * cnc1));
  const int fnc0 = 2 * cnc0, fnc1 = 2 * cnc1;
  for (int e = threadIdx.x; e < 2 * nn; e += blockDim.x) {
    const int sd = e / nn, i = (e % nn) / n1, j = e % n1;
    const double v = Pc[e];   // (P_sd)_{ij}
    R[sd * nn + (PROLONG ? i * n1 + j : j * n1 + i)] = v;
  }
  const int64_t pbase = rhs * cdofs + parent * nloc;
  if (PROLONG) {
    for (int e = threadIdx.x; e < nloc; e += blockDim.x) par[e] = src[pbase + e];
  } else {
    for (int e = threadIdx.x; e < nloc; e += blockDim.x) par[e] = 0.0;
  }
  __syncthreads();
  for (int c = 0; c < 8; ++c) {
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const int64_t fc = (2 * cx + sx) + (int64_t)fnc0 * ((2 * cy + sy) + (int64_t)fnc1 * (2 * cz + sz));
    const int64_t cbase = rhs * fdofs + fc * nloc;
    const double* in = par;
    if (!PROLONG) {
      for (int e = threadIdx.x; e < nloc; e += blockDim.x) b0[e] = src[cbase + e];
      __syncthreads();
      in = b0;
    }
    double* t1 = PROLONG ? b0 : b1;
    double* t2 = PROLONG ? b1 : b0;
    contract_dir<double>(in, t1, R + sx * nn, n1, n1, 0, n1, n1, n1);
    __syncthreads();
    contract_dir<double>(t1, t2, R + sy * nn, n1, n1, 1, n1, n1, n1);
    __syncthreads();
    contract_dir<double>(t2, t1, R + sz * nn, n1, n1, 2, n1, n1, n1);
    __syncthreads();
    if (PROLONG) {
      for (int e = threadIdx.x; e < nloc; e += blockDim.x) dst[cbase + e] += t1[e];
    } else {
      for (int e = threadIdx.x; e < nloc; e += blockDim.x) par[e] += t1[e];
    }
    __syncthreads();   // t1 / b0 are overwritten by the next child
  }
  if (!PROLONG)
    for (int e = threadIdx.x; e < nloc; e += blockDim.x) dst[pbase + e] = par[e];
}

template <typename T>
static tpss_status transfer_t(tpss_ctx* ctx, int fine_level, int nrhs, const T* src, T* dst, bool prolong) {
  const Level& C = ctx->levels[fine_level - 1];
  const Level& F = ctx->levels[fine_level];
  const int n1 = ctx->n1, np = 2 * n1;
  if constexpr (sizeof(T) == sizeof(double)) {
    if (ctx->dim == 3 && n1 > 8) {
      const size_t smem = (size_t)(2 * n1 * n1 + 3 * n1 * n1 * n1) * sizeof(double);
      static bool attr = false;
      if (!attr) {
        TPSS_CHECK_CUDA(cudaFuncSetAttribute(transfer_child_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
        TPSS_CHECK_CUDA(cudaFuncSetAttribute(transfer_child_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
        attr = true;
      }
      dim3 grid((unsigned)C.ncells, (unsigned)nrhs);
      if (prolong)
        transfer_child_kernel<true><<<grid, 256, smem, ctx->stream>>>(src, dst, C.op64.Pc, n1, C.nc[0], C.nc[1],
                                                                      C.ndofs, F.ndofs);
      else
        transfer_child_kernel<false><<<grid, 256, smem, ctx->stream>>>(src, dst, C.op64.Pc, n1, C.nc[0], C.nc[1],
                                                                       C.ndofs, F.ndofs);
      TPSS_CHECK_LAUNCH();
      return TPSS_OK;
    }
  }
  const int big = ctx->dim == 3 ? np * np * np : np * np;
  const size_t smem = (size_t)(2 * np * n1 + 2 * big) * sizeof(T);
  const T* Pc;
  if constexpr (sizeof(T) == 8) Pc = reinterpret_cast<const T*>(C.op64.Pc);
  else Pc = reinterpret_cast<const T*>(C.op32.Pc);
  dim3 grid((unsigned)C.ncells, (unsigned)nrhs);
  const int threads = 128;
  if (smem > 48 * 1024) {
    if (ctx->dim == 3) {
      TPSS_CHECK_CUDA(cudaFuncSetAttribute(transfer_kernel<3, true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      TPSS_CHECK_CUDA(cudaFuncSetAttribute(transfer_kernel<3, false, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    } else {
      TPSS_CHECK_CUDA(cudaFuncSetAttribute(transfer_kernel<2, true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      TPSS_CHECK_CUDA(cudaFuncSetAttribute(transfer_kernel<2, false, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
  }
  if (ctx->dim == 3) {
    if (prolong)
      transfer_kernel<3, true, T><<<grid, threads, smem, ctx->stream>>>(src, dst, Pc, n1, C.nc[0], C.nc[1], C.nc[2], C.ndofs, F.ndofs);
    else
      transfer_kernel<3, false, T><<<grid, threads, smem, ctx->stream>>>(src, dst, Pc, n1, C.nc[0], C.nc[1], C.nc[2], C.ndofs, F.ndofs);
  } else {
    if (prolong)
      transfer_kernel<2, true, T><<<grid, threads, smem, ctx->stream>>>(src, dst, Pc, n1, C.nc[0], C.nc[1], 1, C.ndofs, F.ndofs);
    else
      transfer_kernel<2, false, T><<<grid, threads, smem, ctx->stream>>>(src, dst, Pc, n1, C.nc[0], C.nc[1], 1, C.ndofs, F.ndofs);
  }
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

template <typename T>
tpss_status prolongate_add_t(tpss_ctx* ctx, int fine_level, int nrhs, const T* coarse, T* fine) {
  return transfer_t<T>(ctx, fine_level, nrhs, coarse, fine, true);
}
template <typename T>
tpss_status restrict_t(tpss_ctx* ctx, int fine_level, int nrhs, const T* fine, T* coarse) {
  return transfer_t<T>(ctx, fine_level, nrhs, fine, coarse, false);
}
template tpss_status prolongate_add_t<double>(tpss_ctx*, int, int, const double*, double*);
template tpss_status prolongate_add_t<float>(tpss_ctx*, int, int, const float*, float*);
template tpss_status restrict_t<double>(tpss_ctx*, int, int, const double*, double*);
template tpss_status restrict_t<float>(tpss_ctx*, int, int, const float*, float*);

}  // namespace tpss

using namespace tpss;

extern "C" tpss_status tpss_prolongate_add(tpss_ctx* ctx, int fine_level, int nrhs, const double* coarse,
                                           double* fine) {
  clear_error();
  TPSS_REQUIRE(ctx && coarse && fine, "tpss_prolongate_add: null argument");
  TPSS_REQUIRE(fine_level >= 1 && fine_level < ctx->nlevels, "tpss_prolongate_add: fine_level out of range");
  TPSS_REQUIRE(nrhs >= 1 && nrhs <= 65535, "tpss_prolongate_add: nrhs out of range");
  return prolongate_add_t<double>(ctx, fine_level, nrhs, coarse, fine);
}

extern "C" tpss_status tpss_restrict(tpss_ctx* ctx, int fine_level, int nrhs, const double* fine,
                                     double* coarse) {
  clear_error();
  TPSS_REQUIRE(ctx && coarse && fine, "tpss_restrict: null argument");
  TPSS_REQUIRE(fine_level >= 1 && fine_level < ctx->nlevels, "tpss_restrict: fine_level out of range");
  TPSS_REQUIRE(nrhs >= 1 && nrhs <= 65535, "tpss_restrict: nrhs out of range");
  return restrict_t<double>(ctx, fine_level, nrhs, fine, coarse);
}
