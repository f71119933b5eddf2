// BF16 tensor-core patch smoother, 3D (mixed precision; not in the paper).
//
// One CTA owns one subdomain of a color and loops over all right-hand sides.
// The n^3 patch tensor lives in shared memory in BF16 (the MMA rounds its
// operands to BF16 anyway), with x contiguous, line stride LS = 24 and plane
// stride PS = 24 n + 8 elements: every 8-element row starts on a 16-byte
// boundary and 8 rows at stride LS or PS fall into 8 distinct 16-byte bank
// groups, so ldmatrix / stmatrix are conflict-free.  Padding (x >= n) stays
// zero.  Each mode contraction is an MMA m16n8k16 (BF16 in, FP32 accumulate)
// over 16-line tiles:
//   x-lines: A rows = lines (y,z), loaded with ldmatrix, stored with stmatrix;
//   y/z-lines: A rows = 16 consecutive x at fixed (z) / (y), loaded and stored
//              with the .trans forms (the contraction index is strided).
// Contraction index and output index are padded to 16; W (Z or Z^T, zero
// padded) is held in registers as B fragments for the whole subdomain.  The
// z-step Z^T -> Lambda^{-1} -> Z is chained in registers: the FP32
// accumulator of the first MMA, scaled, is the A fragment of the second.  The
// right-hand side and x of the next system are staged into shared memory with
// cp.async while the current one is contracted (double-buffered x), so the
// final x = x_old + omega y is written without a dependent global load.
#include "bf16_tc.cuh"

namespace tpss {

namespace bf {

// x[cell rows] = SX + omega T, one cell row per iteration.  With dr: also
// dr = omega T (the update) and rres *= 1 - omega (the residual after the
// color on the patch), for the multiplicative residual update.
template <int N, int N1, int NCELL>
__device__ __forceinline__ void tensor_to_x(float* __restrict__ xr, float* __restrict__ dr, float* rres,
                                            const __nv_bfloat16* __restrict__ T, const float* __restrict__ SX,
                                            float omega, const CellBase& cb, int tid) {
  using S = Shape<N>;
  constexpr int V = RowVec<N1>::V;
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int NROW = NCELL * N1 * N1;
  for (int rw = tid; rw < NROW; rw += kThreads) {
    const int c = rw / (N1 * N1), rr = rw % (N1 * N1);
    const int iy = rr % N1, iz = rr / N1;
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const float* xo = SX + c * NLOC1 + rr * N1;
    const __nv_bfloat16* t = T + sx * N1 + LS * (sy * N1 + iy) + S::PS * (sz * N1 + iz);
    const int64_t off = cb.template operator()<NLOC1>(c) + rr * N1;
    float* dst = xr + off;
#pragma unroll
    for (int v = 0; v < N1; v += V) {
      if constexpr (V == 4) {
        const float4 a = *reinterpret_cast<const float4*>(xo + v);
        const uint2 tb = *reinterpret_cast<const uint2*>(t + v);
        const float2 t01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&tb.x));
        const float2 t23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&tb.y));
        float4 o;
        o.x = fmaf(omega, t01.x, a.x);
        o.y = fmaf(omega, t01.y, a.y);
        o.z = fmaf(omega, t23.x, a.z);
        o.w = fmaf(omega, t23.y, a.w);
        *reinterpret_cast<float4*>(dst + v) = o;
        if (dr != nullptr) {
          *reinterpret_cast<float4*>(dr + off + v) = make_float4(omega * t01.x, omega * t01.y, omega * t23.x,
                                                                 omega * t23.y);
          float4 rv = *reinterpret_cast<float4*>(rres + off + v);
          const float s = 1.f - omega;
          rv.x *= s; rv.y *= s; rv.z *= s; rv.w *= s;
          *reinterpret_cast<float4*>(rres + off + v) = rv;
        }
      } else if constexpr (V == 2) {
        const float2 a = *reinterpret_cast<const float2*>(xo + v);
        const float2 tt = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(t + v));
        float2 o;
        o.x = fmaf(omega, tt.x, a.x);
        o.y = fmaf(omega, tt.y, a.y);
        *reinterpret_cast<float2*>(dst + v) = o;
        if (dr != nullptr) {
          *reinterpret_cast<float2*>(dr + off + v) = make_float2(omega * tt.x, omega * tt.y);
          float2 rv = *reinterpret_cast<float2*>(rres + off + v);
          rv.x *= 1.f - omega;
          rv.y *= 1.f - omega;
          *reinterpret_cast<float2*>(rres + off + v) = rv;
        }
      } else {
        dst[v] = fmaf(omega, __bfloat162float(t[v]), xo[v]);
        if (dr != nullptr) {
          dr[off + v] = omega * __bfloat162float(t[v]);
          rres[off + v] *= 1.f - omega;
        }
      }
    }
  }
}

// Dynamic shared memory: [T: Shape<N>::TOTAL bf16][SB: NV f32][SX: 2 x NV f32]
template <int N, bool VERTEX>
__global__ void __launch_bounds__(kThreads, 3)
patch_smooth_bf16_kernel(const int* __restrict__ list, const float* __restrict__ Z0, const float* __restrict__ Z1,
                         const float* __restrict__ Z2, const float* __restrict__ L0, const float* __restrict__ L1,
                         const float* __restrict__ L2, const float* __restrict__ r, float* __restrict__ x,
                         float* __restrict__ d, float omega, int nc0, int nc1, int64_t ndofs, int nrhs,
                         int rpc) {
  using S = Shape<N>;
  constexpr int N1 = VERTEX ? N / 2 : N;
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int NCELL = VERTEX ? 8 : 1;
  constexpr int NV = NCELL * NLOC1;
  // right-hand sides [blockIdx.y * rpc, +rpc) of this CTA
  {
    const int64_t off = (int64_t)blockIdx.y * rpc * ndofs;
    r += off;
    x += off;
    if (d != nullptr) d += off;
    nrhs = min(rpc, nrhs - (int)blockIdx.y * rpc);
  }
  extern __shared__ __align__(16) unsigned char dsm[];
  __nv_bfloat16* T = reinterpret_cast<__nv_bfloat16*>(dsm);
  float* SB = reinterpret_cast<float*>(dsm + ((S::TOTAL * 2 + 15) / 16) * 16);
  float* SX = SB + NV;   // two buffers of NV
  __shared__ float lam[3 * N];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int packed = list[blockIdx.x];
  const int px = unpack_x(packed), py = unpack_y(packed), pz = unpack_z(packed);
  const CellBase cbase{px, py, pz, nc0, nc1};
  // first right-hand side: b -> SB, x -> SX[0]
  stage<NLOC1, NCELL>(SB, r, cbase, tid);
  stage<NLOC1, NCELL>(SX, x, cbase, tid);
  cp_async_commit();
  for (int e = tid; e < S::TOTAL; e += kThreads) T[e] = __float2bfloat16(0.f);
  if (tid < 3 * N) {
    const int d = tid / N, i = tid % N;
    const float* Ld = d == 0 ? L0 : (d == 1 ? L1 : L2);
    const int p = d == 0 ? px : (d == 1 ? py : pz);
    lam[tid] = Ld[(size_t)p * N + i];
  }
  uint32_t bx[2][2], bxt[2][2], by[2][2], byt[2][2], bzz[2][2], bzt[2][2];
  load_bfrag<N, false>(bxt, Z0 + (size_t)px * N * N, lane);
  load_bfrag<N, true>(bx, Z0 + (size_t)px * N * N, lane);
  load_bfrag<N, false>(byt, Z1 + (size_t)py * N * N, lane);
  load_bfrag<N, true>(by, Z1 + (size_t)py * N * N, lane);
  load_bfrag<N, false>(bzt, Z2 + (size_t)pz * N * N, lane);
  load_bfrag<N, true>(bzz, Z2 + (size_t)pz * N * N, lane);
  for (int rhs = 0; rhs < nrhs; ++rhs) {
    float* sx_cur = SX + (rhs & 1) * NV;
    cp_async_wait_all();
    __syncthreads();   // staged data visible; previous scatter done with T and the other SX buffer
    rows_to_tensor<N, N1, NCELL>(T, SB, tid);
    __syncthreads();   // SB consumed
    if (rhs + 1 < nrhs) {   // prefetch the next right-hand side and its x while computing this one
      stage<NLOC1, NCELL>(SB, r + (int64_t)(rhs + 1) * ndofs, cbase, tid);
      stage<NLOC1, NCELL>(SX + ((rhs + 1) & 1) * NV, x + (int64_t)(rhs + 1) * ndofs, cbase, tid);
      cp_async_commit();
    }
    contract<N, 0>(T, bxt, warp, lane);
    __syncthreads();
    contract<N, 1>(T, byt, warp, lane);
    __syncthreads();
    zstep<N>(T, bzt, bzz, lam, warp, lane);
    __syncthreads();
    contract<N, 1>(T, by, warp, lane);
    __syncthreads();
    contract<N, 0>(T, bx, warp, lane);
    __syncthreads();
    tensor_to_x<N, N1, NCELL>(x + (int64_t)rhs * ndofs, d ? d + (int64_t)rhs * ndofs : nullptr,
                              const_cast<float*>(r) + (int64_t)rhs * ndofs, T, sx_cur, omega, cbase, tid);
  }
}

// One (subdomain, right-hand side) per CTA over ALL subdomains in one launch,
// x accumulated with FP32 vector atomics instead of colored read-modify-write
// launches.  With the subdomains in lexicographic order the 2^d patches that
// share a cell run close together in time, so the cell's r and x stay in L2
// across them and HBM sees each vector about once per call instead of once
// per color; the summation order of the 2^d contributions then varies from
// run to run (FP32 rounding).
template <int N, bool VERTEX>
__global__ void __launch_bounds__(kThreads, 4)
patch_smooth_bf16_atomic_kernel(const int* __restrict__ list, const float* __restrict__ Z0,
                                const float* __restrict__ Z1, const float* __restrict__ Z2,
                                const float* __restrict__ L0, const float* __restrict__ L1,
                                const float* __restrict__ L2, const float* __restrict__ r, float* __restrict__ x,
                                float omega, int nc0, int nc1, int64_t ndofs) {
  using S = Shape<N>;
  constexpr int N1 = VERTEX ? N / 2 : N;
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int NCELL = VERTEX ? 8 : 1;
  extern __shared__ __align__(16) unsigned char dsm[];
  __nv_bfloat16* T = reinterpret_cast<__nv_bfloat16*>(dsm);
  float* SB = reinterpret_cast<float*>(dsm + ((S::TOTAL * 2 + 15) / 16) * 16);
  __shared__ float lam[3 * N];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int packed = list[blockIdx.x];
  const int px = unpack_x(packed), py = unpack_y(packed), pz = unpack_z(packed);
  const CellBase cbase{px, py, pz, nc0, nc1};
  const int64_t vbase = (int64_t)blockIdx.y * ndofs;
  stage<NLOC1, NCELL>(SB, r + vbase, cbase, tid);
  cp_async_commit();
  for (int e = tid; e < S::TOTAL; e += kThreads) T[e] = __float2bfloat16(0.f);
  if (tid < 3 * N) {
    const int d = tid / N, i = tid % N;
    const float* Ld = d == 0 ? L0 : (d == 1 ? L1 : L2);
    const int p = d == 0 ? px : (d == 1 ? py : pz);
    lam[tid] = Ld[(size_t)p * N + i];
  }
  uint32_t bx[2][2], bxt[2][2], by[2][2], byt[2][2], bzz[2][2], bzt[2][2];
  load_bfrag<N, false>(bxt, Z0 + (size_t)px * N * N, lane);
  load_bfrag<N, true>(bx, Z0 + (size_t)px * N * N, lane);
  load_bfrag<N, false>(byt, Z1 + (size_t)py * N * N, lane);
  load_bfrag<N, true>(by, Z1 + (size_t)py * N * N, lane);
  load_bfrag<N, false>(bzt, Z2 + (size_t)pz * N * N, lane);
  load_bfrag<N, true>(bzz, Z2 + (size_t)pz * N * N, lane);
  cp_async_wait_all();
  __syncthreads();   // staged r, zeroed tensor and lam visible
  rows_to_tensor<N, N1, NCELL>(T, SB, tid);
  __syncthreads();
  contract<N, 0>(T, bxt, warp, lane);
  __syncthreads();
  contract<N, 1>(T, byt, warp, lane);
  __syncthreads();
  zstep<N>(T, bzt, bzz, lam, warp, lane);
  __syncthreads();
  contract<N, 1>(T, by, warp, lane);
  __syncthreads();
  contract<N, 0>(T, bx, warp, lane);
  __syncthreads();
  tensor_atomic_add<N, N1, NCELL>(x + vbase, T, omega, cbase, tid);
}

template <int N, bool VERTEX>
constexpr size_t smem_bytes_atomic() {
  constexpr int N1 = VERTEX ? N / 2 : N;
  constexpr int NV = (VERTEX ? 8 : 1) * N1 * N1 * N1;
  return ((Shape<N>::TOTAL * 2 + 15) / 16) * 16 + (size_t)NV * 4;
}

template <int N, bool VERTEX>
static tpss_status launch_atomic(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                                 float* x, cudaStream_t s) {
  constexpr size_t smem = smem_bytes_atomic<N, VERTEX>();
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(patch_smooth_bf16_atomic_kernel<N, VERTEX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  if (count <= 0) return TPSS_OK;
  const Level& L = P->ctx->levels[P->level];
  dim3 grid((unsigned)count, (unsigned)nrhs);
  patch_smooth_bf16_atomic_kernel<N, VERTEX><<<grid, kThreads, smem, s>>>(
      list, P->d_Z32[0], P->d_Z32[1], P->d_Z32[2], P->d_lam32[0], P->d_lam32[1], P->d_lam32[2], r, x, omega,
      L.nc[0], L.nc[1], L.ndofs);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

template <int N, bool VERTEX>
constexpr size_t smem_bytes() {
  constexpr int N1 = VERTEX ? N / 2 : N;
  constexpr int NV = (VERTEX ? 8 : 1) * N1 * N1 * N1;
  return ((Shape<N>::TOTAL * 2 + 15) / 16) * 16 + 3 * (size_t)NV * 4;
}

template <int N, bool VERTEX>
static tpss_status launch(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                          float* x, float* d, cudaStream_t s, int rpc) {
  constexpr size_t smem = smem_bytes<N, VERTEX>();
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(patch_smooth_bf16_kernel<N, VERTEX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  if (count <= 0) return TPSS_OK;
  const Level& L = P->ctx->levels[P->level];
  if (rpc < 1 || rpc > nrhs) rpc = nrhs;
  dim3 grid((unsigned)count, (unsigned)((nrhs + rpc - 1) / rpc));
  patch_smooth_bf16_kernel<N, VERTEX><<<grid, kThreads, smem, s>>>(
      list, P->d_Z32[0], P->d_Z32[1], P->d_Z32[2], P->d_lam32[0], P->d_lam32[1], P->d_lam32[2], r, x, d, omega,
      L.nc[0], L.nc[1], L.ndofs, nrhs, rpc);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

}  // namespace bf

// One launch over every subdomain of the list with atomic accumulation into x
// (additive smoother); TPSS_EINVAL (without launching) for shapes it does not
// cover or vectors that are not 16-byte aligned.
tpss_status patch_pass_bf16_atomic(tpss_patches* P, const int* list, int count, float omega, int nrhs,
                                   const float* r, float* x, cudaStream_t s) {
  if (P->ctx->dim != 3) return TPSS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(x)) & 15) return TPSS_EINVAL;
  const bool v = P->kind == TPSS_VERTEX_PATCH;
  switch (P->n) {
    case 4: return v ? bf::launch_atomic<4, true>(P, list, count, omega, nrhs, r, x, s)
                     : bf::launch_atomic<4, false>(P, list, count, omega, nrhs, r, x, s);
    case 6: return v ? bf::launch_atomic<6, true>(P, list, count, omega, nrhs, r, x, s)
                     : bf::launch_atomic<6, false>(P, list, count, omega, nrhs, r, x, s);
    case 8: return v ? bf::launch_atomic<8, true>(P, list, count, omega, nrhs, r, x, s)
                     : bf::launch_atomic<8, false>(P, list, count, omega, nrhs, r, x, s);
    case 10: return v ? bf::launch_atomic<10, true>(P, list, count, omega, nrhs, r, x, s) : TPSS_EINVAL;
    case 12: return v ? bf::launch_atomic<12, true>(P, list, count, omega, nrhs, r, x, s) : TPSS_EINVAL;
    case 14: return v ? bf::launch_atomic<14, true>(P, list, count, omega, nrhs, r, x, s) : TPSS_EINVAL;
    case 16: return v ? bf::launch_atomic<16, true>(P, list, count, omega, nrhs, r, x, s) : TPSS_EINVAL;
    default: return TPSS_EINVAL;
  }
}

// 3D BF16 path; returns TPSS_EINVAL (without launching) for shapes it does not cover.
tpss_status patch_pass_bf16(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                            float* x, cudaStream_t s, float* d, int rpc) {
  if (P->ctx->dim != 3) return TPSS_EINVAL;
  // 16-byte cp.async and vector accesses need 16-byte aligned vectors; other
  // pointers take the generic tensor-core kernel
  if ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(d)) & 15)
    return TPSS_EINVAL;
  const bool v = P->kind == TPSS_VERTEX_PATCH;
  switch (P->n) {
    case 4: return v ? bf::launch<4, true>(P, list, count, omega, nrhs, r, x, d, s, rpc)
                     : bf::launch<4, false>(P, list, count, omega, nrhs, r, x, d, s, rpc);
    case 6: return v ? bf::launch<6, true>(P, list, count, omega, nrhs, r, x, d, s, rpc)
                     : bf::launch<6, false>(P, list, count, omega, nrhs, r, x, d, s, rpc);
    case 8: return v ? bf::launch<8, true>(P, list, count, omega, nrhs, r, x, d, s, rpc)
                     : bf::launch<8, false>(P, list, count, omega, nrhs, r, x, d, s, rpc);
    case 10: return v ? bf::launch<10, true>(P, list, count, omega, nrhs, r, x, d, s, rpc) : TPSS_EINVAL;
    case 12: return v ? bf::launch<12, true>(P, list, count, omega, nrhs, r, x, d, s, rpc) : TPSS_EINVAL;
    case 14: return v ? bf::launch<14, true>(P, list, count, omega, nrhs, r, x, d, s, rpc) : TPSS_EINVAL;
    case 16: return v ? bf::launch<16, true>(P, list, count, omega, nrhs, r, x, d, s, rpc) : TPSS_EINVAL;
    default: return TPSS_EINVAL;
  }
}

}  // namespace tpss
