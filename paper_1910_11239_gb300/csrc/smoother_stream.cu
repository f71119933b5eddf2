// Column-streaming BF16 additive vertex-patch smoother, 3D (mixed precision;
// not in the paper).
//
// The additive smoother of Alg. 2 sums, over all vertex patches j,
// omega R_j^T A_j^{-1} R_j r.  A vertex patch at position (p_x, p_y, p_z)
// covers the 2 x 2 x 2 cells p_t .. p_t + 1.  Here one CTA owns one column of
// patches (p_x, p_y fixed) for one right-hand side and walks p_z upwards:
//
//  * the cells of r are staged plane by plane (4 cells per cell plane) into a
//    ring of three FP32 plane buffers with cp.async, one plane ahead of the
//    patch being solved, so every cell of r is read from memory once per
//    column instead of once per patch;
//  * the local solve is the BF16 tensor-core sequence of bf16_tc.cuh (Z^T
//    along x and y, the fused Z^T -> Lambda^{-1} -> Z step along z, Z along y),
//    and the last contraction (Z along x) adds its FP32 accumulators, times
//    omega, straight into two FP32 plane accumulators in shared memory;
//  * a cell plane is complete once the two patches of the column that cover
//    it are done, and is then written to x once.
//
// Columns with the same parity (p_x mod 2, p_y mod 2) share no cell, so the
// four parity classes are four launches with no write conflict and no
// atomics; the result is deterministic.  A cell's first class (in launch
// order) stores its value (x_is_zero) and later classes add to it, so x needs
// no clearing.  Memory traffic per DoF and right-hand side: r read once per
// class (4 x 4 bytes) and x written once, read and written three times
// (4 + 3 x 8 bytes), against 8 bytes algorithmic; the colored one-patch-per-CTA
// schedule moves about 96.
#include "bf16_tc.cuh"

namespace tpss {
namespace bf {

// First parity class (in launch order 0..3, class = (p_x & 1) + 2 (p_y & 1))
// whose columns cover the cell column (cx, cy): interior cells are covered by
// both parities along a direction, the last cell only by p = n - 2.
__device__ __forceinline__ int first_class(int cx, int cy, int nc0, int nc1) {
  const int xm = (cx == nc0 - 1) ? (nc0 & 1) : 0;
  const int ym = (cy == nc1 - 1) ? (nc1 & 1) : 0;
  return xm + 2 * ym;
}

// Stage the 4 cells (p_x + sx, p_y + sy, cz), sx, sy in {0, 1}, of one
// right-hand side into dst (cell-major, cell c2 = sx + 2 sy).
template <int NLOC1>
__device__ __forceinline__ void stage_plane(float* dst, const float* __restrict__ src, int px, int py, int cz,
                                            int nc0, int nc1, int tid) {
  const uint32_t d = smem_u32(dst);
  auto cell0 = [&](int c2) -> int64_t {
    return ((px + (c2 & 1)) + (int64_t)nc0 * ((py + (c2 >> 1)) + (int64_t)nc1 * cz)) * NLOC1;
  };
  if constexpr (NLOC1 % 4 == 0) {
    constexpr int CH = NLOC1 / 4;
    for (int e = tid; e < 4 * CH; e += kThreads) {
      const int c2 = e / CH, o = (e % CH) * 4;
      cp_async16(d + 4u * (c2 * NLOC1 + o), src + cell0(c2) + o);
    }
  } else {
    for (int e = tid; e < 4 * NLOC1; e += kThreads) {
      const int c2 = e / NLOC1, o = e % NLOC1;
      cp_async4(d + 4u * (c2 * NLOC1 + o), src + cell0(c2) + o);
    }
  }
}

// Two staged planes (lo: cells with sz = 0, hi: sz = 1) -> the BF16 patch
// tensor, one cell row (N1 values along x) per iteration.
template <int N, int N1>
__device__ __forceinline__ void planes_to_tensor(__nv_bfloat16* __restrict__ T, const float* __restrict__ lo,
                                                 const float* __restrict__ hi, int tid) {
  using S = Shape<N>;
  constexpr int V = RowVec<N1>::V;
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int NROW = 8 * N1 * N1;
  for (int rw = tid; rw < NROW; rw += kThreads) {
    const int c = rw / (N1 * N1), rr = rw % (N1 * N1);
    const int iy = rr % N1, iz = rr / N1;
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const float* src = (sz ? hi : lo) + (c & 3) * NLOC1 + rr * N1;
    __nv_bfloat16* dst = T + sx * N1 + LS * (sy * N1 + iy) + S::PS * (sz * N1 + iz);
#pragma unroll
    for (int v = 0; v < N1; v += V) {
      if constexpr (V == 4) {
        const float4 f = *reinterpret_cast<const float4*>(src + v);
        uint2 o;
        o.x = pack2(f.x, f.y);
        o.y = pack2(f.z, f.w);
        *reinterpret_cast<uint2*>(dst + v) = o;
      } else if constexpr (V == 2) {
        const float2 f = *reinterpret_cast<const float2*>(src + v);
        *reinterpret_cast<uint32_t*>(dst + v) = pack2(f.x, f.y);
      } else {
        dst[v] = __float2bfloat16(src[v]);
      }
    }
  }
}

// The last contraction (Z along x) with its FP32 accumulators added, times
// omega, into the plane accumulators: acc_lo for the cells with sz = 0,
// acc_hi for sz = 1 (cell-major like the staged planes).  Every (line, x) of
// the patch belongs to one lane of one warp, so the adds do not race.
template <int N>
__device__ __forceinline__ void contract_x_acc(const __nv_bfloat16* T, const uint32_t (&b)[2][2], float* acc_lo,
                                               float* acc_hi, float omega, int warp, int lane) {
  using S = Shape<N>;
  constexpr int N1 = N / 2;
  constexpr int NLOC1 = N1 * N1 * N1;
  const uint32_t base = smem_u32(T);
  const int j = lane >> 3, q = lane & 7;
  const int g = lane >> 2, t = lane & 3;
  constexpr int TILES = (N * N + 15) / 16;
  for (int tile = warp; tile < TILES; tile += kWarps) {
    uint32_t a[4];
    {
      const int line = tile * 16 + (j & 1) * 8 + q;
      const int off = line < N * N ? (LS * (line % N) + S::PS * (line / N) + 8 * (j >> 1)) : S::ZROW;
      ldsm_x4(a, base + 2u * off);
    }
    float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    mma16816(c[0], a, b[0][0], b[0][1]);
    mma16816(c[1], a, b[1][0], b[1][1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {            // accumulator rows g (h = 0) and g + 8 (h = 1)
      const int line = tile * 16 + g + 8 * h;
      if (line >= N * N) continue;
      const int y = line % N, z = line / N;
      const int sy = y / N1, iy = y % N1, sz = z / N1, iz = z % N1;
      float* acc = (sz ? acc_hi : acc_lo) + 2 * sy * NLOC1 + N1 * (iy + N1 * iz);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int xi = 8 * nt + 2 * t;       // this lane's two columns xi, xi + 1
        if constexpr (N1 % 2 == 0) {
          if (xi < N) {                      // xi even and N1 even: both in one cell
            const int sx = xi / N1, ix = xi % N1;
            float2* p = reinterpret_cast<float2*>(acc + sx * NLOC1 + ix);
            float2 v = *p;
            v.x = fmaf(omega, c[nt][2 * h], v.x);
            v.y = fmaf(omega, c[nt][2 * h + 1], v.y);
            *p = v;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int xx = xi + e;
            if (xx < N) {
              const int sx = xx / N1, ix = xx % N1;
              acc[sx * NLOC1 + ix] = fmaf(omega, c[nt][2 * h + e], acc[sx * NLOC1 + ix]);
            }
          }
        }
      }
    }
  }
}

// Write one finished cell plane of the column (4 cells) to x and clear its
// accumulator: a plain store where this parity class is the cell's first
// and x starts at zero, else x += acc.
template <int N1>
__device__ __forceinline__ void flush_plane(float* __restrict__ x, float* acc, int px, int py, int cz, int nc0,
                                            int nc1, int cls, int x_is_zero, int tid) {
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int V = (NLOC1 % 4 == 0) ? 4 : 1;
  constexpr int CH = NLOC1 / V;
  for (int e = tid; e < 4 * CH; e += kThreads) {
    const int c2 = e / CH, o = (e % CH) * V;
    const int cx = px + (c2 & 1), cy = py + (c2 >> 1);
    const bool store = x_is_zero && first_class(cx, cy, nc0, nc1) == cls;
    float* dst = x + (cx + (int64_t)nc0 * (cy + (int64_t)nc1 * cz)) * NLOC1 + o;
    float* a = acc + c2 * NLOC1 + o;
    if constexpr (V == 4) {
      float4 v = *reinterpret_cast<float4*>(a);
      if (!store) {
        const float4 old = *reinterpret_cast<const float4*>(dst);
        v.x += old.x;
        v.y += old.y;
        v.z += old.z;
        v.w += old.w;
      }
      *reinterpret_cast<float4*>(dst) = v;
      *reinterpret_cast<float4*>(a) = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      const float v = *a;
      *dst = store ? v : v + *dst;
      *a = 0.f;
    }
  }
}

template <int N>
struct StreamSmem {
  static constexpr int N1 = N / 2;
  static constexpr int NP = 4 * N1 * N1 * N1;                          // floats of one column plane
  static constexpr size_t T_BYTES = ((Shape<N>::TOTAL * 2 + 15) / 16) * 16;
  static constexpr size_t SB_OFF = T_BYTES;                             // 3 staged planes of r
  static constexpr size_t ACC_OFF = SB_OFF + 3 * (size_t)NP * 4;        // 2 plane accumulators
  static constexpr size_t BYTES = ACC_OFF + 2 * (size_t)NP * 4;
};

template <int N>
__global__ void __launch_bounds__(kThreads, 3)
patch_stream_bf16_kernel(const float* __restrict__ Z0, const float* __restrict__ Z1, const float* __restrict__ Z2,
                         const float* __restrict__ L0, const float* __restrict__ L1, const float* __restrict__ L2,
                         const float* __restrict__ r, float* __restrict__ x, float omega, int nc0, int nc1, int nc2,
                         int64_t ndofs, int cls, int ncolx, int x_is_zero) {
  using S = Shape<N>;
  using M = StreamSmem<N>;
  constexpr int N1 = N / 2;
  constexpr int NP = M::NP;
  extern __shared__ __align__(16) unsigned char dsm[];
  __nv_bfloat16* T = reinterpret_cast<__nv_bfloat16*>(dsm);
  float* SB = reinterpret_cast<float*>(dsm + M::SB_OFF);
  float* ACC = reinterpret_cast<float*>(dsm + M::ACC_OFF);
  __shared__ float lam[3 * N];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int px = (cls & 1) + 2 * (int)(blockIdx.x % ncolx);
  const int py = (cls >> 1) + 2 * (int)(blockIdx.x / ncolx);
  r += (int64_t)blockIdx.y * ndofs;
  x += (int64_t)blockIdx.y * ndofs;

  stage_plane<N1 * N1 * N1>(SB, r, px, py, 0, nc0, nc1, tid);
  stage_plane<N1 * N1 * N1>(SB + NP, r, px, py, 1, nc0, nc1, tid);
  cp_async_commit();
  for (int e = tid; e < S::TOTAL; e += kThreads) T[e] = __float2bfloat16(0.f);
  for (int e = tid; e < 2 * NP; e += kThreads) ACC[e] = 0.f;
  if (tid < 2 * N) lam[tid] = tid < N ? L0[(size_t)px * N + tid] : L1[(size_t)py * N + tid - N];
  uint32_t bx[2][2], bxt[2][2], by[2][2], byt[2][2];
  load_bfrag<N, false>(bxt, Z0 + (size_t)px * N * N, lane);
  load_bfrag<N, true>(bx, Z0 + (size_t)px * N * N, lane);
  load_bfrag<N, false>(byt, Z1 + (size_t)py * N * N, lane);
  load_bfrag<N, true>(by, Z1 + (size_t)py * N * N, lane);

  for (int pz = 0; pz + 1 < nc2; ++pz) {
    cp_async_wait_all();
    __syncthreads();   // planes pz, pz + 1 staged; the previous patch is done with T, lam and slot (pz + 2) % 3
    if (pz + 2 < nc2) {
      stage_plane<N1 * N1 * N1>(SB + ((pz + 2) % 3) * NP, r, px, py, pz + 2, nc0, nc1, tid);
      cp_async_commit();
    }
    if (tid < N) lam[2 * N + tid] = L2[(size_t)pz * N + tid];
    uint32_t bzz[2][2], bzt[2][2];
    load_bfrag<N, false>(bzt, Z2 + (size_t)pz * N * N, lane);
    load_bfrag<N, true>(bzz, Z2 + (size_t)pz * N * N, lane);
    planes_to_tensor<N, N1>(T, SB + (pz % 3) * NP, SB + ((pz + 1) % 3) * NP, tid);
    __syncthreads();
    contract<N, 0>(T, bxt, warp, lane);
    __syncthreads();
    contract<N, 1>(T, byt, warp, lane);
    __syncthreads();
    zstep<N>(T, bzt, bzz, lam, warp, lane);
    __syncthreads();
    contract<N, 1>(T, by, warp, lane);
    __syncthreads();
    contract_x_acc<N>(T, bx, ACC + (pz & 1) * NP, ACC + ((pz + 1) & 1) * NP, omega, warp, lane);
    __syncthreads();   // plane pz now has both of its patches of this column
    flush_plane<N1>(x, ACC + (pz & 1) * NP, px, py, pz, nc0, nc1, cls, x_is_zero, tid);
  }
  __syncthreads();
  flush_plane<N1>(x, ACC + ((nc2 - 1) & 1) * NP, px, py, nc2 - 1, nc0, nc1, cls, x_is_zero, tid);
}

template <int N>
static tpss_status launch_stream(tpss_patches* P, float omega, int nrhs, const float* r, float* x, int x_is_zero,
                                 cudaStream_t s) {
  constexpr size_t smem = StreamSmem<N>::BYTES;
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(patch_stream_bf16_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr = true;
  }
  const Level& L = P->ctx->levels[P->level];
  const int nc0 = L.nc[0], nc1 = L.nc[1], nc2 = L.nc[2];
  for (int cls = 0; cls < 4; ++cls) {
    // columns p_x = (cls & 1) + 2 i <= nc0 - 2, p_y = (cls >> 1) + 2 j <= nc1 - 2
    const int ax = cls & 1, ay = cls >> 1;
    const int ncolx = ax <= nc0 - 2 ? (nc0 - 2 - ax) / 2 + 1 : 0;
    const int ncoly = ay <= nc1 - 2 ? (nc1 - 2 - ay) / 2 + 1 : 0;
    if (ncolx == 0 || ncoly == 0) continue;
    dim3 grid((unsigned)(ncolx * ncoly), (unsigned)nrhs);
    patch_stream_bf16_kernel<N><<<grid, kThreads, smem, s>>>(
        P->d_Z32[0], P->d_Z32[1], P->d_Z32[2], P->d_lam32[0], P->d_lam32[1], P->d_lam32[2], r, x, omega, nc0, nc1,
        nc2, L.ndofs, cls, ncolx, x_is_zero);
    TPSS_CHECK_LAUNCH();
  }
  return TPSS_OK;
}

}  // namespace bf

// The additive pass of the column-streaming schedule (all four parity
// classes); TPSS_EINVAL without launching for shapes it does not cover (not
// 3D vertex patches, n > 16, fewer than 2 cells along a direction, vectors
// not 16-byte aligned).  x_is_zero: x is written, not read (no clearing
// needed); else x += the smoother's correction of r.
tpss_status patch_pass_bf16_stream(tpss_patches* P, float omega, int nrhs, const float* r, float* x, int x_is_zero,
                                   cudaStream_t s) {
  if (P->ctx->dim != 3 || P->kind != TPSS_VERTEX_PATCH || P->per_sub) return TPSS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(x)) & 15) return TPSS_EINVAL;
  const Level& L = P->ctx->levels[P->level];
  if (L.nc[0] < 2 || L.nc[1] < 2 || L.nc[2] < 2 || nrhs > 65535) return TPSS_EINVAL;
  switch (P->n) {
    case 4: return bf::launch_stream<4>(P, omega, nrhs, r, x, x_is_zero, s);
    case 6: return bf::launch_stream<6>(P, omega, nrhs, r, x, x_is_zero, s);
    case 8: return bf::launch_stream<8>(P, omega, nrhs, r, x, x_is_zero, s);
    case 10: return bf::launch_stream<10>(P, omega, nrhs, r, x, x_is_zero, s);
    case 12: return bf::launch_stream<12>(P, omega, nrhs, r, x, x_is_zero, s);
    case 14: return bf::launch_stream<14>(P, omega, nrhs, r, x, x_is_zero, s);
    case 16: return bf::launch_stream<16>(P, omega, nrhs, r, x, x_is_zero, s);
    default: return TPSS_EINVAL;
  }
}

}  // namespace tpss
