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
// gather of the next right-hand side is issued into registers before the
// contractions of the current one.
#include <cuda_bf16.h>

#include "tpss_internal.cuh"

namespace tpss {

namespace bf {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int LS = 24;

template <int N>
struct Shape {
  static constexpr int PS = LS * N + 8;          // (LS N)/8 = 3N is even for even N: +8 makes it odd
  static constexpr int VOL = PS * N;             // bf16 elements of the tensor
  static constexpr int ZROW = VOL;               // 8 zero elements (16 B)
  static constexpr int DROW = VOL + 8;           // 8 dummy elements (discarded stores)
  static constexpr int TOTAL = VOL + 16;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void stsm_x4(uint32_t addr, const uint32_t (&r)[4]) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};"
               :: "r"(addr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]) : "memory");
}
__device__ __forceinline__ void stsm_x4_t(uint32_t addr, const uint32_t (&r)[4]) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1,%2,%3,%4};"
               :: "r"(addr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]) : "memory");
}
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// B fragments of W (k x i, 16 x 16, zero padded) for the two 8-column tiles:
// b[nt][0] = (W[2t][8nt+g], W[2t+1][8nt+g]), b[nt][1] = (W[2t+8][..], W[2t+9][..]).
// TRANSPOSE = false: W[k][i] = Z[k][i] (applies Z^T); true: W[k][i] = Z[i][k] (applies Z).
template <int N, bool TRANSPOSE>
__device__ __forceinline__ void load_bfrag(uint32_t (&b)[2][2], const float* __restrict__ Z, int lane) {
  const int g = lane >> 2, t = lane & 3;
  auto w = [&](int k, int i) -> float {
    if (k >= N || i >= N) return 0.f;
    return TRANSPOSE ? __ldg(Z + i * N + k) : __ldg(Z + k * N + i);
  };
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    const int i = 8 * nt + g;
    b[nt][0] = pack2(w(2 * t, i), w(2 * t + 1, i));
    b[nt][1] = pack2(w(2 * t + 8, i), w(2 * t + 9, i));
  }
}

// One contraction along DIR for all tiles of the subdomain (warps stride over tiles).
template <int N, int DIR>
__device__ __forceinline__ void contract(__nv_bfloat16* T, const uint32_t (&b)[2][2], int warp, int lane) {
  using S = Shape<N>;
  const uint32_t base = smem_u32(T);
  const int j = lane >> 3, q = lane & 7;          // ldmatrix / stmatrix: matrix j, row q
  constexpr int TILES = DIR == 0 ? (N * N + 15) / 16 : N;
  for (int tile = warp; tile < TILES; tile += kWarps) {
    uint32_t a[4];
    if (DIR == 0) {
      const int line = tile * 16 + (j & 1) * 8 + q;
      const int off = line < N * N ? (LS * (line % N) + S::PS * (line / N) + 8 * (j >> 1)) : S::ZROW;
      ldsm_x4(a, base + 2u * off);
    } else {
      const int k = 8 * (j >> 1) + q;               // contraction index (memory row)
      const int x0 = 8 * (j & 1);
      int off;
      if (k >= N) off = S::ZROW;
      else off = DIR == 1 ? (x0 + LS * k + S::PS * tile) : (x0 + LS * tile + S::PS * k);
      ldsm_x4_t(a, base + 2u * off);
    }
    float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    mma16816(c[0], a, b[0][0], b[0][1]);
    mma16816(c[1], a, b[1][0], b[1][1]);
    uint32_t r[4];
    // matrix jj = (row half jj&1, column half jj>>1) of the 16 x 16 result
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) r[jj] = pack2(c[jj >> 1][(jj & 1) * 2], c[jj >> 1][(jj & 1) * 2 + 1]);
    if (DIR == 0) {
      const int line = tile * 16 + (j & 1) * 8 + q;
      const int off = line < N * N ? (LS * (line % N) + S::PS * (line / N) + 8 * (j >> 1)) : S::DROW;
      stsm_x4(base + 2u * off, r);
    } else {
      const int i = 8 * (j >> 1) + q;                // output index (memory row)
      const int x0 = 8 * (j & 1);
      int off;
      if (i >= N) off = S::DROW;
      else off = DIR == 1 ? (x0 + LS * i + S::PS * tile) : (x0 + LS * tile + S::PS * i);
      stsm_x4_t(base + 2u * off, r);
    }
  }
}

// z-step: Z^T along z, scale by 1/(lx + ly + lz), Z along z, chained in registers.
template <int N>
__device__ __forceinline__ void zstep(__nv_bfloat16* T, const uint32_t (&bt)[2][2], const uint32_t (&bz)[2][2],
                                      const float* __restrict__ lam, int warp, int lane) {
  using S = Shape<N>;
  const uint32_t base = smem_u32(T);
  const int j = lane >> 3, q = lane & 7;
  const int g = lane >> 2, t = lane & 3;
  for (int tile = warp; tile < N; tile += kWarps) {   // tile = y
    uint32_t a[4];
    {
      const int k = 8 * (j >> 1) + q, x0 = 8 * (j & 1);
      const int off = k >= N ? S::ZROW : (x0 + LS * tile + S::PS * k);
      ldsm_x4_t(a, base + 2u * off);
    }
    float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    mma16816(c[0], a, bt[0][0], bt[0][1]);
    mma16816(c[1], a, bt[1][0], bt[1][1]);
    // rows x = g, g+8; columns i = 8 nt + 2t, +1
    const float ly = lam[N + tile];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = g + (e >> 1) * 8, i = 8 * nt + 2 * t + (e & 1);
        c[nt][e] = (x < N && i < N) ? c[nt][e] / (lam[x] + ly + lam[2 * N + i]) : 0.f;
      }
    // accumulator layout of m16n8k16 == A-fragment layout for K = 16
    uint32_t a2[4] = {pack2(c[0][0], c[0][1]), pack2(c[0][2], c[0][3]), pack2(c[1][0], c[1][1]),
                      pack2(c[1][2], c[1][3])};
    float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    mma16816(d[0], a2, bz[0][0], bz[0][1]);
    mma16816(d[1], a2, bz[1][0], bz[1][1]);
    uint32_t r[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) r[jj] = pack2(d[jj >> 1][(jj & 1) * 2], d[jj >> 1][(jj & 1) * 2 + 1]);
    const int i = 8 * (j >> 1) + q, x0 = 8 * (j & 1);
    const int off = i >= N ? S::DROW : (x0 + LS * tile + S::PS * i);
    stsm_x4_t(base + 2u * off, r);
  }
}

template <int N, bool VERTEX>
__global__ void __launch_bounds__(kThreads)
patch_smooth_bf16_kernel(const int* __restrict__ list, const float* __restrict__ Z0, const float* __restrict__ Z1,
                         const float* __restrict__ Z2, const float* __restrict__ L0, const float* __restrict__ L1,
                         const float* __restrict__ L2, const float* __restrict__ r, float* __restrict__ x, float omega,
                         int nc0, int nc1, int64_t ndofs, int nrhs) {
  using S = Shape<N>;
  constexpr int N1 = VERTEX ? N / 2 : N;
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int NCELL = VERTEX ? 8 : 1;
  constexpr int NV = NCELL * NLOC1;                       // values gathered per rhs
  constexpr int PER = (NV + kThreads - 1) / kThreads;     // per thread
  __shared__ __align__(16) __nv_bfloat16 T[S::TOTAL];
  __shared__ float lam[3 * N];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int packed = list[blockIdx.x];
  const int px = unpack_x(packed), py = unpack_y(packed), pz = unpack_z(packed);
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
  // element e of the gather: global offset (relative to the rhs base) and tensor offset
  auto goff = [&](int e) -> int64_t {
    const int c = e / NLOC1, loc = e % NLOC1;
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const int64_t gcell = (px + sx) + (int64_t)nc0 * ((py + sy) + (int64_t)nc1 * (pz + sz));
    return gcell * NLOC1 + loc;
  };
  auto toff = [&](int e) -> int {
    const int c = e / NLOC1, loc = e % NLOC1;
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const int ix = loc % N1, iy = (loc / N1) % N1, iz = loc / (N1 * N1);
    return (sx * N1 + ix) + LS * (sy * N1 + iy) + S::PS * (sz * N1 + iz);
  };
  float pre[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = tid + u * kThreads;
    pre[u] = e < NV ? __ldg(r + goff(e)) : 0.f;
  }
  for (int rhs = 0; rhs < nrhs; ++rhs) {
    __syncthreads();   // previous scatter finished reading T; zero fill done
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * kThreads;
      if (e < NV) T[toff(e)] = __float2bfloat16(pre[u]);
    }
    __syncthreads();
    if (rhs + 1 < nrhs) {
      const float* rn = r + (int64_t)(rhs + 1) * ndofs;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + u * kThreads;
        pre[u] = e < NV ? __ldg(rn + goff(e)) : 0.f;
      }
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
    float* xr = x + (int64_t)rhs * ndofs;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * kThreads;
      if (e < NV) {
        float* p = xr + goff(e);
        *p = fmaf(omega, __bfloat162float(T[toff(e)]), *p);
      }
    }
  }
}

template <int N, bool VERTEX>
static tpss_status launch(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                          float* x, cudaStream_t s) {
  if (count <= 0) return TPSS_OK;
  const Level& L = P->ctx->levels[P->level];
  patch_smooth_bf16_kernel<N, VERTEX><<<count, kThreads, 0, s>>>(
      list, P->d_Z32[0], P->d_Z32[1], P->d_Z32[2], P->d_lam32[0], P->d_lam32[1], P->d_lam32[2], r, x, omega,
      L.nc[0], L.nc[1], L.ndofs, nrhs);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

}  // namespace bf

// 3D BF16 path; returns TPSS_EINVAL (without launching) for shapes it does not cover.
tpss_status patch_pass_bf16(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                            float* x, cudaStream_t s) {
  if (P->ctx->dim != 3) return TPSS_EINVAL;
  const bool v = P->kind == TPSS_VERTEX_PATCH;
  switch (P->n) {
    case 4: return v ? bf::launch<4, true>(P, list, count, omega, nrhs, r, x, s)
                     : bf::launch<4, false>(P, list, count, omega, nrhs, r, x, s);
    case 6: return v ? bf::launch<6, true>(P, list, count, omega, nrhs, r, x, s)
                     : bf::launch<6, false>(P, list, count, omega, nrhs, r, x, s);
    case 8: return v ? bf::launch<8, true>(P, list, count, omega, nrhs, r, x, s)
                     : bf::launch<8, false>(P, list, count, omega, nrhs, r, x, s);
    case 10: return v ? bf::launch<10, true>(P, list, count, omega, nrhs, r, x, s) : TPSS_EINVAL;
    case 12: return v ? bf::launch<12, true>(P, list, count, omega, nrhs, r, x, s) : TPSS_EINVAL;
    case 14: return v ? bf::launch<14, true>(P, list, count, omega, nrhs, r, x, s) : TPSS_EINVAL;
    case 16: return v ? bf::launch<16, true>(P, list, count, omega, nrhs, r, x, s) : TPSS_EINVAL;
    default: return TPSS_EINVAL;
  }
}

}  // namespace tpss
