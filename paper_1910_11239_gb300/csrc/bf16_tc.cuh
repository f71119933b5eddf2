// BF16 tensor-core building blocks of the fast-diagonalization local solve
// (3D patch tensors, MMA m16n8k16 with FP32 accumulation), shared by the
// colored smoother (smoother_bf16.cu) and the batched persistent smoother
// (batch.cu).  See smoother_bf16.cu for the shared-memory layout.
#pragma once

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
        c[nt][e] = (x < N && i < N) ? __fdividef(c[nt][e], lam[x] + ly + lam[2 * N + i]) : 0.f;
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

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage the 2^d cells of one right-hand side (cell-major, NV floats) into
// shared memory with asynchronous copies (16 bytes when cells are 16-byte
// multiples, else 4 bytes).
struct CellBase {
  int px, py, pz, nc0, nc1;
  // first DoF of the patch's cell c (c = sx + 2 sy + 4 sz)
  template <int NLOC1>
  __device__ __forceinline__ int64_t operator()(int c) const {
    return ((px + (c & 1)) + (int64_t)nc0 * ((py + ((c >> 1) & 1)) + (int64_t)nc1 * (pz + ((c >> 2) & 1)))) * NLOC1;
  }
};

template <int NLOC1, int NCELL>
__device__ __forceinline__ void stage(float* dst, const float* __restrict__ src, const CellBase& cb, int tid) {
  const uint32_t d = smem_u32(dst);
  if constexpr (NLOC1 % 4 == 0) {
    constexpr int CH = NLOC1 / 4;
    for (int e = tid; e < NCELL * CH; e += kThreads) {
      const int c = e / CH, o = (e % CH) * 4;
      cp_async16(d + 4u * (c * NLOC1 + o), src + cb.template operator()<NLOC1>(c) + o);
    }
  } else {
    for (int e = tid; e < NCELL * NLOC1; e += kThreads) {
      const int c = e / NLOC1, o = e % NLOC1;
      cp_async4(d + 4u * (c * NLOC1 + o), src + cb.template operator()<NLOC1>(c) + o);
    }
  }
}

// Row-wise copies: a "row" is the N1 values of one cell along x, contiguous
// both in the staged cell-major buffers and in the patch tensor.  V = 4, 2 or
// 1 values per vector access (N1 divisible by 4, by 2, or odd).
template <int N1>
struct RowVec {
  static constexpr int V = (N1 % 4 == 0) ? 4 : ((N1 % 2 == 0) ? 2 : 1);
};

// SB (f32, cell-major) -> T (bf16 patch tensor), one cell row per iteration.
template <int N, int N1, int NCELL>
__device__ __forceinline__ void rows_to_tensor(__nv_bfloat16* __restrict__ T, const float* __restrict__ SB, int tid) {
  using S = Shape<N>;
  constexpr int V = RowVec<N1>::V;
  constexpr int NROW = NCELL * N1 * N1;
  for (int rw = tid; rw < NROW; rw += kThreads) {
    const int c = rw / (N1 * N1), rr = rw % (N1 * N1);
    const int iy = rr % N1, iz = rr / N1;
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const float* src = SB + c * N1 * N1 * N1 + rr * N1;
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

// x[cell rows] += omega T with atomic adds (several CTAs may update the same
// cells), vectorized to 16 / 8 bytes when the rows allow it.
template <int N, int N1, int NCELL>
__device__ __forceinline__ void tensor_atomic_add(float* __restrict__ xr, const __nv_bfloat16* __restrict__ T,
                                                  float omega, const CellBase& cb, int tid) {
  using S = Shape<N>;
  constexpr int V = RowVec<N1>::V;
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int NROW = NCELL * N1 * N1;
  for (int rw = tid; rw < NROW; rw += kThreads) {
    const int c = rw / (N1 * N1), rr = rw % (N1 * N1);
    const int iy = rr % N1, iz = rr / N1;
    const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
    const __nv_bfloat16* t = T + sx * N1 + LS * (sy * N1 + iy) + S::PS * (sz * N1 + iz);
    float* dst = xr + cb.template operator()<NLOC1>(c) + rr * N1;
#pragma unroll
    for (int v = 0; v < N1; v += V) {
      if constexpr (V == 4) {
        const uint2 tb = *reinterpret_cast<const uint2*>(t + v);
        const float2 t01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&tb.x));
        const float2 t23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&tb.y));
        atomicAdd(reinterpret_cast<float4*>(dst + v),
                  make_float4(omega * t01.x, omega * t01.y, omega * t23.x, omega * t23.y));
      } else if constexpr (V == 2) {
        const float2 tt = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(t + v));
        atomicAdd(reinterpret_cast<float2*>(dst + v), make_float2(omega * tt.x, omega * tt.y));
      } else {
        atomicAdd(dst + v, omega * __bfloat162float(t[v]));
      }
    }
  }
}

}  // namespace bf
}  // namespace tpss
