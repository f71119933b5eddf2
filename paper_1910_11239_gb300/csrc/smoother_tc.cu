// Tensor-core variant of the patch smoother (mixed precision; not in the paper).
//
// Each mode contraction of the fast-diagonalization local solve is a small
// GEMM over the lines of the patch tensor:
//     Out (lines x n) = In (lines x n) * W (n x n),
// W = Z for the Z^T application (Out_i = sum_m Z[m][i] In_m) and W = Z^T for
// the Z application.  Lines are the MMA M dimension (one warp owns a tile of
// 16 lines of one patch), the contracted index is K and the output index is
// N, so padding of n to the MMA shape only affects K and N.  The patch tensor
// stays in shared memory in FP32 between contractions; operands are rounded
// to TF32 (m16n8k8) or BF16 (m16n8k16) when the fragments are loaded, and
// accumulation is FP32.  The Lambda^{-1} scale is applied to the accumulator
// fragments of the last Z^T contraction.  Colors, gather and scatter are as in
// the FP64/FP32 kernel (smoother.cu).
#include <cuda_bf16.h>

#include "tpss_internal.cuh"

namespace tpss {

template <int DIM, int N, bool BF16>
struct TcShape {
  static constexpr int LINES = DIM == 3 ? N * N : N;
  static constexpr int TILES = (LINES + 15) / 16;           // 16-line tiles = warps per patch
  static constexpr int KG = BF16 ? 16 : 8;                 // K granularity of one mma
  static constexpr int NP = ((N + KG - 1) / KG) * KG;      // padded n (K and N)
  static constexpr int KC = NP / KG;                       // K chunks
  static constexpr int NT = NP / 8;                        // N tiles of 8
  static constexpr int LS = (N % 2 == 0) ? N + 1 : N;      // odd line stride in shared memory
  static constexpr int PS = LS * N;
  static constexpr int VOL = DIM == 3 ? PS * N : LS * N;
  static constexpr int PPB = TILES >= 8 ? 1 : (8 + TILES - 1) / TILES;
  static constexpr int THREADS = PPB * TILES * 32;
  static constexpr int SLOT = VOL + 2 * DIM * NP * NP + DIM * N;  // tensor, W (Z, Z^T), lambda
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (lower 16 bits)
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int DIM, int N>
__device__ __forceinline__ void tc_line_geom(int t, int line, int& base, int& stride) {
  constexpr int LS = (N % 2 == 0) ? N + 1 : N;
  constexpr int PS = LS * N;
  if (DIM == 3) {
    const int a = line % N, b = line / N;
    if (t == 0) { base = LS * a + PS * b; stride = 1; }
    else if (t == 1) { base = a + PS * b; stride = LS; }
    else { base = a + LS * b; stride = PS; }
  } else {
    if (t == 0) { base = LS * line; stride = 1; }
    else { base = line; stride = LS; }
  }
}

// One contraction along direction t for the warp's 16-line tile, in place.
// W is NP x NP (row = contracted index m, column = output index i), zero
// padded.  SCALE: multiply the result by 1/(lam0[a] + lam1[b] + lamt[i]).
template <int DIM, int N, bool BF16, bool SCALE>
__device__ __forceinline__ void tc_contract(float* __restrict__ buf, const float* __restrict__ W, int t,
                                            int tile, int lane, const float* __restrict__ lams) {
  using S = TcShape<DIM, N, BF16>;
  const int g = lane >> 2, tig = lane & 3;
  const int l0 = tile * 16 + g, l1 = l0 + 8;
  const bool v0 = l0 < S::LINES, v1 = l1 < S::LINES;
  int b0, s0, b1, s1;
  tc_line_geom<DIM, N>(t, v0 ? l0 : 0, b0, s0);
  tc_line_geom<DIM, N>(t, v1 ? l1 : 0, b1, s1);
  auto ld = [&](bool v, int base, int stride, int m) -> float {
    return (v && m < N) ? buf[base + m * stride] : 0.0f;
  };
  uint32_t a[S::KC][4];
#pragma unroll
  for (int kc = 0; kc < S::KC; ++kc) {
    if (BF16) {
      const int m0 = kc * 16 + 2 * tig;
      a[kc][0] = pack_bf16(ld(v0, b0, s0, m0), ld(v0, b0, s0, m0 + 1));
      a[kc][1] = pack_bf16(ld(v1, b1, s1, m0), ld(v1, b1, s1, m0 + 1));
      a[kc][2] = pack_bf16(ld(v0, b0, s0, m0 + 8), ld(v0, b0, s0, m0 + 9));
      a[kc][3] = pack_bf16(ld(v1, b1, s1, m0 + 8), ld(v1, b1, s1, m0 + 9));
    } else {
      const int m0 = kc * 8 + tig;
      a[kc][0] = to_tf32(ld(v0, b0, s0, m0));
      a[kc][1] = to_tf32(ld(v1, b1, s1, m0));
      a[kc][2] = to_tf32(ld(v0, b0, s0, m0 + 4));
      a[kc][3] = to_tf32(ld(v1, b1, s1, m0 + 4));
    }
  }
  __syncwarp();
  const int la0 = DIM == 3 ? l0 % N : l0, lb0 = DIM == 3 ? l0 / N : 0;
  const int la1 = DIM == 3 ? l1 % N : l1, lb1 = DIM == 3 ? l1 / N : 0;
  float sl0 = 0.f, sl1 = 0.f;
  if (SCALE) {
    if (v0) sl0 = lams[la0] + (DIM == 3 ? lams[N + lb0] : 0.f);
    if (v1) sl1 = lams[la1] + (DIM == 3 ? lams[N + lb1] : 0.f);
  }
#pragma unroll
  for (int nt = 0; nt < S::NT; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const int col = nt * 8 + g;  // B fragment column (output index)
#pragma unroll
    for (int kc = 0; kc < S::KC; ++kc) {
      uint32_t bb0, bb1;
      if (BF16) {
        const int r0 = kc * 16 + 2 * tig;
        bb0 = pack_bf16(W[r0 * S::NP + col], W[(r0 + 1) * S::NP + col]);
        bb1 = pack_bf16(W[(r0 + 8) * S::NP + col], W[(r0 + 9) * S::NP + col]);
        mma_bf16(c, a[kc], bb0, bb1);
      } else {
        const int r0 = kc * 8 + tig;
        bb0 = to_tf32(W[r0 * S::NP + col]);
        bb1 = to_tf32(W[(r0 + 4) * S::NP + col]);
        mma_tf32(c, a[kc], bb0, bb1);
      }
    }
    const int i0 = nt * 8 + 2 * tig;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h;
      if (i < N) {
        if (v0) {
          float v = c[h];
          if (SCALE) v = v / (sl0 + lams[(DIM - 1) * N + i]);
          buf[b0 + i * s0] = v;
        }
        if (v1) {
          float v = c[2 + h];
          if (SCALE) v = v / (sl1 + lams[(DIM - 1) * N + i]);
          buf[b1 + i * s1] = v;
        }
      }
    }
  }
}

template <int DIM, int N, bool VERTEX, bool BF16>
__global__ void __launch_bounds__(TcShape<DIM, N, BF16>::THREADS)
patch_smooth_tc_kernel(const int* __restrict__ list, int count, const float* __restrict__ r, float* __restrict__ x,
                       float* __restrict__ d, float omega, int nc0, int nc1, int64_t ndofs, const float* Z0,
                       const float* Z1, const float* Z2, const float* L0, const float* L1, const float* L2) {
  using S = TcShape<DIM, N, BF16>;
  constexpr int N1 = VERTEX ? N / 2 : N;
  constexpr int NLOC1 = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
  constexpr int NCELL = VERTEX ? (1 << DIM) : 1;
  constexpr int TPP = S::TILES * 32;  // threads per patch
  extern __shared__ float smf[];
  const int slot = threadIdx.x / TPP;
  const int lt = threadIdx.x % TPP;
  const int warp = lt / 32, lane = lt % 32;
  const int q = blockIdx.x * S::PPB + slot;
  const bool active = q < count;
  float* buf = smf + slot * S::SLOT;
  float* W = buf + S::VOL;                 // [DIM][2][NP*NP]: Z then Z^T per direction
  float* lams = W + 2 * DIM * S::NP * S::NP;
  const int64_t vbase = (int64_t)blockIdx.y * ndofs;
  const float* Zd[3] = {Z0, Z1, Z2};
  const float* Ld[3] = {L0, L1, L2};
  int pos[3] = {0, 0, 0};
  if (active) {
    const int packed = list[q];
    pos[0] = unpack_x(packed);
    pos[1] = unpack_y(packed);
    pos[2] = unpack_z(packed);
    for (int e = lt; e < DIM * S::NP * S::NP; e += TPP) {
      const int t = e / (S::NP * S::NP), rem = e % (S::NP * S::NP);
      const int m = rem / S::NP, i = rem % S::NP;
      float z = 0.f, zt = 0.f;
      if (m < N && i < N) {
        const float* Zt = Zd[t] + (size_t)pos[t] * N * N;
        z = Zt[m * N + i];
        zt = Zt[i * N + m];
      }
      W[(2 * t) * S::NP * S::NP + rem] = z;
      W[(2 * t + 1) * S::NP * S::NP + rem] = zt;
    }
    for (int e = lt; e < DIM * N; e += TPP) lams[e] = Ld[e / N][(size_t)pos[e / N] * N + e % N];
    for (int e = lt; e < NCELL * NLOC1; e += TPP) {
      const int c = e / NLOC1, loc = e % NLOC1;
      const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
      const int ix = loc % N1, iy = (loc / N1) % N1, iz = DIM == 3 ? loc / (N1 * N1) : 0;
      const int64_t gcell = (pos[0] + sx) + (int64_t)nc0 * ((pos[1] + sy) + (int64_t)nc1 * (DIM == 3 ? pos[2] + sz : 0));
      const int pidx = (sx * N1 + ix) + S::LS * (sy * N1 + iy) + (DIM == 3 ? S::PS * (sz * N1 + iz) : 0);
      buf[pidx] = r[vbase + gcell * NLOC1 + loc];
    }
  }
  __syncthreads();
  // Z^T along every direction; the last one also applies Lambda^{-1}
  for (int t = 0; t < DIM; ++t) {
    if (active) {
      const float* Wt = W + (2 * t) * S::NP * S::NP;
      if (t == DIM - 1) tc_contract<DIM, N, BF16, true>(buf, Wt, t, warp, lane, lams);
      else tc_contract<DIM, N, BF16, false>(buf, Wt, t, warp, lane, lams);
    }
    __syncthreads();
  }
  for (int t = DIM - 1; t >= 0; --t) {
    if (active) tc_contract<DIM, N, BF16, false>(buf, W + (2 * t + 1) * S::NP * S::NP, t, warp, lane, lams);
    __syncthreads();
  }
  if (active) {
    for (int e = lt; e < NCELL * NLOC1; e += TPP) {
      const int c = e / NLOC1, loc = e % NLOC1;
      const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
      const int ix = loc % N1, iy = (loc / N1) % N1, iz = DIM == 3 ? loc / (N1 * N1) : 0;
      const int64_t gcell = (pos[0] + sx) + (int64_t)nc0 * ((pos[1] + sy) + (int64_t)nc1 * (DIM == 3 ? pos[2] + sz : 0));
      const int pidx = (sx * N1 + ix) + S::LS * (sy * N1 + iy) + (DIM == 3 ? S::PS * (sz * N1 + iz) : 0);
      const int64_t gi = vbase + gcell * NLOC1 + loc;
      x[gi] = fmaf(omega, buf[pidx], x[gi]);
      if (d != nullptr) {   // the update and the color's residual, for the multiplicative residual update
        d[gi] = omega * buf[pidx];
        const_cast<float*>(r)[gi] *= 1.f - omega;
      }
    }
  }
}

template <int DIM, int N, bool VERTEX, bool BF16>
static tpss_status launch_tc(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                             float* x, float* d, cudaStream_t s) {
  using S = TcShape<DIM, N, BF16>;
  const size_t smem = (size_t)S::PPB * S::SLOT * sizeof(float);
  if (smem > 48 * 1024)
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(patch_smooth_tc_kernel<DIM, N, VERTEX, BF16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (count <= 0) return TPSS_OK;
  const Level& L = P->ctx->levels[P->level];
  dim3 grid((count + S::PPB - 1) / S::PPB, nrhs);
  patch_smooth_tc_kernel<DIM, N, VERTEX, BF16><<<grid, S::THREADS, smem, s>>>(
      list, count, r, x, d, omega, L.nc[0], L.nc[1], L.ndofs, P->d_Z32[0], P->d_Z32[1],
      DIM == 3 ? P->d_Z32[2] : P->d_Z32[0], P->d_lam32[0], P->d_lam32[1],
      DIM == 3 ? P->d_lam32[2] : P->d_lam32[0]);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

tpss_status patch_pass_tc(tpss_patches* P, const int* list, int count, float omega, int nrhs, const float* r,
                          float* x, cudaStream_t s, float* d) {
  const int dim = P->ctx->dim, n = P->n;
  const bool v = P->kind == TPSS_VERTEX_PATCH;
  const bool bf = P->precision == TPSS_BF16;
#define TPSS_TC_CASE(D, NN, V)                                                                  \
  if (dim == D && n == NN && v == V)                                                           \
    return bf ? launch_tc<D, NN, V, true>(P, list, count, omega, nrhs, r, x, d, s)             \
              : launch_tc<D, NN, V, false>(P, list, count, omega, nrhs, r, x, d, s);
  TPSS_TC_CASE(3, 4, true) TPSS_TC_CASE(3, 6, true) TPSS_TC_CASE(3, 8, true) TPSS_TC_CASE(3, 10, true)
  TPSS_TC_CASE(3, 12, true) TPSS_TC_CASE(3, 14, true) TPSS_TC_CASE(3, 16, true)
  TPSS_TC_CASE(3, 2, false) TPSS_TC_CASE(3, 3, false) TPSS_TC_CASE(3, 4, false) TPSS_TC_CASE(3, 5, false)
  TPSS_TC_CASE(3, 6, false) TPSS_TC_CASE(3, 7, false) TPSS_TC_CASE(3, 8, false)
  TPSS_TC_CASE(2, 4, true) TPSS_TC_CASE(2, 6, true) TPSS_TC_CASE(2, 8, true) TPSS_TC_CASE(2, 10, true)
  TPSS_TC_CASE(2, 12, true) TPSS_TC_CASE(2, 14, true) TPSS_TC_CASE(2, 16, true)
  TPSS_TC_CASE(2, 2, false) TPSS_TC_CASE(2, 3, false) TPSS_TC_CASE(2, 4, false) TPSS_TC_CASE(2, 5, false)
  TPSS_TC_CASE(2, 6, false) TPSS_TC_CASE(2, 7, false) TPSS_TC_CASE(2, 8, false)
#undef TPSS_TC_CASE
  set_error("tensor-core smoother: unsupported subdomain size");
  return TPSS_EINVAL;
}

}  // namespace tpss
