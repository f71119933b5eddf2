// Column-streaming BF16 additive vertex-patch smoother on the 5th-generation
// tensor cores (tcgen05 MMA, accumulators in tensor memory); 3D, mixed
// precision (not in the paper).
//
// Schedule: as the COLUMNS schedule (smoother_stream.cu): one CTA per column
// of vertex patches (p_x, p_y) and right-hand side walks p_z, r staged one
// cell plane at a time with cp.async, x accumulated per cell plane in FP32
// shared memory and written once per parity class of (p_x, p_y).
//
// Local solve (eq. fastinverse, eq. eigenvectormatvec): the six mode
// contractions of (Z_z x Z_y x Z_x) Lambda^{-1} (Z_z x Z_y x Z_x)^T are six
// MMAs D = A B with M = 128 (one or two blocks of 128 rows), N = 16, K = 16,
// BF16 operands from shared memory, FP32 accumulation in TMEM.  Every index
// is padded to 16, so the patch tensor has 256 "lines" (slow index s, fast
// index f, row m = 16 s + f).  A is the tensor with the contracted index as
// K; B holds the 1D eigenvector matrix (K-major, 16 x 16, zero padded).
// After each MMA every thread reads its TMEM rows (row m = thread + 128 b)
// and writes them back to shared memory as the next A, rotating the indices
// so that the next contracted index becomes K:
//
//   A0[(z,y)][x]  --Zx^T--> D1[(z,y)][a] -> A1[(z,a)][y]   (MN-major write)
//   A1            --Zy^T--> D2[(z,a)][b] -> A2[(a,b)][z]   (MN-major)
//   A2            --Zz^T--> D3[(a,b)][c] -> scaled by 1/(lx_a + ly_b + lz_c) -> A3[(a,b)][c] (K-major)
//   A3            --Zz----> D4[(a,b)][z] -> A4[(a,z)][b]   (MN-major)
//   A4            --Zy----> D5[(a,z)][y] -> A5[(z,y)][a]   (MN-major)
//   A5            --Zx----> D6[(z,y)][x] -> omega * D6 added to the plane accumulators
//
// so each thread's TMEM row is stored as two 16-byte rows of core matrices.
// One thread issues the MMAs and a tcgen05.commit arrives on an mbarrier;
// the wait for it is bounded (about a second); on expiry the kernel records
// the failure in a host-visible flag, waits for its own copies, frees its
// TMEM and returns, and the next smoother call on the patch set reports
// TPSS_ETIMEOUT.
#include "tc05.cuh"
#include "tpss_internal.cuh"

namespace tpss {
namespace tcs {

constexpr int kThreads = 128;
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

// byte offsets of the operand layouts (see tc05.cuh): 256 rows x 16 K of BF16
// in core matrices of 8 rows x 16 bytes; K-direction stride 4096 bytes,
// M-direction stride 128 bytes
__device__ __forceinline__ int off_k(int m) { return (m & 7) * 16 + (m >> 3) * 128; }   // + 4096 for k >= 8
__device__ __forceinline__ int off_mn(int slow, int k) { return (k & 7) * 16 + slow * 256 + (k >> 3) * 4096; }

template <int N>
struct Smem {
  static constexpr int N1 = N / 2;
  static constexpr int NLOC1 = N1 * N1 * N1;
  static constexpr int NP = 4 * NLOC1;                 // floats of one column plane (4 cells)
  static constexpr size_t OPA = 0;                     // 8192 bytes: operand A
  static constexpr size_t OPB = 8192;                  // 6 x 512 bytes: operands B
  static constexpr size_t SB = OPB + 6 * 512;          // 3 staged planes of r (FP32)
  static constexpr size_t ACC = SB + 3 * (size_t)NP * 4;   // 2 plane accumulators (FP32)
  static constexpr size_t BYTES = ACC + 2 * (size_t)NP * 4;
};

// B operand s (16 x 16, K-major) from the 1D eigenvector matrix Z (node-major
// Z[i * N + mode]): forward (Z^T applied): B[n][k] = Z[k][n]; back (Z
// applied): B[n][k] = Z[n][k]; zero outside N x N.
template <int N>
__device__ __forceinline__ void write_b(unsigned char* ob, const float* __restrict__ Z, bool back, int tid) {
  __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(ob);
  for (int e = tid; e < 256; e += kThreads) {
    const int n = e >> 4, k = e & 15;
    float v = 0.f;
    if (n < N && k < N) v = back ? __ldg(Z + n * N + k) : __ldg(Z + k * N + n);
    b[((n & 7) * 16 + (n >> 3) * 128 + (k >> 3) * 256 + (k & 7) * 2) / 2] = __float2bfloat16(v);
  }
}

template <int NLOC1>
__device__ __forceinline__ void stage_plane(float* dst, const float* __restrict__ src, int px, int py, int cz,
                                            int nc0, int nc1, int tid) {
  const uint32_t d = tc05::smem_u32(dst);
  auto cell0 = [&](int c2) -> int64_t {
    return ((px + (c2 & 1)) + (int64_t)nc0 * ((py + (c2 >> 1)) + (int64_t)nc1 * cz)) * NLOC1;
  };
  if constexpr (NLOC1 % 4 == 0) {
    constexpr int CH = NLOC1 / 4;
    for (int e = tid; e < 4 * CH; e += kThreads) {
      const int c2 = e / CH, o = (e % CH) * 4;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d + 4u * (c2 * NLOC1 + o)),
                   "l"(src + cell0(c2) + o) : "memory");
    }
  } else {
    for (int e = tid; e < 4 * NLOC1; e += kThreads) {
      const int c2 = e / NLOC1, o = e % NLOC1;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(d + 4u * (c2 * NLOC1 + o)),
                   "l"(src + cell0(c2) + o) : "memory");
    }
  }
}

__device__ __forceinline__ int first_class(int cx, int cy, int nc0, int nc1) {
  const int xm = (cx == nc0 - 1) ? (nc0 & 1) : 0;
  const int ym = (cy == nc1 - 1) ? (nc1 & 1) : 0;
  return xm + 2 * ym;
}

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

// stage s (1..6): A layout of the MMA's operand (0 K-major, 1 MN-major)
__device__ __forceinline__ int a_major(int s) { return (s == 1 || s == 4) ? 0 : 1; }

template <int N>
__global__ void __launch_bounds__(kThreads, 4)
patch_stream_tc05_kernel(const float* __restrict__ Z0, const float* __restrict__ Z1, const float* __restrict__ Z2,
                         const float* __restrict__ L0, const float* __restrict__ L1, const float* __restrict__ L2,
                         const float* __restrict__ r, float* __restrict__ x, float omega, int nc0, int nc1, int nc2,
                         int64_t ndofs, int cls, int ncolx, int x_is_zero, volatile int* fail_flag) {
  using M = Smem<N>;
  constexpr int N1 = N / 2;
  constexpr int NLOC1 = M::NLOC1;
  constexpr int NP = M::NP;
  constexpr int NB = N > 8 ? 2 : 1;   // blocks of 128 rows: slow index < 8 NB
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* opa = dsm + M::OPA;
  unsigned char* opb = dsm + M::OPB;
  float* SB = reinterpret_cast<float*>(dsm + M::SB);
  float* ACC = reinterpret_cast<float*>(dsm + M::ACC);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ float lam[48];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int px = (cls & 1) + 2 * (int)(blockIdx.x % ncolx);
  const int py = (cls >> 1) + 2 * (int)(blockIdx.x / ncolx);
  r += (int64_t)blockIdx.y * ndofs;
  x += (int64_t)blockIdx.y * ndofs;
  const uint32_t mb = tc05::smem_u32(&mbar);

  stage_plane<NLOC1>(SB, r, px, py, 0, nc0, nc1, tid);
  stage_plane<NLOC1>(SB + NP, r, px, py, 1, nc0, nc1, tid);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int e = tid; e < 8192 / 16; e += kThreads) reinterpret_cast<uint4*>(opa)[e] = make_uint4(0, 0, 0, 0);
  for (int e = tid; e < 2 * NP; e += kThreads) ACC[e] = 0.f;
  if (tid < 32) lam[tid] = (tid < 16) ? (tid < N ? L0[(size_t)px * N + tid] : 0.f)
                                      : (tid - 16 < N ? L1[(size_t)py * N + tid - 16] : 0.f);
  write_b<N>(opb + 0 * 512, Z0 + (size_t)px * N * N, false, tid);
  write_b<N>(opb + 1 * 512, Z1 + (size_t)py * N * N, false, tid);
  write_b<N>(opb + 4 * 512, Z1 + (size_t)py * N * N, true, tid);
  write_b<N>(opb + 5 * 512, Z0 + (size_t)px * N * N, true, tid);
  if (tid == 0) tc05::mbar_init(mb, 1);
  if (warp == 0) tc05::alloc(tc05::smem_u32(&tslot), 32);
  tc05::fence_before_sync();
  __syncthreads();
  tc05::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's lanes
  const uint32_t a_base = tc05::smem_u32(opa), b_base = tc05::smem_u32(opb);
  uint32_t phase = 0;
  bool failed = false;

  for (int pz = 0; pz + 1 < nc2 && !failed; ++pz) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();   // planes pz, pz + 1 staged; the previous patch is done with the operands and slot (pz + 2) % 3
    if (pz + 2 < nc2) {
      stage_plane<NLOC1>(SB + ((pz + 2) % 3) * NP, r, px, py, pz + 2, nc0, nc1, tid);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    if (tid < 16) lam[32 + tid] = tid < N ? L2[(size_t)pz * N + tid] : 0.f;
    write_b<N>(opb + 2 * 512, Z2 + (size_t)pz * N * N, false, tid);
    write_b<N>(opb + 3 * 512, Z2 + (size_t)pz * N * N, true, tid);
    // gather: A0[(z, y)][x] (K-major), zero outside the patch
    const float* lo = SB + (pz % 3) * NP;
    const float* hi = SB + ((pz + 1) % 3) * NP;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int m = tid + 128 * b, z = m >> 4, y = m & 15;
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
      if (z < N && y < N) {
        const float* src = (z >= N1 ? hi : lo) + 2 * (y / N1) * NLOC1 + N1 * ((y % N1) + N1 * (z % N1));
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = src[(j / N1) * NLOC1 + (j % N1)];
      }
      tc05::st_row8(opa + off_k(m), v);
      tc05::st_row8(opa + off_k(m) + 4096, v + 8);
    }
    tc05::fence_proxy_async();
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();

    for (int s = 1; s <= 6; ++s) {
      if (tid == 0) {
        const uint32_t idesc = tc05::idesc_bf16(128, 16, a_major(s), 0);
        const uint64_t bdesc = tc05::desc(b_base + 512 * (s - 1), 256, 128);
#pragma unroll
        for (int b = 0; b < NB; ++b)
          tc05::mma(tmem + 16 * b, tc05::desc(a_base + 2048 * b, 4096, 128), bdesc, idesc, 0);
        tc05::commit(mb);
      }
      const bool ok = tc05::mbar_wait_bounded(mb, phase, kWaitCycles);
      phase ^= 1;
      tc05::fence_after_sync();
      float v[16 * NB];
      if constexpr (NB == 2) {
        tc05::ld32(trow, v);
      } else {
        tc05::ld16(trow, v);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int m = tid + 128 * b, sl = m >> 4, fa = m & 15;
        float* w = v + 16 * b;
        if (s == 1 || s == 4) {          // D1[(z,y)][a] -> A1[(z,a)][y];  D4[(a,b)][z] -> A4[(a,z)][b]
          if (NB == 2 || sl < 8) {
            tc05::st_row8(opa + off_mn(sl, fa), w);
            tc05::st_row8(opa + off_mn(sl, fa) + 128, w + 8);
          }
        } else if (s == 2 || s == 5) {   // D2[(z,a)][b] -> A2[(a,b)][z];  D5[(a,z)][y] -> A5[(z,y)][a]
          if (NB == 2 || fa < 8) {
            tc05::st_row8(opa + off_mn(fa, sl), w);
            tc05::st_row8(opa + off_mn(fa, sl) + 128, w + 8);
          }
        } else if (s == 3) {             // D3[(a,b)][c] / (lx_a + ly_b + lz_c) -> A3[(a,b)][c]
          const float sab = lam[sl] + lam[16 + fa];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            w[j] = (sl < N && fa < N && j < N) ? __fdividef(w[j], sab + lam[32 + j]) : 0.f;
          tc05::st_row8(opa + off_k(m), w);
          tc05::st_row8(opa + off_k(m) + 4096, w + 8);
        } else {                         // D6[(z,y)][x]: omega * line -> plane accumulators
          if (sl < N && fa < N) {
            const int sz = sl / N1, iz = sl % N1, sy = fa / N1, iy = fa % N1;
            float* acc = ACC + ((pz + sz) & 1) * NP + 2 * sy * NLOC1 + N1 * (iy + N1 * iz);
#pragma unroll
            for (int j = 0; j < N; ++j) acc[(j / N1) * NLOC1 + (j % N1)] += omega * w[j];
          }
        }
      }
      if (s < 6) {
        tc05::fence_proxy_async();
        tc05::fence_before_sync();
      }
      failed = __syncthreads_or(!ok) != 0;   // also: the next operand is complete
      tc05::fence_after_sync();
      if (failed) break;
    }
    if (failed) break;
    // plane pz now has both of its patches of this column
    flush_plane<N1>(x, ACC + (pz & 1) * NP, px, py, pz, nc0, nc1, cls, x_is_zero, tid);
  }
  if (!failed) {
    __syncthreads();
    flush_plane<N1>(x, ACC + ((nc2 - 1) & 1) * NP, px, py, nc2 - 1, nc0, nc1, cls, x_is_zero, tid);
  } else if (tid == 0) {
    *fail_flag = 1;
    __threadfence_system();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc05::dealloc(tmem, 32);
}

template <int N>
static tpss_status launch(tpss_patches* P, float omega, int nrhs, const float* r, float* x, int x_is_zero,
                          cudaStream_t s) {
  constexpr size_t smem = Smem<N>::BYTES;
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(patch_stream_tc05_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr = true;
  }
  const Level& L = P->ctx->levels[P->level];
  const int nc0 = L.nc[0], nc1 = L.nc[1], nc2 = L.nc[2];
  for (int cls = 0; cls < 4; ++cls) {
    const int ax = cls & 1, ay = cls >> 1;
    const int ncolx = ax <= nc0 - 2 ? (nc0 - 2 - ax) / 2 + 1 : 0;
    const int ncoly = ay <= nc1 - 2 ? (nc1 - 2 - ay) / 2 + 1 : 0;
    if (ncolx == 0 || ncoly == 0) continue;
    dim3 grid((unsigned)(ncolx * ncoly), (unsigned)nrhs);
    patch_stream_tc05_kernel<N><<<grid, kThreads, smem, s>>>(
        P->d_Z32[0], P->d_Z32[1], P->d_Z32[2], P->d_lam32[0], P->d_lam32[1], P->d_lam32[2], r, x, omega, nc0, nc1,
        nc2, L.ndofs, cls, ncolx, x_is_zero, P->d_fail_flag);
    TPSS_CHECK_LAUNCH();
  }
  return TPSS_OK;
}

}  // namespace tcs

// The additive pass of the tcgen05 column-streaming schedule (all four
// parity classes); TPSS_EINVAL without launching for shapes it does not
// cover (the same as the COLUMNS schedule); TPSS_ETIMEOUT if a previous
// launch on this patch set gave up waiting for its MMAs.
tpss_status patch_pass_bf16_tc05(tpss_patches* P, float omega, int nrhs, const float* r, float* x, int x_is_zero,
                                 cudaStream_t s) {
  if (P->ctx->dim != 3 || P->kind != TPSS_VERTEX_PATCH || P->per_sub) return TPSS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(x)) & 15) return TPSS_EINVAL;
  const Level& L = P->ctx->levels[P->level];
  if (L.nc[0] < 2 || L.nc[1] < 2 || L.nc[2] < 2 || nrhs > 65535 || P->n > 16) return TPSS_EINVAL;
  if (P->h_fail_flag == nullptr) {
    // a host-visible word the kernel sets if it gives up waiting (read without a device synchronization)
    void* h = nullptr;
    TPSS_CHECK_CUDA(cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped));
    P->h_fail_flag = static_cast<int*>(h);
    *P->h_fail_flag = 0;
    void* d = nullptr;
    TPSS_CHECK_CUDA(cudaHostGetDevicePointer(&d, h, 0));
    P->d_fail_flag = static_cast<int*>(d);
  }
  if (*reinterpret_cast<volatile int*>(P->h_fail_flag) != 0) {
    *P->h_fail_flag = 0;
    set_error("BF16 tensor-core smoother: an MMA completion wait expired in an earlier call (its result is invalid)");
    return TPSS_ETIMEOUT;
  }
  switch (P->n) {
    case 4: return tcs::launch<4>(P, omega, nrhs, r, x, x_is_zero, s);
    case 6: return tcs::launch<6>(P, omega, nrhs, r, x, x_is_zero, s);
    case 8: return tcs::launch<8>(P, omega, nrhs, r, x, x_is_zero, s);
    case 10: return tcs::launch<10>(P, omega, nrhs, r, x, x_is_zero, s);
    case 12: return tcs::launch<12>(P, omega, nrhs, r, x, x_is_zero, s);
    case 14: return tcs::launch<14>(P, omega, nrhs, r, x, x_is_zero, s);
    case 16: return tcs::launch<16>(P, omega, nrhs, r, x, x_is_zero, s);
    default: return TPSS_EINVAL;
  }
}

}  // namespace tpss
