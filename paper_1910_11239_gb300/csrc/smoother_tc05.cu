// Column-streaming BF16 / TF32 additive vertex-patch smoother on the
// 5th-generation tensor cores (tcgen05 MMA, accumulators in tensor memory);
// 3D, mixed precision (not in the paper).
//
// Schedule: as the COLUMNS schedule (smoother_stream.cu): one CTA per column
// of vertex patches (p_x, p_y) and right-hand side walks p_z, r staged one
// cell plane ahead with cp.async, each cell plane of x written once per
// parity class of (p_x, p_y) when both of its patches in the column are done.
//
// Local solve (eq. fastinverse, eq. eigenvectormatvec): the six mode
// contractions of (Z_z x Z_y x Z_x) Lambda^{-1} (Z_z x Z_y x Z_x)^T are six
// MMAs D = A B with M = 128 (one or two blocks of 128 rows), N = 16, K = 16,
// BF16 operands from shared memory, FP32 accumulation in TMEM.  Every index
// is padded to 16, so the patch tensor has 256 "lines" (slow index s, fast
// index f, row m = 16 s + f).  A is the tensor with the contracted index as
// K; B is the 1D eigenvector matrix (K-major 16 x 16, zero padded, prepared
// once per position at setup and staged with cp.async).  After each MMA every
// thread reads its TMEM rows (row m = thread + 128 b) and writes them back to
// shared memory as the next A, rotating the indices so that the next
// contracted index becomes K:
//
//   A0[(z,y)][x]  --Zx^T--> D1[(z,y)][a] -> A1[(z,a)][y]   (MN-major write)
//   A1            --Zy^T--> D2[(z,a)][b] -> A2[(a,b)][z]   (MN-major)
//   A2            --Zz^T--> D3[(a,b)][c] -> scaled by 1/(lx_a + ly_b + lz_c) -> A3[(a,b)][c] (K-major)
//   A3            --Zz----> D4[(a,b)][z] -> A4[(a,z)][b]   (MN-major)
//   A4            --Zy----> D5[(a,z)][y] -> A5[(z,y)][a]   (MN-major)
//   A5            --Zx----> D6[(z,y)][x] -> omega * D6, the patch's correction
//
// so each thread's TMEM row goes back as two 16-byte rows of core matrices.
// The core matrices of A sit 144 bytes apart along M (not 128) so that these
// writes are free of shared-memory bank conflicts.
//
// TF32 (kind::tf32, K = 8 per MMA): the same walk with FP32 operands rounded
// to TF32, two MMAs per 16-wide contraction and every operand K-major (a
// core matrix row holds 4 values); the rotated stages write their values to
// the next A one by one instead of as MN-major rows.
//
// Output: with k = 7 (16 points per direction) a thread's two rows of D6 are
// the same (y, z) line of the patch's lower and upper cell plane; the upper
// one is kept in registers until the next patch of the column adds the lower
// one of that plane, and the finished line (two cell rows) goes straight to
// x.  Other degrees accumulate in FP32 plane buffers in shared memory and
// write each finished plane.
//
// One thread issues the MMAs; a tcgen05.commit arrives on an mbarrier.  The
// wait for it is bounded (about a second): on expiry the kernel records the
// failure in a host-visible flag, waits for its own copies, frees its TMEM and
// returns, and the next smoother call on the patch set reports TPSS_ETIMEOUT.
#include "tc05.cuh"
#include "tpss_internal.cuh"

namespace tpss {
namespace tcs {

constexpr int kThreads = 128;
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz
constexpr int kMStride = 144;                     // bytes between core matrices along M
constexpr int kKStride = 32 * kMStride;           // bytes between core matrices along K (256 rows)

// per element type: A bytes (2 or 4 core-matrix columns of 8 or 4 values),
// one 16 x 16 B operand, the B operands of one position (Z^T and Z)
template <bool TF> struct Op {
  static constexpr int ABYTES = (TF ? 4 : 2) * kKStride;
  static constexpr int BBYTES = TF ? 1024 : 512;
  static constexpr int BPOS = 2 * BBYTES;
};

// byte offset of row m of a K-major A (K half 0; + kKStride for K half 1)
__device__ __forceinline__ int off_k(int m) { return (m & 7) * 16 + (m >> 3) * kMStride; }
// byte offset of the run of rows 16 slow .. 16 slow + 7 at column k of an
// MN-major A (rows 16 slow + 8 .. + 15: + kMStride)
__device__ __forceinline__ int off_mn(int slow, int k) {
  return (k & 7) * 16 + slow * 2 * kMStride + (k >> 3) * kKStride;
}

template <int N, bool TF>
struct Smem {
  static constexpr int N1 = N / 2;
  static constexpr int NLOC1 = N1 * N1 * N1;
  static constexpr int NP = 4 * NLOC1;                       // floats of one column plane (4 cells)
  static constexpr bool CARRY = (N == 16);                   // finished lines kept in registers
  static constexpr size_t OPA = 0;
  static constexpr size_t OPB = Op<TF>::ABYTES;              // 8 operands B
  static constexpr size_t SB = OPB + 8 * Op<TF>::BBYTES;     // 3 staged planes of r (FP32)
  static constexpr size_t ACC = SB + 3 * (size_t)NP * 4;     // 2 plane accumulators (FP32) unless CARRY
  static constexpr size_t BYTES = ACC + (CARRY ? 0 : 2 * (size_t)NP * 4);
};
// B operand slots (pairs as stored per position: Z^T-apply, Z-apply): 0 / 1 x,
// 2 / 3 y, 4 + 2q / 5 + 2q z of the patch with p_z & 1 == q.  Stage s (1..6)
// of patch p_z uses:
__device__ __forceinline__ int b_slot(int s, int q) {
  return s == 1 ? 0 : s == 2 ? 2 : s == 3 ? 4 + 2 * q : s == 4 ? 5 + 2 * q : s == 5 ? 3 : 1;
}
// A layout of the BF16 MMA of stage s (0 K-major, 1 MN-major)
__device__ __forceinline__ int a_major(int s) { return (s == 1 || s == 4) ? 0 : 1; }

// Global B operands: [t][position][apply Z^T (0) / Z (1)][512 bytes], the
// 16 x 16 K-major BF16 matrix B[n][k] = Z[k][n] (0) or Z[n][k] (1), Z[node][mode].
__global__ void prepare_bop_kernel(const float* __restrict__ Z, int npos, int n, __nv_bfloat16* __restrict__ out) {
  const int p = blockIdx.x, back = blockIdx.y;
  if (p >= npos) return;
  const float* Zp = Z + (size_t)p * n * n;
  __nv_bfloat16* o = out + ((size_t)p * 2 + back) * 256;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int nn = e >> 4, k = e & 15;
    float v = 0.f;
    if (nn < n && k < n) v = back ? Zp[nn * n + k] : Zp[k * n + nn];
    o[((nn & 7) * 16 + (nn >> 3) * 128 + (k >> 3) * 256 + (k & 7) * 2) / 2] = __float2bfloat16(v);
  }
}

// The same for TF32: [t][position][Z^T / Z][1024 bytes], 16 x 16 K-major with
// core matrices of 8 rows x 4 values, rounded to TF32.
__global__ void prepare_bop_tf32_kernel(const float* __restrict__ Z, int npos, int n, float* __restrict__ out) {
  const int p = blockIdx.x, back = blockIdx.y;
  if (p >= npos) return;
  const float* Zp = Z + (size_t)p * n * n;
  float* o = out + ((size_t)p * 2 + back) * 256;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int nn = e >> 4, k = e & 15;
    float v = 0.f;
    if (nn < n && k < n) v = back ? Zp[nn * n + k] : Zp[k * n + nn];
    o[((nn & 7) * 16 + (nn >> 3) * 128 + (k >> 2) * 256 + (k & 3) * 4) / 4] = __uint_as_float(tc05::to_tf32(v));
  }
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
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
      cp16(d + 4u * (c2 * NLOC1 + o), src + cell0(c2) + o);
    }
  } else {
    for (int e = tid; e < 4 * NLOC1; e += kThreads) {
      const int c2 = e / NLOC1, o = e % NLOC1;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(d + 4u * (c2 * NLOC1 + o)),
                   "l"(src + cell0(c2) + o) : "memory");
    }
  }
}

// the B operands of one position (two matrices) -> shared memory
template <bool TF>
__device__ __forceinline__ void stage_b2(unsigned char* dst, const unsigned char* src, int tid) {
  if (tid < Op<TF>::BPOS / 16) cp16(tc05::smem_u32(dst) + 16u * tid, src + 16 * tid);
}

// row m (16 values along K) of a K-major A
template <bool TF>
__device__ __forceinline__ void put_row_k(unsigned char* opa, int m, const float* v) {
  if constexpr (TF) {
#pragma unroll
    for (int c = 0; c < 4; ++c) tc05::st_row4_tf32(opa + off_k(m) + c * kKStride, v + 4 * c);
  } else {
    tc05::st_row8(opa + off_k(m), v);
    tc05::st_row8(opa + off_k(m) + kKStride, v + 8);
  }
}
// rows 16 slow + j (j = 0..15) at column k of A: MN-major rows (BF16) or
// one value per row of the K-major TF32 operand
template <bool TF>
__device__ __forceinline__ void put_col(unsigned char* opa, int slow, int k, const float* v) {
  if constexpr (TF) {
    unsigned char* base = opa + (k & 3) * 4 + (k >> 2) * kKStride;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      *reinterpret_cast<uint32_t*>(base + off_k(16 * slow + j)) = tc05::to_tf32(v[j]);
  } else {
    tc05::st_row8(opa + off_mn(slow, k), v);
    tc05::st_row8(opa + off_mn(slow, k) + kMStride, v + 8);
  }
}

__device__ __forceinline__ int first_class(int cx, int cy, int nc0, int nc1) {
  const int xm = (cx == nc0 - 1) ? (nc0 & 1) : 0;
  const int ym = (cy == nc1 - 1) ? (nc1 & 1) : 0;
  return xm + 2 * ym;
}

// The previous values of cell plane cz of x (read-modify-write cells only)
// -> shared memory, with cp.async, in the element order of flush_plane (each
// thread later reads only what it copied itself).
template <int N1>
__device__ __forceinline__ void prefetch_plane(float* xo, const float* __restrict__ x, int px, int py, int cz,
                                               int nc0, int nc1, int cls, int x_is_zero, int tid) {
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int V = (NLOC1 % 4 == 0) ? 4 : 1;
  constexpr int CH = NLOC1 / V;
  const uint32_t d = tc05::smem_u32(xo);
  for (int e = tid; e < 4 * CH; e += kThreads) {
    const int c2 = e / CH, o = (e % CH) * V;
    const int cx = px + (c2 & 1), cy = py + (c2 >> 1);
    if (x_is_zero && first_class(cx, cy, nc0, nc1) == cls) continue;
    const float* src = x + (cx + (int64_t)nc0 * (cy + (int64_t)nc1 * cz)) * NLOC1 + o;
    if constexpr (V == 4)
      cp16(d + 4u * (c2 * NLOC1 + o), src);
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(d + 4u * (c2 * NLOC1 + o)), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// x (plane cz) = acc, or xo + acc for the read-modify-write cells; acc is cleared
template <int N1>
__device__ __forceinline__ void flush_plane(float* __restrict__ x, float* acc, const float* xo, int px, int py,
                                            int cz, int nc0, int nc1, int cls, int x_is_zero, int tid) {
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int V = (NLOC1 % 4 == 0) ? 4 : 1;
  constexpr int CH = NLOC1 / V;
  asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's prefetched values
  for (int e = tid; e < 4 * CH; e += kThreads) {
    const int c2 = e / CH, o = (e % CH) * V;
    const int cx = px + (c2 & 1), cy = py + (c2 >> 1);
    const bool store = x_is_zero && first_class(cx, cy, nc0, nc1) == cls;
    float* dst = x + (cx + (int64_t)nc0 * (cy + (int64_t)nc1 * cz)) * NLOC1 + o;
    float* a = acc + c2 * NLOC1 + o;
    if constexpr (V == 4) {
      float4 v = *reinterpret_cast<float4*>(a);
      if (!store) {
        const float4 old = *reinterpret_cast<const float4*>(xo + c2 * NLOC1 + o);
        v.x += old.x;
        v.y += old.y;
        v.z += old.z;
        v.w += old.w;
      }
      *reinterpret_cast<float4*>(dst) = v;
      *reinterpret_cast<float4*>(a) = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      const float v = *a;
      *dst = store ? v : v + xo[c2 * NLOC1 + o];
      *a = 0.f;
    }
  }
}

template <int N, bool TF>
__global__ void __launch_bounds__(kThreads, TF ? 4 : 5)   // TF32 at k = 7: 51 KB of shared memory, 4 CTAs
patch_stream_tc05_kernel(const unsigned char* __restrict__ B0, const unsigned char* __restrict__ B1,
                         const unsigned char* __restrict__ B2, const float* __restrict__ L0,
                         const float* __restrict__ L1, const float* __restrict__ L2, const float* __restrict__ r,
                         float* __restrict__ x, float omega, int nc0, int nc1, int nc2, int64_t ndofs, int cls,
                         int ncolx, int x_is_zero, volatile int* fail_flag, int expire_test) {
  using M = Smem<N, TF>;
  constexpr int BB = Op<TF>::BBYTES, BP = Op<TF>::BPOS;
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
  __shared__ __align__(16) float lam[64];   // x, y (columns), z of patch p_z in slot 32 + 16 (p_z & 1)
  const int tid = threadIdx.x, warp = tid >> 5;
  const int px = (cls & 1) + 2 * (int)(blockIdx.x % ncolx);
  const int py = (cls >> 1) + 2 * (int)(blockIdx.x / ncolx);
  r += (int64_t)blockIdx.y * ndofs;
  x += (int64_t)blockIdx.y * ndofs;
  const uint32_t mb = tc05::smem_u32(&mbar);

  // prologue: planes 0 and 1, the column's x and y operands, patch 0's z operands
  stage_plane<NLOC1>(SB, r, px, py, 0, nc0, nc1, tid);
  stage_plane<NLOC1>(SB + NP, r, px, py, 1, nc0, nc1, tid);
  stage_b2<TF>(opb + 0 * BB, B0 + (size_t)px * BP, tid);   // slots 0, 1
  stage_b2<TF>(opb + 2 * BB, B1 + (size_t)py * BP, tid);   // slots 2, 3
  stage_b2<TF>(opb + 4 * BB, B2, tid);                     // patch 0: slots 4, 5
  if (tid < N)                                           // patch 0's z eigenvalues
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(tc05::smem_u32(lam + 32 + tid)),
                 "l"(L2 + tid) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int e = tid; e < Op<TF>::ABYTES / 16; e += kThreads) reinterpret_cast<uint4*>(opa)[e] = make_uint4(0, 0, 0, 0);
  if constexpr (!M::CARRY)
    for (int e = tid; e < 2 * NP; e += kThreads) ACC[e] = 0.f;
  if (tid < 32) lam[tid] = (tid < 16) ? (tid < N ? L0[(size_t)px * N + tid] : 0.f)
                                      : (tid - 16 < N ? L1[(size_t)py * N + tid - 16] : 0.f);
  // (z slots: entries >= N are never read)
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

  // CARRY (k = 7): this thread's line (y = tid & 15, local z = tid >> 4) of the
  // two cells (sx = 0, 1) at (p_x + sx, p_y + y / 8)
  const int ly = tid & 15, liz = tid >> 4;
  float carry[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) carry[j] = 0.f;
  bool store_cell[2] = {false, false};
  int64_t line_off[2] = {0, 0};
  if constexpr (M::CARRY) {
#pragma unroll
    for (int sx = 0; sx < 2; ++sx) {
      const int cx = px + sx, cy = py + (ly >> 3);
      store_cell[sx] = x_is_zero && first_class(cx, cy, nc0, nc1) == cls;
      line_off[sx] = (cx + (int64_t)nc0 * cy) * NLOC1 + 8 * ((ly & 7) + 8 * liz);
    }
  }
  const int64_t plane_stride = (int64_t)nc0 * nc1 * NLOC1;
  // k = 7 plane staging: thread t copies 16 bytes at float 4 t of each of the 4 cells
  int64_t stage_off[4];
#pragma unroll
  for (int c2 = 0; c2 < 4; ++c2) stage_off[c2] = ((px + (c2 & 1)) + (int64_t)nc0 * (py + (c2 >> 1))) * NLOC1 + 4 * tid;

  for (int pz = 0; pz + 1 < nc2 && !failed; ++pz) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();   // planes pz, pz + 1 and patch pz's z operands staged; patch pz - 1 is done
    if (pz + 2 < nc2) {
      if constexpr (NLOC1 == 4 * kThreads) {
        const uint32_t d = tc05::smem_u32(SB + ((pz + 2) % 3) * NP) + 16u * tid;
        const float* src = r + (int64_t)(pz + 2) * plane_stride;
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) cp16(d + 4u * NLOC1 * c2, src + stage_off[c2]);
      } else {
        stage_plane<NLOC1>(SB + ((pz + 2) % 3) * NP, r, px, py, pz + 2, nc0, nc1, tid);
      }
      stage_b2<TF>(opb + (4 + 2 * ((pz + 1) & 1)) * BB, B2 + (size_t)(pz + 1) * BP, tid);
      if (tid < N)   // the next patch's z eigenvalues
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                     :: "r"(tc05::smem_u32(lam + 32 + 16 * ((pz + 1) & 1) + tid)), "l"(L2 + (size_t)(pz + 1) * N + tid)
                     : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const float* lamz = lam + 32 + 16 * (pz & 1);
    // previous values of this thread's line of plane pz (read-modify-write classes)
    float xold[16];
    if constexpr (M::CARRY) {
#pragma unroll
      for (int sx = 0; sx < 2; ++sx) {
        const float* src = x + line_off[sx] + pz * plane_stride;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (!store_cell[sx]) v = *reinterpret_cast<const float4*>(src + 4 * q);
          xold[8 * sx + 4 * q] = v.x;
          xold[8 * sx + 4 * q + 1] = v.y;
          xold[8 * sx + 4 * q + 2] = v.z;
          xold[8 * sx + 4 * q + 3] = v.w;
        }
      }
    }
    // gather: A0[(z, y)][x] (K-major), zero outside the patch
    const float* lo = SB + (pz % 3) * NP;
    const float* hi = SB + ((pz + 1) % 3) * NP;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int m = tid + 128 * b, z = m >> 4, y = m & 15;
      float v[16];
      if constexpr (N1 == 8) {
        const float* src = (b ? hi : lo) + 2 * (y >> 3) * NLOC1 + 8 * ((y & 7) + 8 * (z & 7));
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
          const float4 a0 = *reinterpret_cast<const float4*>(src + sx * NLOC1);
          const float4 a1 = *reinterpret_cast<const float4*>(src + sx * NLOC1 + 4);
          v[8 * sx] = a0.x; v[8 * sx + 1] = a0.y; v[8 * sx + 2] = a0.z; v[8 * sx + 3] = a0.w;
          v[8 * sx + 4] = a1.x; v[8 * sx + 5] = a1.y; v[8 * sx + 6] = a1.z; v[8 * sx + 7] = a1.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
        if (z < N && y < N) {
          const float* src = (z >= N1 ? hi : lo) + 2 * (y / N1) * NLOC1 + N1 * ((y % N1) + N1 * (z % N1));
#pragma unroll
          for (int j = 0; j < N; ++j) v[j] = src[(j / N1) * NLOC1 + (j % N1)];
        }
      }
      put_row_k<TF>(opa, m, v);
    }
    tc05::fence_proxy_async();
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    if constexpr (!M::CARRY) {   // r of plane pz (and of the last plane) is consumed: its slots take x
      prefetch_plane<N1>(SB + (pz % 3) * NP, x, px, py, pz, nc0, nc1, cls, x_is_zero, tid);
      if (pz + 2 == nc2)
        prefetch_plane<N1>(SB + ((pz + 1) % 3) * NP, x, px, py, pz + 1, nc0, nc1, cls, x_is_zero, tid);
    }

#pragma unroll
    for (int s = 1; s <= 6; ++s) {   // unrolled: every stage's index rotation is resolved at compile time
      if (tid == 0) {
        const uint32_t bslot = b_base + BB * b_slot(s, pz & 1);
        if constexpr (TF) {   // K = 16 as two MMAs of K = 8 (core-matrix columns 2h, 2h + 1)
          constexpr uint32_t idesc = tc05::idesc_tf32(128, 16);
#pragma unroll
          for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              tc05::mma_tf32(tmem + 16 * b,
                             tc05::desc(a_base + 16 * kMStride * b + 2 * h * kKStride, kKStride, kMStride),
                             tc05::desc(bslot + 512 * h, 256, 128), idesc, h);
        } else {
          const uint32_t idesc = tc05::idesc_bf16(128, 16, a_major(s), 0);
          const uint64_t bdesc = tc05::desc(bslot, 256, 128);
#pragma unroll
          for (int b = 0; b < NB; ++b)
            tc05::mma(tmem + 16 * b, tc05::desc(a_base + 16 * kMStride * b, kKStride, kMStride), bdesc, idesc, 0);
        }
        tc05::commit(mb);
      }
      bool ok = tc05::mbar_wait_bounded(mb, phase, kWaitCycles);
      // expire_test: after the first MMA has completed, wait (with a short
      // bound) for the next phase, which no commit completes, so that the
      // failure path runs with no MMA in flight
      if (expire_test && pz == 0 && s == 1) ok = ok && tc05::mbar_wait_bounded(mb, phase ^ 1, 2000000LL);
      phase ^= 1;
      tc05::fence_after_sync();
      float v[16 * NB];
      if constexpr (NB == 2) {
        tc05::ld32(trow, v);
      } else {
        tc05::ld16(trow, v);
      }
      if (s == 6 && M::CARRY) {
        // rows: block 0 = line (liz, ly) of plane pz (lower cells), block 1 = plane pz + 1
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          xold[j] += carry[j] + omega * v[j];
          carry[j] = omega * v[16 + j];
        }
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
          float* dst = x + line_off[sx] + pz * plane_stride;
          *reinterpret_cast<float4*>(dst) = make_float4(xold[8 * sx], xold[8 * sx + 1], xold[8 * sx + 2],
                                                        xold[8 * sx + 3]);
          *reinterpret_cast<float4*>(dst + 4) = make_float4(xold[8 * sx + 4], xold[8 * sx + 5],
                                                            xold[8 * sx + 6], xold[8 * sx + 7]);
        }
      } else {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int m = tid + 128 * b, sl = m >> 4, fa = m & 15;
          float* w = v + 16 * b;
          if (s == 1 || s == 4) {          // D1[(z,y)][a] -> A1[(z,a)][y];  D4[(a,b)][z] -> A4[(a,z)][b]
            if (NB == 2 || sl < 8) put_col<TF>(opa, sl, fa, w);
          } else if (s == 2 || s == 5) {   // D2[(z,a)][b] -> A2[(a,b)][z];  D5[(a,z)][y] -> A5[(z,y)][a]
            if (NB == 2 || fa < 8) put_col<TF>(opa, fa, sl, w);
          } else if (s == 3) {             // D3[(a,b)][c] / (lx_a + ly_b + lz_c) -> A3[(a,b)][c]
            const float sab = lam[sl] + lam[16 + fa];
#pragma unroll
            for (int j = 0; j < 16; ++j)
              w[j] = (sl < N && fa < N && j < N) ? __fdividef(w[j], sab + lamz[j]) : 0.f;
            put_row_k<TF>(opa, m, w);
          } else if constexpr (!M::CARRY) {   // D6[(z,y)][x]: omega * line -> plane accumulators
            if (sl < N && fa < N) {
              const int sz = sl / N1, iz = sl % N1, sy = fa / N1, iy = fa % N1;
              float* acc = ACC + ((pz + sz) & 1) * NP + 2 * sy * NLOC1 + N1 * (iy + N1 * iz);
#pragma unroll
              for (int j = 0; j < N; ++j) acc[(j / N1) * NLOC1 + (j % N1)] += omega * w[j];
            }
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
    if constexpr (!M::CARRY)   // plane pz now has both of its patches of this column
      flush_plane<N1>(x, ACC + (pz & 1) * NP, SB + (pz % 3) * NP, px, py, pz, nc0, nc1, cls, x_is_zero, tid);
  }
  if (!failed) {
    if constexpr (M::CARRY) {   // the last plane has only the last patch's contribution
#pragma unroll
      for (int sx = 0; sx < 2; ++sx) {
        float* dst = x + line_off[sx] + (int64_t)(nc2 - 1) * plane_stride;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float4 o = make_float4(carry[8 * sx + 4 * q], carry[8 * sx + 4 * q + 1], carry[8 * sx + 4 * q + 2],
                                 carry[8 * sx + 4 * q + 3]);
          if (!store_cell[sx]) {
            const float4 old = *reinterpret_cast<const float4*>(dst + 4 * q);
            o.x += old.x;
            o.y += old.y;
            o.z += old.z;
            o.w += old.w;
          }
          *reinterpret_cast<float4*>(dst + 4 * q) = o;
        }
      }
    } else {
      __syncthreads();
      flush_plane<N1>(x, ACC + ((nc2 - 1) & 1) * NP, SB + ((nc2 - 1) % 3) * NP, px, py, nc2 - 1, nc0, nc1, cls,
                      x_is_zero, tid);
    }
  } else if (tid == 0) {
    *fail_flag = 1;
    __threadfence_system();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc05::dealloc(tmem, 32);
}

template <int N, bool TF>
static tpss_status launch(tpss_patches* P, float omega, int nrhs, const float* r, float* x, int x_is_zero,
                          cudaStream_t s) {
  constexpr size_t smem = Smem<N, TF>::BYTES;
  constexpr int BP = Op<TF>::BPOS;
  static bool attr = false;
  if (!attr) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(patch_stream_tc05_kernel<N, TF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const Level& L = P->ctx->levels[P->level];
  const int nc0 = L.nc[0], nc1 = L.nc[1], nc2 = L.nc[2];
  const unsigned char* B0 = static_cast<const unsigned char*>(P->d_bop);
  const unsigned char* B1 = B0 + (size_t)P->npos[0] * BP;
  const unsigned char* B2 = B1 + (size_t)P->npos[1] * BP;
  for (int cls = 0; cls < 4; ++cls) {
    const int ax = cls & 1, ay = cls >> 1;
    const int ncolx = ax <= nc0 - 2 ? (nc0 - 2 - ax) / 2 + 1 : 0;
    const int ncoly = ay <= nc1 - 2 ? (nc1 - 2 - ay) / 2 + 1 : 0;
    if (ncolx == 0 || ncoly == 0) continue;
    dim3 grid((unsigned)(ncolx * ncoly), (unsigned)nrhs);
    patch_stream_tc05_kernel<N, TF><<<grid, kThreads, smem, s>>>(B0, B1, B2, P->d_lam32[0], P->d_lam32[1],
                                                              P->d_lam32[2], r, x, omega, nc0, nc1, nc2, L.ndofs,
                                                              cls, ncolx, x_is_zero, P->d_fail_flag,
                                                              P->expire_test);
    TPSS_CHECK_LAUNCH();
  }
  return TPSS_OK;
}

}  // namespace tcs

// Per-position B operands of the tcgen05 smoother (BF16 or TF32,
// [t][position][Z^T / Z][16 x 16 K-major]) and its failure flag; for BF16
// and TF32 3D vertex patch sets with n <= 16, built once at setup.
tpss_status tc05_prepare(tpss_patches* P) {
  if (P->ctx->dim != 3 || P->kind != TPSS_VERTEX_PATCH || P->per_sub || P->n > 16) return TPSS_OK;
  if (P->precision != TPSS_BF16 && P->precision != TPSS_TF32) return TPSS_OK;
  const bool tf = P->precision == TPSS_TF32;
  const size_t per = 2 * 256;   // elements per position
  const size_t total = per * (P->npos[0] + P->npos[1] + P->npos[2]);
  TPSS_TRY(dalloc(&P->d_bop, total * (tf ? sizeof(float) : sizeof(__nv_bfloat16))));
  size_t off = 0;
  for (int t = 0; t < 3; ++t) {
    const dim3 grid((unsigned)P->npos[t], 2);
    if (tf)
      tcs::prepare_bop_tf32_kernel<<<grid, 256, 0, P->ctx->stream>>>(P->d_Z32[t], P->npos[t], P->n,
                                                                      static_cast<float*>(P->d_bop) + off);
    else
      tcs::prepare_bop_kernel<<<grid, 256, 0, P->ctx->stream>>>(P->d_Z32[t], P->npos[t], P->n,
                                                                 static_cast<__nv_bfloat16*>(P->d_bop) + off);
    TPSS_CHECK_LAUNCH();
    off += per * P->npos[t];
  }
  void* h = nullptr;
  TPSS_CHECK_CUDA(cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped));
  P->h_fail_flag = static_cast<int*>(h);
  *P->h_fail_flag = 0;
  void* d = nullptr;
  TPSS_CHECK_CUDA(cudaHostGetDevicePointer(&d, h, 0));
  P->d_fail_flag = static_cast<int*>(d);
  return TPSS_OK;
}

// The additive pass of the tcgen05 column-streaming schedule (all four
// parity classes); TPSS_EINVAL without launching for shapes it does not
// cover (the same as the COLUMNS schedule); TPSS_ETIMEOUT if a previous
// launch on this patch set gave up waiting for its MMAs.
tpss_status patch_pass_tc05(tpss_patches* P, float omega, int nrhs, const float* r, float* x, int x_is_zero,
                            cudaStream_t s) {
  if (P->ctx->dim != 3 || P->kind != TPSS_VERTEX_PATCH || P->per_sub || P->d_bop == nullptr) return TPSS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(x)) & 15) return TPSS_EINVAL;
  const Level& L = P->ctx->levels[P->level];
  if (L.nc[0] < 2 || L.nc[1] < 2 || L.nc[2] < 2 || nrhs > 65535 || P->n > 16) return TPSS_EINVAL;
  if (*reinterpret_cast<volatile int*>(P->h_fail_flag) != 0) {
    *P->h_fail_flag = 0;
    set_error("tcgen05 smoother: an MMA completion wait expired in an earlier call (its result is invalid)");
    return TPSS_ETIMEOUT;
  }
  struct ClearTest {   // the test hook applies to one call
    tpss_patches* P;
    ~ClearTest() { P->expire_test = 0; }
  } clear_test{P};
  const bool tf = P->precision == TPSS_TF32;
#define TPSS_TC05_CASE(n)                                                                                    \
  case n:                                                                                                    \
    return tf ? tcs::launch<n, true>(P, omega, nrhs, r, x, x_is_zero, s)                                     \
              : tcs::launch<n, false>(P, omega, nrhs, r, x, x_is_zero, s);
  switch (P->n) {
    TPSS_TC05_CASE(4)
    TPSS_TC05_CASE(6)
    TPSS_TC05_CASE(8)
    TPSS_TC05_CASE(10)
    TPSS_TC05_CASE(12)
    TPSS_TC05_CASE(14)
    TPSS_TC05_CASE(16)
    default: return TPSS_EINVAL;
  }
#undef TPSS_TC05_CASE
}

}  // namespace tpss
