// Column-streaming BF16 / TF32 additive vertex-patch smoother on the
// 5th-generation tensor cores (tcgen05 MMA, accumulators in tensor memory);
// 3D, mixed precision (not in the paper).
//
// Schedule: as the COLUMNS schedule (smoother_stream.cu): one CTA per column
// of vertex patches (p_x, p_y) and right-hand side walks p_z, r staged one
// cell plane ahead with cp.async, each cell plane of x written once per
// parity class of (p_x, p_y) when both of its patches in the column are done.
// With two or more right-hand sides, the second half runs on a second stream
// (fork and join by events), so that its class launches fill the SMs that the
// last wave of each class launch of the first half leaves idle.
//
// Local solve (eq. fastinverse, eq. eigenvectormatvec): the six mode
// contractions of (Z_z x Z_y x Z_x) Lambda^{-1} (Z_z x Z_y x Z_x)^T are six
// MMAs D = A B with M = 128 (two blocks of 128 rows), N = 16, K = 16,
// BF16 operands from shared memory, FP32 accumulation in TMEM.  Every index
// is padded to 16 slots, slot 8 c + i for node i < k + 1 of the patch's cell
// c (modes take the same slots, mode j at 8 (j / (k+1)) + j % (k+1)), so the
// patch tensor has 256 "lines" (slow index s, fast index f, row m = 16 s +
// f) and each cell of the patch owns an 8 x 8 x 8 corner of it.  A is the
// tensor with the contracted index as K; B is the 1D eigenvector matrix
// (K-major 16 x 16, zero padded, prepared
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
// The core matrices of A sit 144 bytes apart along M (not 128), and stages 2
// and 5 order their two stores by row group, so that these writes are free
// of shared-memory bank conflicts.  The cell lines of r are staged with the
// two 16-byte halves of every other group of 4 lines swapped (k = 7), which
// makes the gather's reads conflict-free too.
//
// TF32 (kind::tf32, K = 8 per MMA): the same walk with FP32 operands rounded
// to TF32, two MMAs per 16-wide contraction and every operand K-major (a
// core matrix row holds 4 values); the rotated stages write their values to
// the next A one by one instead of as MN-major rows, stages 1 and 4 with
// core-matrix strides that keep those stores conflict-free.
//
// Output: a thread's two rows of D6 (m and m + 128) are the same (y, z) line
// of the patch's lower and upper cell plane; the upper one is kept in
// registers until the next patch of the column adds the lower one of that
// plane, and the finished line (two cell rows of k + 1 values) goes straight
// to x, which is read (for the read-modify-write classes) and written once
// per parity class.
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
// TF32, the operands written one value per row with rows 16 slow + j, k fixed
// per thread (stages 1 and 4): core matrices 160 bytes apart along M and
// 5136 along K, so that a warp's 32 stores (4 k & 3 x 4 k >> 2 x 2 slow) fall
// in 32 distinct banks; the MMAs of stages 2 and 5 read them with these strides
constexpr int kMStrideT = 160;
constexpr int kKStrideT = 32 * kMStrideT + 16;

// per element type: A bytes (2 or 4 core-matrix columns of 8 or 4 values),
// one 16 x 16 B operand, the B operands of one position (Z^T and Z)
template <bool TF> struct Op {
  static constexpr int ABYTES = TF ? 4 * kKStrideT : 2 * kKStride;
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

// node (or mode) of slot sl of a direction with n1 nodes per cell; -1 for padding
__host__ __device__ __forceinline__ int slot_index(int sl, int n1) {
  return (sl & 7) < n1 ? (sl >> 3) * n1 + (sl & 7) : -1;
}

template <int N, bool TF>
struct Smem {
  static constexpr int N1 = N / 2;
  static constexpr int NLOC1 = N1 * N1 * N1;
  static constexpr int NP = 4 * NLOC1;                       // floats of one column plane (4 cells)
  static constexpr size_t OPA = 0;
  static constexpr size_t OPB = Op<TF>::ABYTES;              // 8 operands B
  static constexpr size_t SB = OPB + 8 * Op<TF>::BBYTES;     // 2 staged planes of r (FP32)
  static constexpr size_t BYTES = SB + 2 * (size_t)NP * 4;
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
// 16 x 16 K-major BF16 matrix B[n][k] = Z[k][n] (0) or Z[n][k] (1), Z[node][mode],
// both indices in slots (zero at padding slots).
__global__ void prepare_bop_kernel(const float* __restrict__ Z, int npos, int n, __nv_bfloat16* __restrict__ out) {
  const int p = blockIdx.x, back = blockIdx.y;
  if (p >= npos) return;
  const float* Zp = Z + (size_t)p * n * n;
  __nv_bfloat16* o = out + ((size_t)p * 2 + back) * 256;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int nn = e >> 4, k = e & 15, in = slot_index(nn, n / 2), ik = slot_index(k, n / 2);
    float v = 0.f;
    if (in >= 0 && ik >= 0) v = back ? Zp[in * n + ik] : Zp[ik * n + in];
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
    const int nn = e >> 4, k = e & 15, in = slot_index(nn, n / 2), ik = slot_index(k, n / 2);
    float v = 0.f;
    if (in >= 0 && ik >= 0) v = back ? Zp[in * n + ik] : Zp[ik * n + in];
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
// one value per row of the K-major TF32 operand (strides kMStrideT / kKStrideT
// unless ALT).  ALT: neighbouring threads differ in `slow` (not in k); the
// BF16 threads with bit 2 of slow set write their two 16-byte rows in the
// other order, so that the 8 rows one store instruction writes per quarter
// warp fall in 8 distinct bank groups.
template <bool TF, bool ALT>
__device__ __forceinline__ void put_col(unsigned char* opa, int slow, int k, const float* v) {
  if constexpr (TF) {
    constexpr int MS = ALT ? kMStride : kMStrideT, KS = ALT ? kKStride : kKStrideT;
    unsigned char* base = opa + (k & 3) * 4 + (k >> 2) * KS;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int r = 16 * slow + j;
      *reinterpret_cast<uint32_t*>(base + (r & 7) * 16 + (r >> 3) * MS) = tc05::to_tf32(v[j]);
    }
  } else if constexpr (ALT) {
    const uint4 lo = tc05::pack8(v), hi = tc05::pack8(v + 8);
    const bool swap = (slow >> 2) & 1;
    unsigned char* p = opa + off_mn(slow, k);
    *reinterpret_cast<uint4*>(p + (swap ? kMStride : 0)) = swap ? hi : lo;
    *reinterpret_cast<uint4*>(p + (swap ? 0 : kMStride)) = swap ? lo : hi;
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

// n1 consecutive floats (a cell line; 16-byte aligned when n1 % 4 == 0, 8-byte
// when n1 % 2 == 0) <-> v[0 .. n1)
template <int N1>
__device__ __forceinline__ void ld_line(const float* p, float* v) {
  if constexpr (N1 % 4 == 0) {
#pragma unroll
    for (int q = 0; q < N1 / 4; ++q) {
      const float4 a = reinterpret_cast<const float4*>(p)[q];
      v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
    }
  } else if constexpr (N1 % 2 == 0) {
#pragma unroll
    for (int q = 0; q < N1 / 2; ++q) {
      const float2 a = reinterpret_cast<const float2*>(p)[q];
      v[2 * q] = a.x; v[2 * q + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = p[q];
  }
}
template <int N1>
__device__ __forceinline__ void st_line(float* p, const float* v) {
  if constexpr (N1 % 4 == 0) {
#pragma unroll
    for (int q = 0; q < N1 / 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else if constexpr (N1 % 2 == 0) {
#pragma unroll
    for (int q = 0; q < N1 / 2; ++q) reinterpret_cast<float2*>(p)[q] = make_float2(v[2 * q], v[2 * q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < N1; ++q) p[q] = v[q];
  }
}

template <int N, bool TF>
__global__ void __launch_bounds__(kThreads, TF ? 4 : (N >= 14 ? 5 : 6))   // BF16 k <= 5: 6 CTAs per SM without spills
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
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* opa = dsm + M::OPA;
  unsigned char* opb = dsm + M::OPB;
  float* SB = reinterpret_cast<float*>(dsm + M::SB);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ __align__(16) float lam[64];   // slots of x, y (the column's), z of patch p_z at 32 + 16 (p_z & 1)
  const int tid = threadIdx.x, warp = tid >> 5;
  const int px = (cls & 1) + 2 * (int)(blockIdx.x % ncolx);
  const int py = (cls >> 1) + 2 * (int)(blockIdx.x / ncolx);
  r += (int64_t)blockIdx.y * ndofs;
  x += (int64_t)blockIdx.y * ndofs;
  const uint32_t mb = tc05::smem_u32(&mbar);

  const int64_t plane_stride = (int64_t)nc0 * nc1 * NLOC1;
  // k = 7 plane staging: thread t copies 16 bytes at float 4 t of each of the 4
  // cells (half t & 1 of cell line t / 2); the two halves of the lines with
  // bit 2 of y set trade places in shared memory, so that the gather's 16-byte
  // reads of 8 lines hit 8 distinct bank groups
  int64_t stage_off[4];
#pragma unroll
  for (int c2 = 0; c2 < 4; ++c2) stage_off[c2] = ((px + (c2 & 1)) + (int64_t)nc0 * (py + (c2 >> 1))) * NLOC1 + 4 * tid;
  const uint32_t stage_dst = 16u * ((tid & ~1) | ((tid & 1) ^ ((tid >> 3) & 1)));
  auto stage_r = [&](int cz) {   // cell plane cz of r -> ring slot cz % 2
    if constexpr (NLOC1 == 4 * kThreads) {
      const uint32_t d = tc05::smem_u32(SB + (cz % 2) * NP) + stage_dst;
      const float* src = r + (int64_t)cz * plane_stride;
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) cp16(d + 4u * NLOC1 * c2, src + stage_off[c2]);
    } else {
      stage_plane<NLOC1>(SB + (cz % 2) * NP, r, px, py, cz, nc0, nc1, tid);
    }
  };

  // prologue: planes 0 and 1, the column's x and y operands, patch 0's z operands
  stage_r(0);
  stage_r(1);
  stage_b2<TF>(opb + 0 * BB, B0 + (size_t)px * BP, tid);   // slots 0, 1
  stage_b2<TF>(opb + 2 * BB, B1 + (size_t)py * BP, tid);   // slots 2, 3
  stage_b2<TF>(opb + 4 * BB, B2, tid);                     // patch 0: slots 4, 5
  if (tid < 16 && (tid & 7) < N1)                          // patch 0's z eigenvalues
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(tc05::smem_u32(lam + 32 + tid)),
                 "l"(L2 + slot_index(tid, N1)) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int e = tid; e < Op<TF>::ABYTES / 16; e += kThreads) reinterpret_cast<uint4*>(opa)[e] = make_uint4(0, 0, 0, 0);
  if (tid < 32) {
    const int sl = tid & 15, i = slot_index(sl, N1);
    lam[tid] = i < 0 ? 0.f : (tid < 16 ? L0[(size_t)px * N + i] : L1[(size_t)py * N + i]);
  } else if (tid < 64 && ((tid & 7) >= N1)) {
    lam[tid] = 0.f;   // z padding slots (never written by the copies)
  }
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

  // this thread's line: y slot tid & 15 (cell row sy, node iy), z node iz =
  // tid >> 4 of the lower (rows m = tid) and upper (m = tid + 128) cell plane,
  // in the two cells sx = 0, 1 at (p_x + sx, p_y + sy)
  const int ly = tid & 15, iz = tid >> 4, sy = ly >> 3, iy = ly & 7;
  const bool line = iy < N1 && iz < N1;
  const int lofs = N1 * (iy + N1 * iz);   // the line's offset inside a cell
  float carry[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) carry[j] = 0.f;
  bool store_cell[2];
  int64_t line_off[2];
#pragma unroll
  for (int sx = 0; sx < 2; ++sx) {
    const int cx = px + sx, cy = py + sy;
    store_cell[sx] = x_is_zero && first_class(cx, cy, nc0, nc1) == cls;
    line_off[sx] = (cx + (int64_t)nc0 * cy) * NLOC1 + lofs;
  }

  for (int pz = 0; pz + 1 < nc2 && !failed; ++pz) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();   // planes pz, pz + 1 and patch pz's z operands staged; patch pz - 1 is done
    if (pz + 2 < nc2) {
      stage_b2<TF>(opb + (4 + 2 * ((pz + 1) & 1)) * BB, B2 + (size_t)(pz + 1) * BP, tid);
      if (tid < 16 && (tid & 7) < N1)   // the next patch's z eigenvalues
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                     :: "r"(tc05::smem_u32(lam + 32 + 16 * ((pz + 1) & 1) + tid)),
                        "l"(L2 + (size_t)(pz + 1) * N + slot_index(tid, N1)) : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const float* lamz = lam + 32 + 16 * (pz & 1);
    // previous values of this thread's line of plane pz (read-modify-write cells)
    float xold[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) xold[j] = 0.f;
    if (line) {
#pragma unroll
      for (int sx = 0; sx < 2; ++sx)
        if (!store_cell[sx]) ld_line<N1>(x + line_off[sx] + pz * plane_stride, xold + 8 * sx);
    }
    // gather: A0[(z, y)][x] (K-major), zero outside the cells' nodes
    const float* lo = SB + (pz % 2) * NP;
    const float* hi = SB + ((pz + 1) % 2) * NP;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
      if (line) {
        const float* src = (b ? hi : lo) + 2 * sy * NLOC1 + lofs;
        if constexpr (NLOC1 == 4 * kThreads) {   // halves swapped for lines with iy & 4
          const int sw = (iy >> 2) & 1;
#pragma unroll
          for (int sx = 0; sx < 2; ++sx)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float4 a = *reinterpret_cast<const float4*>(src + sx * NLOC1 + 4 * (h ^ sw));
              v[8 * sx + 4 * h] = a.x; v[8 * sx + 4 * h + 1] = a.y;
              v[8 * sx + 4 * h + 2] = a.z; v[8 * sx + 4 * h + 3] = a.w;
            }
        } else {
#pragma unroll
          for (int sx = 0; sx < 2; ++sx) ld_line<N1>(src + sx * NLOC1, v + 8 * sx);
        }
      }
      put_row_k<TF>(opa, tid + 128 * b, v);
    }
    tc05::fence_proxy_async();
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    if (pz + 2 < nc2) {   // plane pz is gathered: its slot takes plane pz + 2
      stage_r(pz + 2);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }

#pragma unroll
    for (int s = 1; s <= 6; ++s) {   // unrolled: every stage's index rotation is resolved at compile time
      if (tid == 0) {
        const uint32_t bslot = b_base + BB * b_slot(s, pz & 1);
        if constexpr (TF) {   // K = 16 as two MMAs of K = 8 (core-matrix columns 2h, 2h + 1)
          constexpr uint32_t idesc = tc05::idesc_tf32(128, 16);
          // A of stages 2 and 5 was written with the strides kMStrideT / kKStrideT
          const int ms = (s == 2 || s == 5) ? kMStrideT : kMStride, ks = (s == 2 || s == 5) ? kKStrideT : kKStride;
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              tc05::mma_tf32(tmem + 16 * b, tc05::desc(a_base + 16 * ms * b + 2 * h * ks, ks, ms),
                             tc05::desc(bslot + 512 * h, 256, 128), idesc, h);
        } else {
          const uint32_t idesc = tc05::idesc_bf16(128, 16, a_major(s), 0);
          const uint64_t bdesc = tc05::desc(bslot, 256, 128);
#pragma unroll
          for (int b = 0; b < 2; ++b)
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
      float v[32];
      tc05::ld32(trow, v);
      if (s == 6) {
        // rows: block 0 = the line of plane pz (lower cells), block 1 = plane pz + 1
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          xold[j] += carry[j] + omega * v[j];
          carry[j] = omega * v[16 + j];
        }
        if (line) {
#pragma unroll
          for (int sx = 0; sx < 2; ++sx) st_line<N1>(x + line_off[sx] + pz * plane_stride, xold + 8 * sx);
        }
      } else {
        float lz[16];   // z eigenvalues of this patch (s == 3), four 16-byte reads
        if (s == 3) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 a = reinterpret_cast<const float4*>(lamz)[q];
            lz[4 * q] = a.x; lz[4 * q + 1] = a.y; lz[4 * q + 2] = a.z; lz[4 * q + 3] = a.w;
          }
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int m = tid + 128 * b, sl = m >> 4, fa = m & 15;
          float* w = v + 16 * b;
          if (s == 1 || s == 4) {          // D1[(z,y)][a] -> A1[(z,a)][y];  D4[(a,b)][z] -> A4[(a,z)][b]
            put_col<TF, false>(opa, sl, fa, w);
          } else if (s == 2 || s == 5) {   // D2[(z,a)][b] -> A2[(a,b)][z];  D5[(a,z)][y] -> A5[(z,y)][a]
            put_col<TF, true>(opa, fa, sl, w);
          } else {                         // D3[(a,b)][c] / (lx_a + ly_b + lz_c) -> A3[(a,b)][c]
            const float sab = lam[sl] + lam[16 + fa];
            const bool ab = (sl & 7) < N1 && (fa & 7) < N1;
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = (ab && (j & 7) < N1) ? __fdividef(w[j], sab + lz[j]) : 0.f;
            put_row_k<TF>(opa, m, w);
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
  }
  if (!failed) {
    // the last plane has only the last patch's contribution
    if (line) {
#pragma unroll
      for (int sx = 0; sx < 2; ++sx) {
        float* dst = x + line_off[sx] + (int64_t)(nc2 - 1) * plane_stride;
        float o[8];
        if (!store_cell[sx]) ld_line<N1>(dst, o);
#pragma unroll
        for (int j = 0; j < N1; ++j) o[j] = store_cell[sx] ? carry[8 * sx + j] : o[j] + carry[8 * sx + j];
        st_line<N1>(dst, o);
      }
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
  // Two or more right-hand sides: the second half goes to a second stream, so
  // that its class launches fill the SMs left idle by the last wave of each
  // class launch of the first half (the halves share no data).
  const int halves = (nrhs >= 2 && P->aux_stream != nullptr) ? 2 : 1;
  if (halves == 2) {
    TPSS_CHECK_CUDA(cudaEventRecord(P->fork_event, s));
    TPSS_CHECK_CUDA(cudaStreamWaitEvent(P->aux_stream, P->fork_event, 0));
  }
  for (int cls = 0; cls < 4; ++cls) {
    const int ax = cls & 1, ay = cls >> 1;
    const int ncolx = ax <= nc0 - 2 ? (nc0 - 2 - ax) / 2 + 1 : 0;
    const int ncoly = ay <= nc1 - 2 ? (nc1 - 2 - ay) / 2 + 1 : 0;
    if (ncolx == 0 || ncoly == 0) continue;
    for (int h = 0; h < halves; ++h) {
      const int r0 = h == 0 ? 0 : nrhs / 2, nr = halves == 1 ? nrhs : (h == 0 ? nrhs / 2 : nrhs - nrhs / 2);
      const int64_t off = (int64_t)r0 * L.ndofs;
      dim3 grid((unsigned)(ncolx * ncoly), (unsigned)nr);
      patch_stream_tc05_kernel<N, TF><<<grid, kThreads, smem, h == 0 ? s : P->aux_stream>>>(
          B0, B1, B2, P->d_lam32[0], P->d_lam32[1], P->d_lam32[2], r + off, x + off, omega, nc0, nc1, nc2, L.ndofs,
          cls, ncolx, x_is_zero, P->d_fail_flag, P->expire_test);
      TPSS_CHECK_LAUNCH();
    }
  }
  if (halves == 2) {
    TPSS_CHECK_CUDA(cudaEventRecord(P->join_event, P->aux_stream));
    TPSS_CHECK_CUDA(cudaStreamWaitEvent(s, P->join_event, 0));
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
