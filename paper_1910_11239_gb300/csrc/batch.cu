// Batched multigrid for many independent problems of uneven size and degree
// (not in the paper).
//
// A batch holds one context per problem (3D, vertex-patch additive smoother,
// V-cycle in FP32 inside an FP64 outer PCG) and nrhs right-hand sides per
// problem.  Levels are aligned from the finest one ("depth" 0); at every depth
// ONE persistent kernel smooths all problems and all right-hand sides that
// have a smoothing level there: CTAs pull work items (problem, rhs, group of
// patches of one degree) from an atomic counter, dispatch on the patch size n
// to a templated fast-diagonalization routine (gather, Z^T, Lambda^{-1}, Z)
// and scatter with FP32 atomic adds (overlapping patches of one problem may
// be processed concurrently; FP32 summation order is therefore not fixed).
// In BF16 batches every level leaves the persistent kernel: each problem's
// additive pass runs the library's deterministic per-problem smoother (the
// tcgen05 column walk for k >= 4, the colored BF16 launches below) on one of
// a few side streams, so the problems' launches overlap.
// Work items are sorted by cost, largest first.  The number of patches per
// work item is chosen per n by an autotuner that times the candidates at
// setup.  Operators, transfers and coarse solves are launched per problem
// (batched over right-hand sides), and the whole V-cycle is captured once
// into a CUDA graph that every preconditioner application replays.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "bf16_tc.cuh"
#include "tpss_internal.cuh"

namespace tpss {

template <typename T>
tpss_status smooth_additive_t(tpss_patches* P, T omega, int nrhs, const T* b, T* x, int x_is_zero);

struct BatchLevelDesc {
  const float* Z[3];
  const float* lam[3];
  const int* list;     // all patches of the level (packed positions)
  const float* r;      // nrhs vectors of ndofs
  float* x;
  int nc0, nc1;
  int64_t ndofs;
  int n;
  int variant;         // local solver routine: 0 FP32 SIMT, 1 BF16 tensor cores
};

struct BatchItem {
  int prob, first, count, rhs;
};

constexpr int kBatchThreads = 256;

template <int N>
struct BShape {
  static constexpr int LINES = N * N;
  static constexpr int LS = (N % 2 == 0) ? N + 1 : N;
  static constexpr int PS = LS * N;
  static constexpr int VOL = PS * N;
  static constexpr int SLOT = VOL + 6 * N * N + 3 * N;
};

inline int bshape_slot(int n) {
  const int ls = (n % 2 == 0) ? n + 1 : n;
  return ls * n * n + 6 * n * n + 3 * n;
}

template <int N>
__device__ void batch_group(const BatchLevelDesc& D, const BatchItem& it, float omega, float* smem) {
  using S = BShape<N>;
  constexpr int N1 = N / 2;
  constexpr int NLOC1 = N1 * N1 * N1;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int cnt = it.count;
  const int64_t vbase = (int64_t)it.rhs * D.ndofs;
  // per patch: load Z, Z^T, lambda, gather 8 cells
  for (int e = tid; e < cnt * 3 * N * N; e += nth) {
    const int c = e / (3 * N * N), rem = e % (3 * N * N);
    const int t = rem / (N * N), i = rem % (N * N);
    const int packed = D.list[it.first + c];
    const int pos = t == 0 ? unpack_x(packed) : (t == 1 ? unpack_y(packed) : unpack_z(packed));
    const float z = D.Z[t][(size_t)pos * N * N + i];
    float* slot = smem + c * S::SLOT;
    slot[S::VOL + t * N * N + i] = z;
    slot[S::VOL + 3 * N * N + t * N * N + (i % N) * N + i / N] = z;
  }
  for (int e = tid; e < cnt * 3 * N; e += nth) {
    const int c = e / (3 * N), rem = e % (3 * N), t = rem / N, i = rem % N;
    const int packed = D.list[it.first + c];
    const int pos = t == 0 ? unpack_x(packed) : (t == 1 ? unpack_y(packed) : unpack_z(packed));
    smem[c * S::SLOT + S::VOL + 6 * N * N + rem] = D.lam[t][(size_t)pos * N + i];
  }
  for (int e = tid; e < cnt * 8 * NLOC1; e += nth) {
    const int c = e / (8 * NLOC1), rem = e % (8 * NLOC1);
    const int cell = rem / NLOC1, loc = rem % NLOC1;
    const int packed = D.list[it.first + c];
    const int px = unpack_x(packed), py = unpack_y(packed), pz = unpack_z(packed);
    const int sx = cell & 1, sy = (cell >> 1) & 1, sz = (cell >> 2) & 1;
    const int ix = loc % N1, iy = (loc / N1) % N1, iz = loc / (N1 * N1);
    const int64_t gcell = (px + sx) + (int64_t)D.nc0 * ((py + sy) + (int64_t)D.nc1 * (pz + sz));
    smem[c * S::SLOT + (sx * N1 + ix) + S::LS * (sy * N1 + iy) + S::PS * (sz * N1 + iz)] =
        D.r[vbase + gcell * NLOC1 + loc];
  }
  __syncthreads();
  auto geom = [](int t, int line, int& base, int& stride) {
    const int a = line % N, b = line / N;
    if (t == 0) { base = S::LS * a + S::PS * b; stride = 1; }
    else if (t == 1) { base = a + S::PS * b; stride = S::LS; }
    else { base = a + S::LS * b; stride = S::PS; }
  };
  // Z^T along x, y
  for (int t = 0; t < 2; ++t) {
    for (int lg = tid; lg < cnt * S::LINES; lg += nth) {
      float* slot = smem + (lg / S::LINES) * S::SLOT;
      int base, stride;
      geom(t, lg % S::LINES, base, stride);
      const float* W = slot + S::VOL + t * N * N;
      float acc[N];
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] = 0.f;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const float v = slot[base + m * stride];
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = fmaf(W[m * N + i], v, acc[i]);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) slot[base + i * stride] = acc[i];
    }
    __syncthreads();
  }
  // z: Z^T, Lambda^{-1}, Z fused
  for (int lg = tid; lg < cnt * S::LINES; lg += nth) {
    float* slot = smem + (lg / S::LINES) * S::SLOT;
    const int line = lg % S::LINES;
    int base, stride;
    geom(2, line, base, stride);
    const float* W = slot + S::VOL + 2 * N * N;
    const float* WT = slot + S::VOL + 3 * N * N + 2 * N * N;
    const float* lam = slot + S::VOL + 6 * N * N;
    float acc[N];
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = 0.f;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const float v = slot[base + m * stride];
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] = fmaf(W[m * N + i], v, acc[i]);
    }
    const float s0 = lam[line % N] + lam[N + line / N];
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = acc[i] / (s0 + lam[2 * N + i]);
    float out[N];
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = 0.f;
#pragma unroll
    for (int m = 0; m < N; ++m) {
#pragma unroll
      for (int i = 0; i < N; ++i) out[i] = fmaf(WT[m * N + i], acc[m], out[i]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) slot[base + i * stride] = out[i];
  }
  __syncthreads();
  // Z along y, x
  for (int t = 1; t >= 0; --t) {
    for (int lg = tid; lg < cnt * S::LINES; lg += nth) {
      float* slot = smem + (lg / S::LINES) * S::SLOT;
      int base, stride;
      geom(t, lg % S::LINES, base, stride);
      const float* W = slot + S::VOL + 3 * N * N + t * N * N;
      float acc[N];
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] = 0.f;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const float v = slot[base + m * stride];
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = fmaf(W[m * N + i], v, acc[i]);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) slot[base + i * stride] = acc[i];
    }
    __syncthreads();
  }
  // scatter with atomics (patches of one problem overlap)
  for (int e = tid; e < cnt * 8 * NLOC1; e += nth) {
    const int c = e / (8 * NLOC1), rem = e % (8 * NLOC1);
    const int cell = rem / NLOC1, loc = rem % NLOC1;
    const int packed = D.list[it.first + c];
    const int px = unpack_x(packed), py = unpack_y(packed), pz = unpack_z(packed);
    const int sx = cell & 1, sy = (cell >> 1) & 1, sz = (cell >> 2) & 1;
    const int ix = loc % N1, iy = (loc / N1) % N1, iz = loc / (N1 * N1);
    const int64_t gcell = (px + sx) + (int64_t)D.nc0 * ((py + sy) + (int64_t)D.nc1 * (pz + sz));
    const float v = smem[c * S::SLOT + (sx * N1 + ix) + S::LS * (sy * N1 + iy) + S::PS * (sz * N1 + iz)];
    atomicAdd(D.x + vbase + gcell * NLOC1 + loc, omega * v);
  }
  __syncthreads();
}

// BF16 tensor-core variant of a work item: `count` patches of one problem and
// right-hand side, one after another, with the routines of bf16_tc.cuh.  The
// right-hand side of the next patch is staged by cp.async (double buffer)
// while the current one is contracted; the scatter uses FP32 atomics.
// Dynamic shared memory: [T: Shape<16> bf16][SB: 2 x 8 NLOC1(16) f32].
constexpr int kBf16SbOffset = ((bf::Shape<16>::TOTAL * 2 + 15) / 16) * 16;
constexpr size_t kBf16Smem = kBf16SbOffset + 2 * 8 * 512 * sizeof(float);

template <int N>
__device__ void batch_group_bf16(const BatchLevelDesc& D, const BatchItem& it, float omega, unsigned char* dsm,
                                 float* lam) {
  using S = bf::Shape<N>;
  constexpr int N1 = N / 2;
  constexpr int NLOC1 = N1 * N1 * N1;
  constexpr int NV = 8 * NLOC1;
  __nv_bfloat16* T = reinterpret_cast<__nv_bfloat16*>(dsm);
  float* SB = reinterpret_cast<float*>(dsm + kBf16SbOffset);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const float* rb = D.r + (int64_t)it.rhs * D.ndofs;
  float* xb = D.x + (int64_t)it.rhs * D.ndofs;
  auto cellbase = [&](int c) -> bf::CellBase {
    const int packed = D.list[it.first + c];
    return bf::CellBase{unpack_x(packed), unpack_y(packed), unpack_z(packed), D.nc0, D.nc1};
  };
  __syncthreads();   // the previous item is done with T and SB
  for (int e = tid; e < S::TOTAL; e += blockDim.x) T[e] = __float2bfloat16(0.f);
  bf::stage<NLOC1, 8>(SB, rb, cellbase(0), tid);
  bf::cp_async_commit();
  for (int c = 0; c < it.count; ++c) {
    const bf::CellBase cb = cellbase(c);
    bf::cp_async_wait_all();
    __syncthreads();   // staged data visible; zero fill / previous patch done with T
    if (tid < 3 * N) {
      const int d = tid / N, i = tid % N;
      lam[tid] = D.lam[d][(size_t)(d == 0 ? cb.px : (d == 1 ? cb.py : cb.pz)) * N + i];
    }
    bf::rows_to_tensor<N, N1, 8>(T, SB + (c & 1) * NV, tid);
    uint32_t bx[2][2], bxt[2][2], by[2][2], byt[2][2], bzz[2][2], bzt[2][2];
    bf::load_bfrag<N, false>(bxt, D.Z[0] + (size_t)cb.px * N * N, lane);
    bf::load_bfrag<N, true>(bx, D.Z[0] + (size_t)cb.px * N * N, lane);
    bf::load_bfrag<N, false>(byt, D.Z[1] + (size_t)cb.py * N * N, lane);
    bf::load_bfrag<N, true>(by, D.Z[1] + (size_t)cb.py * N * N, lane);
    bf::load_bfrag<N, false>(bzt, D.Z[2] + (size_t)cb.pz * N * N, lane);
    bf::load_bfrag<N, true>(bzz, D.Z[2] + (size_t)cb.pz * N * N, lane);
    __syncthreads();   // T and lam ready; the other SB buffer is free
    if (c + 1 < it.count) {
      bf::stage<NLOC1, 8>(SB + ((c + 1) & 1) * NV, rb, cellbase(c + 1), tid);
      bf::cp_async_commit();
    }
    bf::contract<N, 0>(T, bxt, warp, lane);
    __syncthreads();
    bf::contract<N, 1>(T, byt, warp, lane);
    __syncthreads();
    bf::zstep<N>(T, bzt, bzz, lam, warp, lane);
    __syncthreads();
    bf::contract<N, 1>(T, by, warp, lane);
    __syncthreads();
    bf::contract<N, 0>(T, bx, warp, lane);
    __syncthreads();
    bf::tensor_atomic_add<N, N1, 8>(xb, T, omega, cb, tid);
  }
}

// FP32-only persistent smoother (batches without BF16): a separate kernel so
// that its register allocation is not set by the tensor-core routines.
__global__ void __launch_bounds__(kBatchThreads)
batch_smooth_simt_kernel(const BatchLevelDesc* __restrict__ desc, const BatchItem* __restrict__ items, int nitems,
                         int* __restrict__ counter, float omega) {
  extern __shared__ __align__(16) unsigned char bdsm[];
  __shared__ int cur;
  float* fsm = reinterpret_cast<float*>(bdsm);
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int i = cur;
    __syncthreads();
    if (i >= nitems) break;
    const BatchItem it = items[i];
    const BatchLevelDesc D = desc[it.prob];
    switch (D.n) {
      case 4: batch_group<4>(D, it, omega, fsm); break;
      case 6: batch_group<6>(D, it, omega, fsm); break;
      case 8: batch_group<8>(D, it, omega, fsm); break;
      case 10: batch_group<10>(D, it, omega, fsm); break;
      case 12: batch_group<12>(D, it, omega, fsm); break;
      case 14: batch_group<14>(D, it, omega, fsm); break;
      case 16: batch_group<16>(D, it, omega, fsm); break;
      default: break;
    }
  }
}

// The persistent smoother with both routines: every CTA pulls work items
// until the list is exhausted and runs the routine chosen for the item's
// patch size.
__global__ void __launch_bounds__(kBatchThreads)
batch_smooth_kernel(const BatchLevelDesc* __restrict__ desc, const BatchItem* __restrict__ items, int nitems,
                    int* __restrict__ counter, float omega) {
  extern __shared__ __align__(16) unsigned char bdsm[];
  __shared__ float lam[3 * 16];
  __shared__ int cur;
  float* fsm = reinterpret_cast<float*>(bdsm);
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int i = cur;
    __syncthreads();
    if (i >= nitems) break;
    const BatchItem it = items[i];
    const BatchLevelDesc D = desc[it.prob];
    if (D.variant == 1) {
      switch (D.n) {
        case 4: batch_group_bf16<4>(D, it, omega, bdsm, lam); break;
        case 6: batch_group_bf16<6>(D, it, omega, bdsm, lam); break;
        case 8: batch_group_bf16<8>(D, it, omega, bdsm, lam); break;
        case 10: batch_group_bf16<10>(D, it, omega, bdsm, lam); break;
        case 12: batch_group_bf16<12>(D, it, omega, bdsm, lam); break;
        case 14: batch_group_bf16<14>(D, it, omega, bdsm, lam); break;
        case 16: batch_group_bf16<16>(D, it, omega, bdsm, lam); break;
        default: break;
      }
    } else {
      switch (D.n) {
        case 4: batch_group<4>(D, it, omega, fsm); break;
        case 6: batch_group<6>(D, it, omega, fsm); break;
        case 8: batch_group<8>(D, it, omega, fsm); break;
        case 10: batch_group<10>(D, it, omega, fsm); break;
        case 12: batch_group<12>(D, it, omega, fsm); break;
        case 14: batch_group<14>(D, it, omega, fsm); break;
        case 16: batch_group<16>(D, it, omega, fsm); break;
        default: break;
      }
    }
  }
}

// y_r = Ainv b_r for nrhs vectors (FP64 inverse, FP32 vectors), one warp per row
// (four right-hand sides per warp and row: the row of A is read once for them)
__global__ void batch_dense_mv_kernel(const double* __restrict__ A, const float* __restrict__ b, float* __restrict__ y,
                                      int64_t n, int nrhs) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (row >= n) return;
  const int r0 = 4 * blockIdx.y, nr = nrhs - r0 < 4 ? nrhs - r0 : 4;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t c = lane; c < n; c += 32) {
    const double a = A[row * n + c];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nr) s[q] = fma(a, (double)b[(int64_t)(r0 + q) * n + c], s[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0 && q < nr) y[(int64_t)(r0 + q) * n + row] = (float)s[q];
  }
}

// ------------------------------------------------------------ segmented CG
__global__ void seg_dot_kernel(const double* __restrict__ x, const double* __restrict__ y,
                               const int64_t* __restrict__ off, const int64_t* __restrict__ len,
                               double* __restrict__ partials, int chunks) {
  const int s = blockIdx.y;
  const int64_t o = off[s], n = len[s];
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v = fma(x[o + i], y[o + i], v);
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
  __shared__ double ws[32];
  if (threadIdx.x % 32 == 0) ws[threadIdx.x / 32] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < blockDim.x / 32 ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
    if (threadIdx.x == 0) partials[(int64_t)s * chunks + blockIdx.x] = v;
  }
}

__global__ void seg_dot_final_kernel(const double* __restrict__ partials, int chunks, double* __restrict__ out) {
  const int s = blockIdx.x;
  double v = 0.0;
  for (int i = threadIdx.x; i < chunks; i += blockDim.x) v += partials[(int64_t)s * chunks + i];
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
  __shared__ double ws[32];
  if (threadIdx.x % 32 == 0) ws[threadIdx.x / 32] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < blockDim.x / 32 ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
    if (threadIdx.x == 0) out[s] = v;
  }
}

// per-system scalars, column-major [field][S]: 0 rz, 1 pq, 2 rr, 3 rz_new, 4 r.zold, 5 active
__global__ void seg_xr_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                              const double* __restrict__ q, const int64_t* __restrict__ off,
                              const int64_t* __restrict__ len, const double* __restrict__ sc, int S) {
  const int s = blockIdx.y;
  if (sc[5 * S + s] == 0.0) return;
  const double alpha = sc[0 * S + s] / sc[1 * S + s];
  const int64_t o = off[s], n = len[s];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[o + i] = fma(alpha, p[o + i], x[o + i]);
    r[o + i] = fma(-alpha, q[o + i], r[o + i]);
  }
}

__global__ void seg_p_kernel(double* __restrict__ p, const double* __restrict__ z, const int64_t* __restrict__ off,
                             const int64_t* __restrict__ len, const double* __restrict__ sc, int S, int flexible) {
  const int s = blockIdx.y;
  if (sc[5 * S + s] == 0.0) return;
  const double beta = (sc[3 * S + s] - (flexible ? sc[4 * S + s] : 0.0)) / sc[0 * S + s];
  const int64_t o = off[s], n = len[s];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[o + i] = fma(beta, p[o + i], z[o + i]);
}

__global__ void seg_shift_kernel(double* sc, int S) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S && sc[5 * S + s] != 0.0) sc[0 * S + s] = sc[3 * S + s];
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f32_to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

}  // namespace tpss

using namespace tpss;

struct BatchProb {
  tpss_ctx* ctx = nullptr;
  int L = 0;                          // finest level
  std::vector<char> route;            // per level: 0 persistent kernel, 1 tcgen05 columns, 2 colored launches
  int64_t off = 0;                    // offset of the problem's block (nrhs vectors) in concatenated vectors
  std::vector<float*> b, x, r;        // per level, nrhs vectors (finest b/x point into the concatenated buffers)
};

struct tpss_batch {
  std::vector<BatchProb> probs;
  int nrhs = 1;
  int nsys = 0;
  int maxdepth = 0;                   // max over problems of L
  float omega = 0.125f;
  int flexible = 1;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t total = 0;                  // concatenated finest length (all problems, all rhs)
  float* fb = nullptr;                // finest b (FP32, concatenated)
  float* fx = nullptr;                // finest x (FP32, concatenated)
  // per depth: device level descriptors (indexed by problem) and work items
  std::vector<BatchLevelDesc*> d_desc;
  std::vector<BatchLevelDesc*> d_desc_post;   // same, reading the residual buffers
  std::vector<BatchItem*> d_items;
  BatchLevelDesc* d_desc_fin = nullptr;       // finest level, caller's vectors (tpss_batch_smooth_additive)
  std::vector<BatchLevelDesc> h_desc_fin;
  std::vector<int> nitems;
  std::vector<size_t> smem;
  std::vector<int> grid;                      // persistent grid size per depth
  int* d_counter = nullptr;           // one counter per depth and phase (2 * maxdepth + 1)
  int ppb[17] = {0};                  // patches per work item, by n (autotuned)
  int variant[17] = {0};              // local solver routine by n: 0 FP32 SIMT, 1 BF16 (autotuned)
  // graph of the FP32 V-cycle (input fb, output fx)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int use_graph = 1;
  int bf16 = 0;                       // 1: BF16 tensor-core persistent smoother
  int columns = 1;                    // BF16: k >= 4 levels on the tcgen05 column smoother (flags & 4 clears)
  // side streams of the tcgen05 column smoother passes (fork / join events)
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_join;
  cudaEvent_t side_fork = nullptr;
  // CG state (FP64, concatenated)
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *zold = nullptr;
  int64_t* d_off = nullptr;
  int64_t* d_len = nullptr;
  std::vector<int64_t> off, len;
  double* sc = nullptr;               // 6 * nsys
  double* partials = nullptr;
  int chunks = 0;
};

namespace tpss {

static tpss_status build_items(tpss_batch* B, int depth, std::vector<BatchItem>& items, size_t& smem_bytes,
                               int only_n = 0, int ppb_override = 0, int variant_override = -1) {
  items.clear();
  smem_bytes = 0;
  struct Cost {
    double c;
    BatchItem it;
  };
  std::vector<Cost> tmp;
  for (int p = 0; p < (int)B->probs.size(); ++p) {
    const BatchProb& bp = B->probs[p];
    const int l = bp.L - depth;
    if (l < 1 || bp.route[l]) continue;
    tpss_patches* P = bp.ctx->mg->patches[l];
    const int n = P->n;
    if (only_n && n != only_n) continue;
    const int g = ppb_override ? ppb_override : B->ppb[n];
    const int total = (int)P->nsub;
    const int var = variant_override >= 0 ? variant_override : B->variant[n];
    smem_bytes = std::max(smem_bytes, var == 1 ? kBf16Smem : (size_t)g * bshape_slot(n) * sizeof(float));
    for (int r = 0; r < B->nrhs; ++r)
      for (int f = 0; f < total; f += g) {
        const int cnt = std::min(g, total - f);
        tmp.push_back({(double)cnt * std::pow((double)n, 4.0), BatchItem{p, f, cnt, r}});
      }
  }
  std::stable_sort(tmp.begin(), tmp.end(), [](const Cost& a, const Cost& b) { return a.c > b.c; });
  for (auto& c : tmp) items.push_back(c.it);
  return TPSS_OK;
}

static tpss_status grid_size(tpss_batch* B, int nitems, size_t smem, int* grid) {
  int per_sm = 0;
  if (B->bf16)
    TPSS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_smooth_kernel, kBatchThreads, smem));
  else
    TPSS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_smooth_simt_kernel, kBatchThreads,
                                                                  smem));
  if (per_sm < 1) {
    set_error("batch smoother: work item does not fit on an SM");
    return TPSS_EINVAL;
  }
  *grid = std::max(1, std::min(nitems, per_sm * B->num_sms));
  return TPSS_OK;
}

static tpss_status launch_level(tpss_batch* B, const BatchLevelDesc* desc, const BatchItem* items, int nitems,
                                size_t smem, int grid, int* counter, cudaStream_t s) {
  if (nitems == 0) return TPSS_OK;
  TPSS_CHECK_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
  if (B->bf16)
    batch_smooth_kernel<<<grid, kBatchThreads, smem, s>>>(desc, items, nitems, counter, B->omega);
  else
    batch_smooth_simt_kernel<<<grid, kBatchThreads, smem, s>>>(desc, items, nitems, counter, B->omega);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// The additive passes of the problems whose level at this depth leaves the
// persistent kernel (route 1: tcgen05 column smoother, 2: colored launches),
// x += omega sum_j R_j^T A_j^{-1} R_j r (x_is_zero: x holds zeros), spread
// over the side streams after a fork from the batch
// stream; side_join makes the batch stream wait for them (issue the
// persistent launch in between).  fin: the finest level with the caller's
// vectors.  *forked: whether a join is due.
static tpss_status side_passes(tpss_batch* B, int depth, bool post, int x_is_zero, bool* forked,
                               const float* fin_b = nullptr, float* fin_x = nullptr) {
  *forked = false;
  bool any = false;
  for (const BatchProb& bp : B->probs) {
    const int l = bp.L - depth;
    any = any || (l >= 1 && bp.route[l]);
  }
  if (!any) return TPSS_OK;
  const int K = (int)B->side.size();
  *forked = true;
  TPSS_CHECK_CUDA(cudaEventRecord(B->side_fork, B->stream));
  for (int k = 0; k < K; ++k) TPSS_CHECK_CUDA(cudaStreamWaitEvent(B->side[k], B->side_fork, 0));
  int next = 0;
  for (const BatchProb& bp : B->probs) {
    const int l = bp.L - depth;
    if (l < 1 || !bp.route[l]) continue;
    tpss_patches* P = bp.ctx->mg->patches[l];
    const float* r = fin_b ? fin_b + bp.off : (post ? bp.r[l] : bp.b[l]);
    float* x = fin_x ? fin_x + bp.off : bp.x[l];
    if (bp.route[l] == 1) {
      TPSS_TRY(patch_pass_tc05(P, B->omega, B->nrhs, r, x, x_is_zero, B->side[next]));
    } else {   // one launch per color; x holds zeros or the current iterate
      for (size_t c = 0; c + 1 < P->add_offsets.size(); ++c) {
        const int o = P->add_offsets[c], cnt = P->add_offsets[c + 1] - o;
        TPSS_TRY(patch_pass<float>(P, P->d_add_list + o, cnt, B->omega, B->nrhs, r, x, B->side[next]));
      }
    }
    next = (next + 1) % K;
  }
  return TPSS_OK;
}
static tpss_status side_join(tpss_batch* B, bool forked) {
  if (!forked) return TPSS_OK;
  for (size_t k = 0; k < B->side.size(); ++k) {
    TPSS_CHECK_CUDA(cudaEventRecord(B->side_join[k], B->side[k]));
    TPSS_CHECK_CUDA(cudaStreamWaitEvent(B->stream, B->side_join[k], 0));
  }
  return TPSS_OK;
}
// A tcgen05 pass of the batch gave up waiting for its MMAs (in a replayed
// graph the per-call check does not run): report it once, clear the flags.
static tpss_status side_failed(tpss_batch* B) {
  bool bad = false;
  for (const BatchProb& bp : B->probs)
    for (int l = 1; l < (int)bp.route.size(); ++l) {
      tpss_patches* P = bp.ctx->mg->patches[l];
      if (bp.route[l] == 1 && P->h_fail_flag && *reinterpret_cast<volatile int*>(P->h_fail_flag) != 0) {
        *P->h_fail_flag = 0;
        bad = true;
      }
    }
  if (bad) {
    set_error("batch: a tcgen05 smoother pass gave up waiting for its MMAs (results invalid)");
    return TPSS_ETIMEOUT;
  }
  return TPSS_OK;
}

// Does level l of problem bp go through the tcgen05 column smoother?
static bool uses_tc05(const tpss_batch* B, const BatchProb& bp, int l) {
  const tpss_patches* P = bp.ctx->mg->patches[l];
  const Level& L = bp.ctx->levels[l];
  return B->bf16 && B->columns && P != nullptr && P->d_bop != nullptr && P->additive_schedule == TPSS_ADDITIVE_TCGEN05 &&
         P->kind == TPSS_VERTEX_PATCH && !P->per_sub && P->n <= 16 && L.nc[0] >= 2 && L.nc[1] >= 2 && L.nc[2] >= 2;
}

static tpss_status set_descs(tpss_batch* B, int depth) {
  std::vector<BatchLevelDesc> pre(B->probs.size()), post(B->probs.size());
  for (int p = 0; p < (int)B->probs.size(); ++p) {
    const BatchProb& bp = B->probs[p];
    const int l = bp.L - depth;
    BatchLevelDesc d{};
    if (l >= 1) {
      tpss_patches* P = bp.ctx->mg->patches[l];
      const Level& L = bp.ctx->levels[l];
      for (int t = 0; t < 3; ++t) {
        d.Z[t] = P->d_Z32[t];
        d.lam[t] = P->d_lam32[t];
      }
      d.list = P->d_add_list;
      d.nc0 = L.nc[0];
      d.nc1 = L.nc[1];
      d.ndofs = L.ndofs;
      d.n = P->n;
      d.variant = B->variant[P->n];
      d.x = bp.x[l];
      d.r = bp.b[l];
    }
    pre[p] = d;
    d.r = l >= 1 ? bp.r[l] : nullptr;
    post[p] = d;
  }
  TPSS_CHECK_CUDA(cudaMemcpyAsync(B->d_desc[depth], pre.data(), pre.size() * sizeof(BatchLevelDesc),
                                  cudaMemcpyHostToDevice, B->stream));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(B->d_desc_post[depth], post.data(), post.size() * sizeof(BatchLevelDesc),
                                  cudaMemcpyHostToDevice, B->stream));
  TPSS_CHECK_CUDA(cudaStreamSynchronize(B->stream));
  return TPSS_OK;
}

// Per-problem work f(bp) (operators, transfers, coarse solves: launches on
// bp.ctx->stream) spread over the side streams between a fork from and a
// join into the batch stream, so that the problems' launches run side by
// side instead of one after another; serial on the batch stream without
// side streams.
template <typename F>
static tpss_status on_sides(tpss_batch* B, F&& f) {
  const int K = (int)B->side.size();
  if (K == 0) {
    for (BatchProb& bp : B->probs) TPSS_TRY(f(bp));
    return TPSS_OK;
  }
  TPSS_CHECK_CUDA(cudaEventRecord(B->side_fork, B->stream));
  for (int k = 0; k < K; ++k) TPSS_CHECK_CUDA(cudaStreamWaitEvent(B->side[k], B->side_fork, 0));
  int k = 0;
  for (BatchProb& bp : B->probs) {
    cudaStream_t keep = bp.ctx->stream;
    bp.ctx->stream = B->side[k];
    const tpss_status st = f(bp);
    bp.ctx->stream = keep;
    if (st != TPSS_OK) return st;
    k = (k + 1) % K;
  }
  return side_join(B, true);
}

// One FP32 V-cycle for every problem and right-hand side: fx = MG(0, fb).
static tpss_status batch_vcycle_rec(tpss_batch* B, int depth) {
  cudaStream_t s = B->stream;
  const int nr = B->nrhs;
  bool any = false;
  for (const BatchProb& bp : B->probs) any = any || bp.L - depth > 0;
  TPSS_TRY(on_sides(B, [&](BatchProb& bp) -> tpss_status {
    const int l = bp.L - depth;
    if (l == 0) {
      MGState* mg = bp.ctx->mg;
      const int64_t n = bp.ctx->levels[0].ndofs;
      dim3 grid((unsigned)((n * 32 + 255) / 256), (unsigned)((nr + 3) / 4));
      batch_dense_mv_kernel<<<grid, 256, 0, bp.ctx->stream>>>(mg->coarse_inv, bp.b[0], bp.x[0], n, nr);
      TPSS_CHECK_LAUNCH();
    } else if (l > 0) {
      TPSS_CHECK_CUDA(cudaMemsetAsync(bp.x[l], 0, (size_t)bp.ctx->levels[l].ndofs * nr * sizeof(float),
                                      bp.ctx->stream));
    }
    return TPSS_OK;
  }));
  if (!any) return TPSS_OK;
  // pre-smoothing (x = 0, r = b): one persistent launch for all problems
  // (the tcgen05 levels on the side streams)
  bool forked = false;
  TPSS_TRY(side_passes(B, depth, false, 1, &forked));
  TPSS_TRY(launch_level(B, B->d_desc[depth], B->d_items[depth], B->nitems[depth], B->smem[depth],
                        B->grid[depth], B->d_counter + 2 * depth, s));
  TPSS_TRY(side_join(B, forked));
  TPSS_TRY(on_sides(B, [&](BatchProb& bp) -> tpss_status {
    const int l = bp.L - depth;
    if (l < 1) return TPSS_OK;
    TPSS_TRY(apply_operator_t<float>(bp.ctx, l, nr, bp.x[l], bp.r[l], bp.b[l]));
    return restrict_t<float>(bp.ctx, l, nr, bp.r[l], bp.b[l - 1]);
  }));
  TPSS_TRY(batch_vcycle_rec(B, depth + 1));
  TPSS_TRY(on_sides(B, [&](BatchProb& bp) -> tpss_status {
    const int l = bp.L - depth;
    if (l < 1) return TPSS_OK;
    TPSS_TRY(prolongate_add_t<float>(bp.ctx, l, nr, bp.x[l - 1], bp.x[l]));
    return apply_operator_t<float>(bp.ctx, l, nr, bp.x[l], bp.r[l], bp.b[l]);
  }));
  // post-smoothing with the residual
  TPSS_TRY(side_passes(B, depth, true, 0, &forked));
  TPSS_TRY(launch_level(B, B->d_desc_post[depth], B->d_items[depth], B->nitems[depth], B->smem[depth],
                        B->grid[depth], B->d_counter + 2 * depth + 1, s));
  TPSS_TRY(side_join(B, forked));
  return TPSS_OK;
}

static tpss_status batch_vcycle(tpss_batch* B) {
  if (B->graph_exec) {
    TPSS_CHECK_CUDA(cudaGraphLaunch(B->graph_exec, B->stream));
    return TPSS_OK;
  }
  return batch_vcycle_rec(B, 0);
}

static tpss_status autotune(tpss_batch* B) {
  // time every (routine, patches per work item) candidate on the finest-level
  // items of each patch size and keep the fastest
  const int cands_simt[] = {1, 2, 3, 4, 6, 8};
  const int cands_bf16[] = {1, 2, 4, 8, 16, 32};
  cudaEvent_t e0, e1;
  TPSS_CHECK_CUDA(cudaEventCreate(&e0));
  TPSS_CHECK_CUDA(cudaEventCreate(&e1));
  std::vector<int> ns;
  for (auto& bp : B->probs) ns.push_back(bp.ctx->mg->patches[bp.L]->n);
  std::sort(ns.begin(), ns.end());
  ns.erase(std::unique(ns.begin(), ns.end()), ns.end());
  BatchItem* d_tmp = nullptr;
  for (int n : ns) {
    double best = 1e30;
    int bestg = 1, bestv = 0;
    for (int var = 0; var <= (B->bf16 ? 1 : 0); ++var) {
      for (int ci = 0; ci < 6; ++ci) {
        const int g = var ? cands_bf16[ci] : cands_simt[ci];
        if (!var && (size_t)g * bshape_slot(n) * sizeof(float) > 100 * 1024) continue;
        if (!var && g * n * n > 4 * kBatchThreads) continue;
        std::vector<BatchItem> items;
        size_t smem = 0;
        build_items(B, 0, items, smem, n, g, var);
        if (items.empty()) continue;
        B->variant[n] = var;
        TPSS_TRY(set_descs(B, 0));
        dfree(d_tmp);
        d_tmp = nullptr;
        TPSS_TRY(dalloc_t(&d_tmp, items.size()));
        TPSS_CHECK_CUDA(cudaMemcpyAsync(d_tmp, items.data(), items.size() * sizeof(BatchItem),
                                        cudaMemcpyHostToDevice, B->stream));
        double t_best = 1e30;
        int grid = 1;
        TPSS_TRY(grid_size(B, (int)items.size(), smem, &grid));
        for (int rep = 0; rep < 3; ++rep) {
          TPSS_CHECK_CUDA(cudaEventRecord(e0, B->stream));
          TPSS_TRY(launch_level(B, B->d_desc[0], d_tmp, (int)items.size(), smem, grid, B->d_counter, B->stream));
          TPSS_CHECK_CUDA(cudaEventRecord(e1, B->stream));
          TPSS_CHECK_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          t_best = std::min(t_best, (double)ms);
        }
        if (t_best < best) {
          best = t_best;
          bestg = g;
          bestv = var;
        }
      }
    }
    B->ppb[n] = bestg;
    B->variant[n] = bestv;
  }
  dfree(d_tmp);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return TPSS_OK;
}

static void free_batch(tpss_batch* B) {
  if (B->graph_exec) cudaGraphExecDestroy(B->graph_exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (auto* d : B->d_desc) dfree(d);
  for (auto* d : B->d_desc_post) dfree(d);
  for (auto* d : B->d_items) dfree(d);
  dfree(B->d_desc_fin);
  dfree(B->d_counter);
  dfree(B->fb);
  dfree(B->fx);
  for (BatchProb& bp : B->probs) {
    for (int l = 0; l < (int)bp.b.size(); ++l) {
      if (l != bp.L) {
        dfree(bp.b[l]);
        dfree(bp.x[l]);
      }
      dfree(bp.r[l]);
    }
    if (bp.ctx) tpss_destroy(bp.ctx);
  }
  for (cudaStream_t st : B->side) cudaStreamDestroy(st);
  for (cudaEvent_t e : B->side_join) cudaEventDestroy(e);
  if (B->side_fork) cudaEventDestroy(B->side_fork);
  dfree(B->r); dfree(B->z); dfree(B->p); dfree(B->q); dfree(B->zold);
  dfree(B->d_off); dfree(B->d_len); dfree(B->sc); dfree(B->partials);
}

}  // namespace tpss

extern "C" tpss_status tpss_batch_create(const tpss_problem_desc* descs, int nprob, int nrhs,
                                         const tpss_mg_params* params, int flags, void* cuda_stream,
                                         tpss_batch** out) {
  clear_error();
  TPSS_REQUIRE(descs && params && out, "tpss_batch_create: null argument");
  *out = nullptr;
  TPSS_REQUIRE(nprob >= 1 && nprob <= 4096, "tpss_batch_create: nprob out of range");
  TPSS_REQUIRE(nrhs >= 1 && nrhs <= 64, "tpss_batch_create: nrhs out of range");
  TPSS_REQUIRE(params->smoother == TPSS_AVS, "tpss_batch_create: the batch uses the additive vertex-patch smoother");
  TPSS_REQUIRE(params->omega > 0.0, "tpss_batch_create: omega must be positive");
  for (int p = 0; p < nprob; ++p) {
    TPSS_REQUIRE(descs[p].dim == 3, "tpss_batch_create: batched problems are 3D");
    TPSS_REQUIRE(descs[p].nlevels >= 2, "tpss_batch_create: each problem needs >= 2 levels");
  }
  tpss_batch* B = new tpss_batch();
  B->nrhs = nrhs;
  B->nsys = nprob * nrhs;
  B->omega = (float)params->omega;
  B->flexible = 1;
  B->use_graph = (flags & 1) ? 0 : 1;
  B->bf16 = params->precision == TPSS_BF16 ? 1 : 0;
  B->columns = (flags & 4) ? 0 : 1;
  B->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, dev);
  tpss_status st = TPSS_OK;
  auto fail = [&](tpss_status s) {
    cudaStreamSynchronize(B->stream);
    free_batch(B);
    delete B;
    return s;
  };
  tpss_mg_params mp = *params;
  mp.precision = B->bf16 ? TPSS_BF16 : TPSS_FP32;
  B->probs.resize(nprob);
  for (int p = 0; p < nprob; ++p) {
    BatchProb& bp = B->probs[p];
    if ((st = tpss_create(&descs[p], cuda_stream, &bp.ctx)) != TPSS_OK) return fail(st);
    if ((st = tpss_mg_setup(bp.ctx, &mp)) != TPSS_OK) return fail(st);
    bp.L = bp.ctx->nlevels - 1;
    B->maxdepth = std::max(B->maxdepth, bp.L);
    bp.off = (B->total + 3) / 4 * 4;   // 16-byte aligned problem blocks (vector and cp.async accesses)
    B->total = bp.off + bp.ctx->levels[bp.L].ndofs * nrhs;
    for (int l = 0; l <= bp.L; ++l)
      if ((st = ensure_level_scratch(bp.ctx, l, nrhs)) != TPSS_OK) return fail(st);
    bp.route.assign(bp.L + 1, 0);
    for (int l = 1; l <= bp.L; ++l)
      bp.route[l] = uses_tc05(B, bp, l) ? 1 : (B->bf16 && B->columns) ? 2 : 0;
  }
  {
    {
      const int K = 4;   // side streams: per-problem passes, operators and transfers run side by side
      B->side.assign(K, nullptr);
      B->side_join.assign(K, nullptr);
      for (int k = 0; k < K; ++k) {
        if (cudaStreamCreateWithFlags(&B->side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->side_join[k], cudaEventDisableTiming) != cudaSuccess) {
          set_error("tpss_batch_create: side stream creation failed");
          return fail(TPSS_ECUDA);
        }
      }
      if (cudaEventCreateWithFlags(&B->side_fork, cudaEventDisableTiming) != cudaSuccess) {
        set_error("tpss_batch_create: side stream creation failed");
        return fail(TPSS_ECUDA);
      }
    }
  }
  if ((st = dalloc_t(&B->fb, B->total)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->fx, B->total)) != TPSS_OK) return fail(st);
  for (BatchProb& bp : B->probs) {
    bp.b.assign(bp.L + 1, nullptr);
    bp.x.assign(bp.L + 1, nullptr);
    bp.r.assign(bp.L + 1, nullptr);
    for (int l = 0; l <= bp.L; ++l) {
      const size_t n = (size_t)bp.ctx->levels[l].ndofs * nrhs;
      if (l == bp.L) {
        bp.b[l] = B->fb + bp.off;
        bp.x[l] = B->fx + bp.off;
      } else {
        if ((st = dalloc_t(&bp.b[l], n)) != TPSS_OK) return fail(st);
        if ((st = dalloc_t(&bp.x[l], n)) != TPSS_OK) return fail(st);
      }
      if ((st = dalloc_t(&bp.r[l], n)) != TPSS_OK) return fail(st);
    }
  }
  const int D = B->maxdepth;  // depths 0..D-1 have smoothing levels
  B->d_desc.assign(D, nullptr);
  B->d_desc_post.assign(D, nullptr);
  B->d_items.assign(D, nullptr);
  B->nitems.assign(D, 0);
  B->smem.assign(D, 0);
  B->grid.assign(D, 1);
  if ((st = dalloc_t(&B->d_counter, 2 * D + 2)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->d_desc_fin, nprob)) != TPSS_OK) return fail(st);
  for (int d = 0; d < D; ++d) {
    if ((st = dalloc_t(&B->d_desc[d], nprob)) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&B->d_desc_post[d], nprob)) != TPSS_OK) return fail(st);
    if ((st = set_descs(B, d)) != TPSS_OK) return fail(st);
  }
  for (int n = 0; n <= 16; ++n) {
    B->variant[n] = 0;
    B->ppb[n] = std::max(1, 256 / std::max(1, n * n));
  }
  cudaFuncSetAttribute(batch_smooth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024 + 1024);
  cudaFuncSetAttribute(batch_smooth_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024 + 1024);
  cudaMemsetAsync(B->fb, 0, B->total * sizeof(float), B->stream);
  cudaMemsetAsync(B->fx, 0, B->total * sizeof(float), B->stream);
  if (!(flags & 2))
    if ((st = autotune(B)) != TPSS_OK) return fail(st);
  for (int d = 0; d < D; ++d)
    if ((st = set_descs(B, d)) != TPSS_OK) return fail(st);
  for (int d = 0; d < D; ++d) {
    std::vector<BatchItem> items;
    size_t smem = 0;
    build_items(B, d, items, smem);
    B->nitems[d] = (int)items.size();
    B->smem[d] = smem;
    if ((st = grid_size(B, std::max(1, B->nitems[d]), smem, &B->grid[d])) != TPSS_OK) return fail(st);
    if ((st = dalloc_t(&B->d_items[d], std::max<size_t>(1, items.size()))) != TPSS_OK) return fail(st);
    if (!items.empty())
      if (cudaMemcpyAsync(B->d_items[d], items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                          B->stream) != cudaSuccess) {
        set_error("tpss_batch_create: copy of work items failed");
        return fail(TPSS_ECUDA);
      }
  }
  // CG state
  const int S = B->nsys;
  B->off.resize(S);
  B->len.resize(S);
  for (int p = 0; p < nprob; ++p)
    for (int r = 0; r < nrhs; ++r) {
      const int64_t n = B->probs[p].ctx->levels[B->probs[p].L].ndofs;
      B->off[p * nrhs + r] = B->probs[p].off + r * n;
      B->len[p * nrhs + r] = n;
    }
  B->chunks = 64;
  if ((st = dalloc_t(&B->r, B->total)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->z, B->total)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->p, B->total)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->q, B->total)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->zold, B->total)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->d_off, S)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->d_len, S)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->sc, 6 * S)) != TPSS_OK) return fail(st);
  if ((st = dalloc_t(&B->partials, (size_t)S * B->chunks)) != TPSS_OK) return fail(st);
  if (cudaMemcpyAsync(B->d_off, B->off.data(), S * sizeof(int64_t), cudaMemcpyHostToDevice, B->stream) != cudaSuccess ||
      cudaMemcpyAsync(B->d_len, B->len.data(), S * sizeof(int64_t), cudaMemcpyHostToDevice, B->stream) != cudaSuccess ||
      cudaStreamSynchronize(B->stream) != cudaSuccess) {
    set_error("tpss_batch_create: setup copies failed");
    return fail(TPSS_ECUDA);
  }
  // warm-up V-cycle (loads modules, sets kernel attributes), then capture the graph
  cudaMemsetAsync(B->fb, 0, B->total * sizeof(float), B->stream);
  if ((st = batch_vcycle_rec(B, 0)) != TPSS_OK) return fail(st);
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) {
    set_error("tpss_batch_create: warm-up V-cycle failed");
    return fail(TPSS_ECUDA);
  }
  if (B->use_graph) {
    if (B->stream == nullptr) {
      B->use_graph = 0;  // the legacy default stream cannot be captured
    } else {
      if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("tpss_batch_create: stream capture failed to start");
        return fail(TPSS_ECUDA);
      }
      tpss_status cs = batch_vcycle_rec(B, 0);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(B->stream, &g);
      if (cs != TPSS_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        set_error("tpss_batch_create: V-cycle capture failed");
        return fail(TPSS_ECUDA);
      }
      B->graph = g;
      if (cudaGraphInstantiate(&B->graph_exec, g, 0) != cudaSuccess) {
        set_error("tpss_batch_create: graph instantiation failed");
        return fail(TPSS_ECUDA);
      }
    }
  }
  *out = B;
  return TPSS_OK;
}

extern "C" tpss_status tpss_batch_destroy(tpss_batch* B) {
  if (!B) return TPSS_OK;
  cudaStreamSynchronize(B->stream);
  free_batch(B);
  delete B;
  return TPSS_OK;
}

extern "C" tpss_status tpss_batch_summary(const tpss_batch* B, int64_t* total, int* nsys, int* uses_graph) {
  clear_error();
  TPSS_REQUIRE(B, "tpss_batch_summary: null batch");
  if (total) *total = B->total;
  if (nsys) *nsys = B->nsys;
  if (uses_graph) *uses_graph = B->graph_exec != nullptr;
  return TPSS_OK;
}

extern "C" tpss_status tpss_batch_info(const tpss_batch* B, int prob, int64_t* ndofs, int64_t* offset,
                                       int* ppb_of_finest) {
  clear_error();
  TPSS_REQUIRE(B, "tpss_batch_info: null batch");
  TPSS_REQUIRE(prob >= 0 && prob < (int)B->probs.size(), "tpss_batch_info: prob out of range");
  const BatchProb& bp = B->probs[prob];
  if (ndofs) *ndofs = bp.ctx->levels[bp.L].ndofs;
  if (offset) *offset = bp.off;
  if (ppb_of_finest) *ppb_of_finest = B->ppb[bp.ctx->mg->patches[bp.L]->n];
  return TPSS_OK;
}

extern "C" tpss_status tpss_batch_smooth_additive(tpss_batch* B, const float* b, float* x) {
  clear_error();
  TPSS_REQUIRE(B && b && x, "tpss_batch_smooth_additive: null argument");
  TPSS_REQUIRE(b != x, "tpss_batch_smooth_additive: b and x must not alias");
  TPSS_REQUIRE(((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15) == 0,
               "tpss_batch_smooth_additive: b and x must be 16-byte aligned");
  // finest level of every problem, x = omega sum_j R_j^T A_j^{-1} R_j b, one persistent launch
  std::vector<BatchLevelDesc> desc(B->probs.size());
  for (int p = 0; p < (int)B->probs.size(); ++p) {
    const BatchProb& bp = B->probs[p];
    tpss_patches* P = bp.ctx->mg->patches[bp.L];
    const Level& L = bp.ctx->levels[bp.L];
    BatchLevelDesc d{};
    for (int t = 0; t < 3; ++t) {
      d.Z[t] = P->d_Z32[t];
      d.lam[t] = P->d_lam32[t];
    }
    d.list = P->d_add_list;
    d.nc0 = L.nc[0];
    d.nc1 = L.nc[1];
    d.ndofs = L.ndofs;
    d.n = P->n;
    d.variant = B->variant[P->n];
    d.r = b + bp.off;
    d.x = x + bp.off;
    desc[p] = d;
  }
  B->h_desc_fin = desc;
  TPSS_CHECK_CUDA(cudaMemcpyAsync(B->d_desc_fin, B->h_desc_fin.data(), desc.size() * sizeof(BatchLevelDesc),
                                  cudaMemcpyHostToDevice, B->stream));
  TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, B->total * sizeof(float), B->stream));
  bool forked = false;
  TPSS_TRY(side_passes(B, 0, false, 1, &forked, b, x));
  TPSS_TRY(launch_level(B, B->d_desc_fin, B->d_items[0], B->nitems[0], B->smem[0], B->grid[0],
                        B->d_counter + 2 * B->maxdepth, B->stream));
  return side_join(B, forked);
}

extern "C" tpss_status tpss_batch_vcycle(tpss_batch* B, const double* b, double* x) {
  clear_error();
  TPSS_REQUIRE(B && b && x, "tpss_batch_vcycle: null argument");
  TPSS_REQUIRE(b != x, "tpss_batch_vcycle: b and x must not alias");
  const int g = B->num_sms * 8;
  f64_to_f32_kernel<<<g, 256, 0, B->stream>>>(b, B->fb, B->total);
  TPSS_TRY(batch_vcycle(B));
  f32_to_f64_kernel<<<g, 256, 0, B->stream>>>(B->fx, x, B->total);
  TPSS_CHECK_LAUNCH();
  return side_failed(B);
}

namespace tpss {
static tpss_status seg_dot(tpss_batch* B, const double* x, const double* y, double* out) {
  dim3 grid(B->chunks, B->nsys);
  seg_dot_kernel<<<grid, 256, 0, B->stream>>>(x, y, B->d_off, B->d_len, B->partials, B->chunks);
  seg_dot_final_kernel<<<B->nsys, 64, 0, B->stream>>>(B->partials, B->chunks, out);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}
}  // namespace tpss

extern "C" tpss_status tpss_batch_pcg_solve(tpss_batch* B, const double* b, double* x, double rtol, int maxit,
                                            int* iters, double* rel_res) {
  clear_error();
  TPSS_REQUIRE(B && b && x && iters && rel_res, "tpss_batch_pcg_solve: null argument");
  TPSS_REQUIRE(rtol > 0.0 && maxit >= 1, "tpss_batch_pcg_solve: rtol must be > 0 and maxit >= 1");
  const int S = B->nsys;
  cudaStream_t s = B->stream;
  const int g = B->num_sms * 8;
  double* sc = B->sc;
  dim3 sgrid(B->chunks, S);
  TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, B->total * sizeof(double), s));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(B->r, b, B->total * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TPSS_TRY(seg_dot(B, B->r, B->r, sc + 2 * S));
  std::vector<double> h(6 * S, 0.0), rr0(S);
  TPSS_CHECK_CUDA(cudaMemcpyAsync(h.data(), sc, 6 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
  TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
  std::vector<double> active(S, 1.0);
  for (int k = 0; k < S; ++k) {
    rr0[k] = h[2 * S + k];
    iters[k] = 0;
    rel_res[k] = rr0[k] > 0.0 ? 1.0 : 0.0;
    if (!(rr0[k] > 0.0)) active[k] = 0.0;
    if (!std::isfinite(rr0[k])) {
      set_error("tpss_batch_pcg_solve: right-hand side is not finite");
      return TPSS_EBREAKDOWN;
    }
  }
  TPSS_CHECK_CUDA(cudaMemcpyAsync(sc + 5 * S, active.data(), S * sizeof(double), cudaMemcpyHostToDevice, s));
  TPSS_TRY(tpss_batch_vcycle(B, B->r, B->z));
  TPSS_CHECK_CUDA(cudaMemcpyAsync(B->p, B->z, B->total * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TPSS_TRY(seg_dot(B, B->r, B->z, sc + 0 * S));
  int nactive = (int)std::count(active.begin(), active.end(), 1.0);
  for (int it = 1; it <= maxit && nactive > 0; ++it) {
    TPSS_TRY(on_sides(B, [&](BatchProb& bp) {
      return apply_operator_t<double>(bp.ctx, bp.L, B->nrhs, B->p + bp.off, B->q + bp.off, nullptr);
    }));
    TPSS_TRY(seg_dot(B, B->p, B->q, sc + 1 * S));
    seg_xr_kernel<<<sgrid, 256, 0, s>>>(x, B->r, B->p, B->q, B->d_off, B->d_len, sc, S);
    TPSS_TRY(seg_dot(B, B->r, B->r, sc + 2 * S));
    TPSS_CHECK_CUDA(cudaMemcpyAsync(h.data(), sc, 6 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
    TPSS_CHECK_CUDA(cudaStreamSynchronize(s));
    bool changed = false;
    for (int k = 0; k < S; ++k) {
      if (active[k] == 0.0) continue;
      if (!std::isfinite(h[1 * S + k]) || !(h[1 * S + k] > 0.0) || !std::isfinite(h[2 * S + k])) {
        set_error("tpss_batch_pcg_solve: breakdown in system " + std::to_string(k));
        return TPSS_EBREAKDOWN;
      }
      iters[k] = it;
      rel_res[k] = std::sqrt(std::max(h[2 * S + k], 0.0) / rr0[k]);
      if (rel_res[k] <= rtol) {
        active[k] = 0.0;
        --nactive;
        changed = true;
      }
    }
    if (nactive == 0) break;
    if (changed)
      TPSS_CHECK_CUDA(cudaMemcpyAsync(sc + 5 * S, active.data(), S * sizeof(double), cudaMemcpyHostToDevice, s));
    std::swap(B->z, B->zold);
    TPSS_TRY(tpss_batch_vcycle(B, B->r, B->z));
    TPSS_TRY(seg_dot(B, B->r, B->z, sc + 3 * S));
    TPSS_TRY(seg_dot(B, B->r, B->zold, sc + 4 * S));
    seg_p_kernel<<<sgrid, 256, 0, s>>>(B->p, B->z, B->d_off, B->d_len, sc, S, B->flexible);
    seg_shift_kernel<<<(S + 127) / 128, 128, 0, s>>>(sc, S);
    TPSS_CHECK_LAUNCH();
  }
  (void)g;
  TPSS_TRY(side_failed(B));
  if (nactive > 0) {
    set_error("tpss_batch_pcg_solve: not all systems converged within maxit");
    return TPSS_ENOTCONV;
  }
  return TPSS_OK;
}
