// Schwarz smoothers with fast-diagonalization local solvers (Sec. 2.3, 3.2).
//
// One CTA processes PPB subdomains (cells or vertex patches) of one color;
// each subdomain owns n^(d-1) threads, one per line of its n^d patch tensor.
// Per subdomain j (eq. fastinverse, eq. eigenvectormatvec):
//   gather     u = R_j r            (2^d cells of (k+1)^d values, or one cell)
//   Z^T        along x, y (, z)     (sum factorization, n^(d+1) FMAs each)
//   scale      u_ijl *= 1/(lambda_i + lambda_j + lambda_l)
//   Z          along z, y, x
//   scatter    x += omega R_j^T u
// The last Z^T contraction, the scale and the first Z contraction act on the
// same line and are fused in registers.  Subdomains of one color share no
// cell, so the scatter is a plain read-modify-write; colors run as separate
// launches in a fixed order, which makes the additive result deterministic.
//
// The tensor lives in shared memory with an odd line stride (n+1 for even n)
// so that the strided x-line accesses do not collide in the same bank.
#include <algorithm>

#include "tpss_internal.cuh"

namespace tpss {

template <int DIM, int N>
struct PatchShape {
  static constexpr int LINES = DIM == 3 ? N * N : N;
  static constexpr int LS = (N % 2 == 0) ? N + 1 : N;
  static constexpr int PS = LS * N;
  static constexpr int VOL = DIM == 3 ? PS * N : LS * N;
  static constexpr int VOLC = DIM == 3 ? N * N * N : N * N;
  // subdomains per CTA: about 256 threads, except n = 14 (196 lines: one
  // subdomain would leave 12.5% of the lanes of its last warp idle), and at
  // most what fits in 200 KB of shared memory (FP64 slot size; binds only
  // for the 2D subdomains with n > 16)
  static constexpr int PPB_LINES =
      LINES == 196 ? 2 : ((256 + LINES / 2) / LINES > 0 ? (256 + LINES / 2) / LINES : 1);
  static constexpr int SLOT_BYTES = (VOL + 2 * DIM * N * N + DIM * N) * 8;
  static constexpr int PPB_SMEM = (200 * 1024) / SLOT_BYTES > 0 ? (200 * 1024) / SLOT_BYTES : 1;
  static constexpr int PPB = PPB_LINES < PPB_SMEM ? PPB_LINES : PPB_SMEM;
  static constexpr int THREADS = PPB * LINES;
};

template <typename T>
struct SmoothArgs {
  const T* Z[3];       // [npos_t][n*n] row-major, column j = eigenvector j
  const T* lam[3];     // [npos_t][n]
  const double* inv;   // FP64 path: [nsub][n^d] inverse eigenvalue sums
  const int* list;     // packed subdomain positions of this color
  int count;
  const T* r;
  T* x;
  T* d;                // optional: d = omega u on the subdomain's DoFs (the update of x) ...
  T* rw;               // ... and then r *= 1 - omega there (r writable)
  T omega;
  int nc0, nc1;        // cells per direction (x, y)
  int np0, np1;        // subdomain positions per direction (x, y)
  int64_t ndofs;
  int per_sub;         // 1: Z, lam per subdomain (index sub), else per position along t
};

template <int DIM, int N>
__device__ __forceinline__ void line_geom(int t, int line, int& base, int& stride) {
  using S = PatchShape<DIM, N>;
  if (DIM == 3) {
    const int a = line % N, b = line / N;
    if (t == 0) { base = S::LS * a + S::PS * b; stride = 1; }
    else if (t == 1) { base = a + S::PS * b; stride = S::LS; }
    else { base = a + S::LS * b; stride = S::PS; }
  } else {
    if (t == 0) { base = S::LS * line; stride = 1; }
    else { base = line; stride = S::LS; }
  }
}

// out_i = sum_m W[m*N + i] v_m on one line, in place.
template <int N, typename T>
__device__ __forceinline__ void contract_line(T* __restrict__ buf, const T* __restrict__ W, int base, int stride) {
  T acc[N];
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = 0;
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const T v = buf[base + m * stride];
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(W[m * N + i], v, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) buf[base + i * stride] = acc[i];
}

template <int DIM, int N, bool VERTEX, typename T>
__global__ void __launch_bounds__(PatchShape<DIM, N>::THREADS)
patch_smooth_kernel(SmoothArgs<T> a) {
  using S = PatchShape<DIM, N>;
  constexpr int N1 = VERTEX ? N / 2 : N;
  constexpr int NLOC1 = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
  constexpr int NCELL = VERTEX ? (1 << DIM) : 1;
  constexpr int SLOT = S::VOL + 2 * DIM * N * N + DIM * N;
  extern __shared__ unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int slot = threadIdx.x / S::LINES;
  const int line = threadIdx.x % S::LINES;
  const int q = blockIdx.x * S::PPB + slot;
  const bool active = q < a.count;
  T* buf = smem + slot * SLOT;
  T* Zs = buf + S::VOL;             // [DIM][N*N]   Z
  T* ZTs = Zs + DIM * N * N;        // [DIM][N*N]   Z^T
  T* lams = ZTs + DIM * N * N;      // [DIM][N]
  const int64_t vbase = (int64_t)blockIdx.y * a.ndofs;
  int pos[3] = {0, 0, 0};
  if (active) {
    const int packed = a.list[q];
    pos[0] = unpack_x(packed);
    pos[1] = unpack_y(packed);
    pos[2] = unpack_z(packed);
    const int64_t psub = pos[0] + (int64_t)a.np0 * (pos[1] + (int64_t)a.np1 * pos[2]);
    for (int e = line; e < DIM * N * N; e += S::LINES) {
      const int t = e / (N * N), i = e % (N * N);
      const T z = a.Z[t][(size_t)(a.per_sub ? psub : pos[t]) * N * N + i];
      Zs[t * N * N + i] = z;
      ZTs[t * N * N + (i % N) * N + i / N] = z;
    }
    if (sizeof(T) == 4)
      for (int e = line; e < DIM * N; e += S::LINES)
        lams[e] = a.lam[e / N][(size_t)(a.per_sub ? psub : pos[e / N]) * N + e % N];
    // gather R_j r
    for (int e = line; e < NCELL * NLOC1; e += S::LINES) {
      const int c = e / NLOC1, loc = e % NLOC1;
      const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
      const int ix = loc % N1, iy = (loc / N1) % N1, iz = DIM == 3 ? loc / (N1 * N1) : 0;
      const int64_t gcell = (pos[0] + sx) + (int64_t)a.nc0 * ((pos[1] + sy) + (int64_t)a.nc1 * (DIM == 3 ? pos[2] + sz : 0));
      const int pidx = (sx * N1 + ix) + S::LS * (sy * N1 + iy) + (DIM == 3 ? S::PS * (sz * N1 + iz) : 0);
      buf[pidx] = a.r[vbase + gcell * NLOC1 + loc];
    }
  }
  __syncthreads();
  int base, stride;
  // Z^T along all directions but the last
  for (int t = 0; t < DIM - 1; ++t) {
    if (active) {
      line_geom<DIM, N>(t, line, base, stride);
      contract_line<N, T>(buf, Zs + t * N * N, base, stride);
    }
    __syncthreads();
  }
  // last direction: Z^T, scale by Lambda^{-1}, Z -- fused on the line
  if (active) {
    constexpr int TL = DIM - 1;
    line_geom<DIM, N>(TL, line, base, stride);
    T acc[N];
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = 0;
    const T* W = Zs + TL * N * N;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const T v = buf[base + m * stride];
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] = fma(W[m * N + i], v, acc[i]);
    }
    const int la = DIM == 3 ? line % N : line, lb = DIM == 3 ? line / N : 0;
    if (sizeof(T) == 8) {
      const int64_t sub = pos[0] + (int64_t)a.np0 * (pos[1] + (int64_t)a.np1 * pos[2]);
      const double* inv = a.inv + sub * S::VOLC + la + (DIM == 3 ? N * lb : 0);
      constexpr int ISTR = DIM == 3 ? N * N : N;
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] *= (T)__ldg(inv + i * ISTR);
    } else {
      const T s0 = lams[la] + (DIM == 3 ? lams[N + lb] : (T)0);
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] = acc[i] / (s0 + lams[TL * N + i]);
    }
    const T* WT = ZTs + TL * N * N;
    T out[N];
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
#pragma unroll
      for (int i = 0; i < N; ++i) out[i] = fma(WT[m * N + i], acc[m], out[i]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) buf[base + i * stride] = out[i];
  }
  __syncthreads();
  // Z along the remaining directions (reverse order)
  for (int t = DIM - 2; t >= 0; --t) {
    if (active) {
      line_geom<DIM, N>(t, line, base, stride);
      contract_line<N, T>(buf, ZTs + t * N * N, base, stride);
    }
    __syncthreads();
  }
  // scatter x += omega R_j^T u
  if (active) {
    for (int e = line; e < NCELL * NLOC1; e += S::LINES) {
      const int c = e / NLOC1, loc = e % NLOC1;
      const int sx = c & 1, sy = (c >> 1) & 1, sz = (c >> 2) & 1;
      const int ix = loc % N1, iy = (loc / N1) % N1, iz = DIM == 3 ? loc / (N1 * N1) : 0;
      const int64_t gcell = (pos[0] + sx) + (int64_t)a.nc0 * ((pos[1] + sy) + (int64_t)a.nc1 * (DIM == 3 ? pos[2] + sz : 0));
      const int pidx = (sx * N1 + ix) + S::LS * (sy * N1 + iy) + (DIM == 3 ? S::PS * (sz * N1 + iz) : 0);
      const int64_t gi = vbase + gcell * NLOC1 + loc;
      a.x[gi] = fma(a.omega, buf[pidx], a.x[gi]);
      if (a.d != nullptr) {
        a.d[gi] = a.omega * buf[pidx];
        a.rw[gi] *= T(1) - a.omega;
      }
    }
  }
}

template <int DIM, int N, bool VERTEX, typename T>
static tpss_status launch_smooth(const SmoothArgs<T>& a, int nrhs, cudaStream_t s) {
  using S = PatchShape<DIM, N>;
  constexpr int SLOT = S::VOL + 2 * DIM * N * N + DIM * N;
  const size_t smem = (size_t)S::PPB * SLOT * sizeof(T);
  static bool attr_set = false;
  if (smem > 48 * 1024 && !attr_set) {
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(patch_smooth_kernel<DIM, N, VERTEX, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  if (a.count <= 0) return TPSS_OK;
  dim3 grid((a.count + S::PPB - 1) / S::PPB, nrhs);
  patch_smooth_kernel<DIM, N, VERTEX, T><<<grid, S::THREADS, smem, s>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

template <typename T>
tpss_status patch_pass(tpss_patches* P, const int* list, int count, T omega, int nrhs, const T* r, T* x,
                       cudaStream_t s, T* d) {
  if constexpr (sizeof(T) == 4) {
    float* df = reinterpret_cast<float*>(d);
    if (P->precision == TPSS_BF16 && P->ctx->dim == 3) {
      const tpss_status st = patch_pass_bf16(P, list, count, (float)omega, nrhs, reinterpret_cast<const float*>(r),
                                             reinterpret_cast<float*>(x), s, df);
      if (st != TPSS_EINVAL) return st;   // else: shape not covered, use the generic tensor-core kernel
    }
    if (P->precision == TPSS_TF32 || P->precision == TPSS_BF16)
      return patch_pass_tc(P, list, count, (float)omega, nrhs, reinterpret_cast<const float*>(r),
                           reinterpret_cast<float*>(x), s, df);
  }
  const tpss_ctx* ctx = P->ctx;
  const Level& L = ctx->levels[P->level];
  SmoothArgs<T> a{};
  for (int t = 0; t < 3; ++t) {
    if constexpr (sizeof(T) == 8) {
      a.Z[t] = reinterpret_cast<const T*>(P->d_Z[t]);
      a.lam[t] = reinterpret_cast<const T*>(P->d_lam[t]);
    } else {
      a.Z[t] = reinterpret_cast<const T*>(P->d_Z32[t]);
      a.lam[t] = reinterpret_cast<const T*>(P->d_lam32[t]);
    }
  }
  a.inv = P->d_inv;
  a.list = list;
  a.count = count;
  a.r = r;
  a.x = x;
  a.d = d;
  a.rw = const_cast<T*>(r);
  a.omega = omega;
  a.nc0 = L.nc[0];
  a.nc1 = L.nc[1];
  a.np0 = P->npos[0];
  a.np1 = P->npos[1];
  a.ndofs = L.ndofs;
  a.per_sub = P->per_sub;
  const bool v = P->kind == TPSS_VERTEX_PATCH;
  const int n = P->n;
#define TPSS_SM_CASE(D, NN, V)                                                     \
  if (ctx->dim == D && n == NN && v == V) return launch_smooth<D, NN, V, T>(a, nrhs, s);
  if constexpr (sizeof(T) == sizeof(double)) {   // degrees 8..15: FP64 only
    if (ctx->dim == 3 && v && n > kMaxSharedPatchN) return patch_pass_large(P, list, count, omega, nrhs, r, x, s, d);
    TPSS_SM_CASE(3, 9, false) TPSS_SM_CASE(3, 10, false) TPSS_SM_CASE(3, 11, false) TPSS_SM_CASE(3, 12, false)
    TPSS_SM_CASE(3, 13, false) TPSS_SM_CASE(3, 14, false) TPSS_SM_CASE(3, 15, false) TPSS_SM_CASE(3, 16, false)
    TPSS_SM_CASE(2, 9, false) TPSS_SM_CASE(2, 10, false) TPSS_SM_CASE(2, 11, false) TPSS_SM_CASE(2, 12, false)
    TPSS_SM_CASE(2, 13, false) TPSS_SM_CASE(2, 14, false) TPSS_SM_CASE(2, 15, false) TPSS_SM_CASE(2, 16, false)
    TPSS_SM_CASE(2, 18, true) TPSS_SM_CASE(2, 20, true) TPSS_SM_CASE(2, 22, true) TPSS_SM_CASE(2, 24, true)
    TPSS_SM_CASE(2, 26, true) TPSS_SM_CASE(2, 28, true) TPSS_SM_CASE(2, 30, true) TPSS_SM_CASE(2, 32, true)
  }
  TPSS_SM_CASE(3, 4, true) TPSS_SM_CASE(3, 6, true) TPSS_SM_CASE(3, 8, true) TPSS_SM_CASE(3, 10, true)
  TPSS_SM_CASE(3, 12, true) TPSS_SM_CASE(3, 14, true) TPSS_SM_CASE(3, 16, true)
  TPSS_SM_CASE(3, 2, false) TPSS_SM_CASE(3, 3, false) TPSS_SM_CASE(3, 4, false) TPSS_SM_CASE(3, 5, false)
  TPSS_SM_CASE(3, 6, false) TPSS_SM_CASE(3, 7, false) TPSS_SM_CASE(3, 8, false)
  TPSS_SM_CASE(2, 4, true) TPSS_SM_CASE(2, 6, true) TPSS_SM_CASE(2, 8, true) TPSS_SM_CASE(2, 10, true)
  TPSS_SM_CASE(2, 12, true) TPSS_SM_CASE(2, 14, true) TPSS_SM_CASE(2, 16, true)
  TPSS_SM_CASE(2, 2, false) TPSS_SM_CASE(2, 3, false) TPSS_SM_CASE(2, 4, false) TPSS_SM_CASE(2, 5, false)
  TPSS_SM_CASE(2, 6, false) TPSS_SM_CASE(2, 7, false) TPSS_SM_CASE(2, 8, false)
#undef TPSS_SM_CASE
  set_error("smoother: unsupported subdomain size");
  return TPSS_EINVAL;
}

template tpss_status patch_pass<double>(tpss_patches*, const int*, int, double, int, const double*, double*, cudaStream_t,
                                        double*);
template tpss_status patch_pass<float>(tpss_patches*, const int*, int, float, int, const float*, float*, cudaStream_t,
                                       float*);

template <typename T>
static T* residual_buffer(Level& L);
template <>
double* residual_buffer<double>(Level& L) { return L.t64[4]; }
template <>
float* residual_buffer<float>(Level& L) { return L.t32[4]; }
template <typename T>
static T* update_buffer(Level& L);
template <>
double* update_buffer<double>(Level& L) { return L.t64[0]; }
template <>
float* update_buffer<float>(Level& L) { return L.t32[0]; }

template <typename T>
tpss_status smooth_additive_t(tpss_patches* P, T omega, int nrhs, const T* b, T* x, int x_is_zero) {
  tpss_ctx* ctx = P->ctx;
  cudaStream_t s = ctx->stream;
  Level& L = ctx->levels[P->level];
  const T* r = b;
  // surrogate cell solvers (mapped meshes): residual, local solves and the
  // update in one launch, into a scratch vector (neighbours read x)
  if (P->per_sub && !x_is_zero) {
    TPSS_TRY(ensure_level_scratch(ctx, P->level, nrhs));
    T* rb = residual_buffer<T>(L);
    TPSS_TRY(mapped_fused_t<T>(P, nullptr, P->nsub, nrhs, x, b, rb, nullptr, 0, omega, T(0), T(0)));
    TPSS_CHECK_CUDA(cudaMemcpyAsync(x, rb, (size_t)L.ndofs * nrhs * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return TPSS_OK;
  }
  if constexpr (sizeof(T) == 4) {
    // BF16 / TF32 3D vertex patches, column-streaming schedule: writes x itself
    if ((P->precision == TPSS_BF16 && (P->additive_schedule == TPSS_ADDITIVE_COLUMNS ||
                                       P->additive_schedule == TPSS_ADDITIVE_TCGEN05)) ||
        (P->precision == TPSS_TF32 && P->additive_schedule == TPSS_ADDITIVE_TCGEN05)) {
      if (!x_is_zero) {
        TPSS_TRY(ensure_level_scratch(ctx, P->level, nrhs));
        T* rb = residual_buffer<T>(L);
        TPSS_TRY(apply_operator_t<T>(ctx, P->level, nrhs, x, rb, b));
        r = rb;
      }
      const float* rf = reinterpret_cast<const float*>(r);
      float* xf = reinterpret_cast<float*>(x);
      tpss_status st = TPSS_EINVAL;
      if (P->additive_schedule == TPSS_ADDITIVE_TCGEN05)
        st = patch_pass_tc05(P, (float)omega, nrhs, rf, xf, x_is_zero, s);
      if (st == TPSS_EINVAL && P->precision == TPSS_BF16)
        st = patch_pass_bf16_stream(P, (float)omega, nrhs, rf, xf, x_is_zero, s);
      if (st != TPSS_EINVAL) return st;   // else: shape or alignment not covered, colored launches
      if (!x_is_zero) {                   // r already holds the residual
        const int nc = (int)P->add_offsets.size() - 1;
        for (int c = 0; c < nc; ++c) {
          const int o = P->add_offsets[c], cnt = P->add_offsets[c + 1] - o;
          TPSS_TRY(patch_pass<T>(P, P->d_add_list + o, cnt, omega, nrhs, r, x, s));
        }
        return TPSS_OK;
      }
    }
  }
  if (x_is_zero) {
    TPSS_CHECK_CUDA(cudaMemsetAsync(x, 0, (size_t)L.ndofs * nrhs * sizeof(T), s));
  } else {
    TPSS_TRY(ensure_level_scratch(ctx, P->level, nrhs));
    T* rb = residual_buffer<T>(L);
    TPSS_TRY(apply_operator_t<T>(ctx, P->level, nrhs, x, rb, b));
    r = rb;
  }
  if constexpr (sizeof(T) == 4) {
    // BF16 3D: one launch over all subdomains, atomic accumulation into x
    if (P->precision == TPSS_BF16 && P->additive_schedule == TPSS_ADDITIVE_ATOMIC) {
      const tpss_status st = patch_pass_bf16_atomic(P, P->d_lex_list, (int)P->nsub, (float)omega, nrhs,
                                                    reinterpret_cast<const float*>(r), reinterpret_cast<float*>(x), s);
      if (st != TPSS_EINVAL) return st;   // else: shape or alignment not covered, colored launches
    }
  }
  if (P->additive_schedule == TPSS_ADDITIVE_PLANES && P->d_plane_list != nullptr) {
    // 3D vertex patches plane by plane: the cells of two neighbouring cell
    // planes stay in L2 across the plane's 4 color launches
    const int ncell_slots = ctx->num_sms * 3;
    for (size_t g = 0; g + 1 < P->plane_offsets.size(); ++g) {
      const int o = P->plane_offsets[g], cnt = P->plane_offsets[g + 1] - o;
      if (cnt == 0) continue;
      if constexpr (sizeof(T) == 4) {
        if (P->precision == TPSS_BF16) {
          // enough CTAs for ~4 waves: split the right-hand sides over CTAs
          const int rpc = std::max(1, std::min(nrhs, (int)((int64_t)cnt * nrhs / (4 * ncell_slots))));
          const tpss_status st = patch_pass_bf16(P, P->d_plane_list + o, cnt, (float)omega, nrhs,
                                                 reinterpret_cast<const float*>(r), reinterpret_cast<float*>(x), s,
                                                 nullptr, rpc);
          if (st == TPSS_OK) continue;
          if (st != TPSS_EINVAL) return st;
        }
      }
      TPSS_TRY(patch_pass<T>(P, P->d_plane_list + o, cnt, omega, nrhs, r, x, s));
    }
    return TPSS_OK;
  }
  // Two or more right-hand sides: the second half runs on a second stream
  // (fork and join by events), so that its color launches fill the SMs the
  // last wave of each color launch of the first half leaves idle; the halves
  // share no data and each sum keeps its order.  Not for the large 3D vertex
  // patches, whose CTAs share the patch set's global tensor slabs, nor where
  // the second half would start off the 16-byte alignment of the first (the
  // vectorized kernels need it).
  const int nc = (int)P->add_offsets.size() - 1;
  const bool large = ctx->dim == 3 && P->kind == TPSS_VERTEX_PATCH && P->n > kMaxSharedPatchN;
  const bool aligned = ((int64_t)(nrhs / 2) * L.ndofs * (int64_t)sizeof(T)) % 16 == 0;
  const int halves = (nrhs >= 2 && P->aux_stream != nullptr && !large && aligned) ? 2 : 1;
  if (halves == 2) {
    TPSS_CHECK_CUDA(cudaEventRecord(P->fork_event, s));
    TPSS_CHECK_CUDA(cudaStreamWaitEvent(P->aux_stream, P->fork_event, 0));
  }
  for (int c = 0; c < nc; ++c) {
    const int o = P->add_offsets[c], cnt = P->add_offsets[c + 1] - o;
    for (int h = 0; h < halves; ++h) {
      const int r0 = h == 0 ? 0 : nrhs / 2, nr = halves == 1 ? nrhs : (h == 0 ? nrhs / 2 : nrhs - nrhs / 2);
      const int64_t off = (int64_t)r0 * L.ndofs;
      TPSS_TRY(patch_pass<T>(P, P->d_add_list + o, cnt, omega, nr, r + off, x + off, h == 0 ? s : P->aux_stream));
    }
  }
  if (halves == 2) {
    TPSS_CHECK_CUDA(cudaEventRecord(P->join_event, P->aux_stream));
    TPSS_CHECK_CUDA(cudaStreamWaitEvent(s, P->join_event, 0));
  }
  return TPSS_OK;
}

// Multiplicative sweep over the colors (Alg. 3).  With P->mult_update set
// (default; used where it is exact: red-black cells and the 2^(d+1)-color
// vertex coloring) the residual is formed once and then updated after each
// color from the color's update d (smoother_mult.cu); otherwise
// r = b - A x is recomputed before every color.  The update takes the local
// solves as exact; with FP32 / TF32 / BF16 contractions it therefore omits
// their rounding error from the residual it carries (a change of the
// preconditioner at that level, which the flexible PCG of the mixed path
// absorbs; tests compare iteration counts with the recomputed residual).
template <typename T>
tpss_status smooth_multiplicative_t(tpss_patches* P, T omega, int reverse, int nrhs, const T* b, T* x) {
  tpss_ctx* ctx = P->ctx;
  cudaStream_t s = ctx->stream;
  Level& L = ctx->levels[P->level];
  TPSS_TRY(ensure_level_scratch(ctx, P->level, nrhs));
  T* rb = residual_buffer<T>(L);
  const bool alt = P->kind == TPSS_VERTEX_PATCH && P->mul_colors_active != P->mul_colors_default;
  const std::vector<int>& offs = alt ? P->mul8_offsets : P->mul_offsets;
  const int* list = alt ? P->d_mul8_list : P->d_mul_list;
  const int nc = (int)offs.size() - 1;
  const bool update = P->mult_update && !alt;
  if (update) {
    T* dx = update_buffer<T>(L);   // an operator temporary, free after the first residual
    TPSS_TRY(apply_operator_t<T>(ctx, P->level, nrhs, x, rb, b));
    int last = -1;
    for (int i = 0; i < nc; ++i) {
      const int c = reverse ? nc - 1 - i : i;
      if (offs[c + 1] > offs[c]) last = i;
    }
    for (int i = 0; i <= last; ++i) {
      const int c = reverse ? nc - 1 - i : i;
      const int o = offs[c], cnt = offs[c + 1] - o;
      if (cnt == 0) continue;
      TPSS_TRY(patch_pass<T>(P, list + o, cnt, omega, nrhs, rb, x, s, dx));
      if (i < last) TPSS_TRY(mult_residual_update<T>(P, c, nrhs, dx, rb, s));
    }
    return TPSS_OK;
  }
  for (int i = 0; i < nc; ++i) {
    const int c = reverse ? nc - 1 - i : i;
    const int o = offs[c], cnt = offs[c + 1] - o;
    if (cnt == 0) continue;
    // surrogate cell solvers (mapped meshes): the residual on the color's
    // cells only, local solves and update in one launch, in place (no two
    // cells of a red-black color share a face)
    if (P->per_sub) {
      TPSS_TRY(mapped_fused_t<T>(P, list + o, cnt, nrhs, x, b, x, nullptr, 0, omega, T(0), T(0)));
      continue;
    }
    TPSS_TRY(apply_operator_t<T>(ctx, P->level, nrhs, x, rb, b));
    TPSS_TRY(patch_pass<T>(P, list + o, cnt, omega, nrhs, rb, x, s));
  }
  return TPSS_OK;
}

template tpss_status smooth_additive_t<double>(tpss_patches*, double, int, const double*, double*, int);
template tpss_status smooth_additive_t<float>(tpss_patches*, float, int, const float*, float*, int);
template tpss_status smooth_multiplicative_t<double>(tpss_patches*, double, int, int, const double*, double*);
template tpss_status smooth_multiplicative_t<float>(tpss_patches*, float, int, int, const float*, float*);

}  // namespace tpss

using namespace tpss;

extern "C" tpss_status tpss_smooth_additive(tpss_patches* P, double omega, int nrhs, const double* b, double* x,
                                            int x_is_zero) {
  clear_error();
  TPSS_REQUIRE(P && b && x, "tpss_smooth_additive: null argument");
  TPSS_REQUIRE(P->precision == TPSS_FP64, "tpss_smooth_additive: patches were set up for FP32 (use _f32)");
  TPSS_REQUIRE(nrhs >= 1 && nrhs <= 65535, "tpss_smooth_additive: nrhs out of range");
  TPSS_REQUIRE((const void*)b != (const void*)x, "tpss_smooth_additive: b and x must not alias");
  return smooth_additive_t<double>(P, omega, nrhs, b, x, x_is_zero);
}

extern "C" tpss_status tpss_smooth_additive_f32(tpss_patches* P, float omega, int nrhs, const float* b, float* x,
                                                int x_is_zero) {
  clear_error();
  TPSS_REQUIRE(P && b && x, "tpss_smooth_additive_f32: null argument");
  TPSS_REQUIRE(P->precision != TPSS_FP64, "tpss_smooth_additive_f32: patches were set up for FP64");
  TPSS_REQUIRE(nrhs >= 1 && nrhs <= 65535, "tpss_smooth_additive_f32: nrhs out of range");
  TPSS_REQUIRE((const void*)b != (const void*)x, "tpss_smooth_additive_f32: b and x must not alias");
  return smooth_additive_t<float>(P, omega, nrhs, b, x, x_is_zero);
}

extern "C" tpss_status tpss_smooth_multiplicative(tpss_patches* P, double omega, int reverse_colors, int nrhs,
                                                  const double* b, double* x) {
  clear_error();
  TPSS_REQUIRE(P && b && x, "tpss_smooth_multiplicative: null argument");
  TPSS_REQUIRE(P->precision == TPSS_FP64, "tpss_smooth_multiplicative: patches were set up for FP32");
  TPSS_REQUIRE(nrhs >= 1 && nrhs <= 65535, "tpss_smooth_multiplicative: nrhs out of range");
  TPSS_REQUIRE((const void*)b != (const void*)x, "tpss_smooth_multiplicative: b and x must not alias");
  return smooth_multiplicative_t<double>(P, omega, reverse_colors, nrhs, b, x);
}

extern "C" tpss_status tpss_smooth_multiplicative_f32(tpss_patches* P, float omega, int reverse_colors, int nrhs,
                                                      const float* b, float* x) {
  clear_error();
  TPSS_REQUIRE(P && b && x, "tpss_smooth_multiplicative_f32: null argument");
  TPSS_REQUIRE(P->precision != TPSS_FP64, "tpss_smooth_multiplicative_f32: patches were set up for FP64");
  TPSS_REQUIRE(nrhs >= 1 && nrhs <= 65535, "tpss_smooth_multiplicative_f32: nrhs out of range");
  TPSS_REQUIRE((const void*)b != (const void*)x, "tpss_smooth_multiplicative_f32: b and x must not alias");
  return smooth_multiplicative_t<float>(P, omega, reverse_colors, nrhs, b, x);
}
