// FP64 vertex-patch smoother for 3D subdomains with n = 2(k+1) > 16 points
// per direction (k = 8..15).  The local solve is the same fast
// diagonalization as in smoother.cu (eq. fastinverse, eq. eigenvectormatvec):
//   u = Z_x Z_y Z_z Lambda^{-1} Z_z^T Z_y^T Z_x^T R_j r,  x += omega R_j^T u,
// but the n^3 FP64 patch tensor (up to 256 KB) does not fit in shared memory,
// so it is processed in three phases:
//   1. z-planes are gathered into shared memory a few at a time, contracted
//      with Z^T along x and y there, and stored in a per-CTA global scratch
//      slab (n^3 doubles, written and re-read by the same CTA, so it stays in
//      L2);
//   2. lines along z (n^2 of them, coalesced in the slab) get Z^T, the scaling
//      by 1/(lambda_x + lambda_y + lambda_z) and Z, fused in registers;
//   3. z-planes come back into shared memory, get Z along y and x, and are
//      scattered to x.
// The kernel is persistent: one cluster of 1, 2, 4 or 8 CTAs per resident
// slot loops over (right-hand side, subdomain) work items, so the scratch is
// bounded by the number of resident CTAs, not by the mesh; the cluster size
// is chosen per launch so that few subdomains per color (multiplicative
// sweeps, small meshes) still occupy the SMs and the last round of a launch
// leaves few of them idle.  The eigenvalue sums are divided
// on the fly (n^3 divisions against 6 n^4 FMAs per subdomain) instead of
// reading an n^3-per-subdomain inverse table.
#include <algorithm>

#include "tpss_internal.cuh"

namespace tpss {

constexpr int kLargeThreads = 256;

template <int N>
struct LargeShape {
  static constexpr int N1 = N / 2;
  static constexpr int NLOC1 = N1 * N1 * N1;
  static constexpr int LS = N + 1;                    // odd line stride: conflict-free x-lines
  static constexpr int PS = LS * N;                   // one plane in shared memory
  static constexpr int PLANES = kLargeThreads / N;    // planes per group: one thread per line
  static constexpr size_t SMEM = (size_t)(3 * N * N + 3 * N + PLANES * PS) * sizeof(double);
};

struct LargeArgs {
  const double* Z[3];     // [npos_t][n*n], column j = eigenvector j
  const double* lam[3];   // [npos_t][n]
  const int* list;        // packed subdomain positions of one color
  int count;
  int nrhs;
  const double* r;
  double* x;
  double* d;              // optional: d = omega u (the update of x), and then
  double* rw;             // r *= 1 - omega on the patch's DoFs
  double omega;
  int nc0, nc1;
  int64_t ndofs;
  double* scratch;        // [clusters][n^3]
  int cs;                 // CTAs per cluster (1, 2, 4 or 8)
};

// One line of a plane in shared memory, in place:
//   TRANS = false: out_i = sum_m W[m*N + i] v_m   (Z^T v)
//   TRANS = true:  out_i = sum_m W[i*N + m] v_m   (Z v)
// All lanes of a warp read the same W entry (broadcast).
template <int N, bool TRANS>
__device__ __forceinline__ void contract_line_large(double* __restrict__ buf, const double* __restrict__ W,
                                                    int base, int stride) {
  double acc[N];
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = 0.0;
#pragma unroll 2   // full unrolling of m hoists the loads and spills the accumulators
  for (int m = 0; m < N; ++m) {
    const double v = buf[base + m * stride];
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(TRANS ? W[i * N + m] : W[m * N + i], v, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) buf[base + i * stride] = acc[i];
}

// 1/d for d > 0 in the FP32 range: a single-precision seed refined by two
// Newton-Raphson steps r <- r + r (1 - d r), each of which doubles the number
// of correct bits (24 -> 48 -> full double precision, within a couple of
// ulp).  Straight-line FMAs, unlike a double division, so the accumulators
// of the line stay in registers.
__device__ __forceinline__ double recip_newton(double d) {
  double r = (double)__frcp_rn((float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  return fma(r, fma(-d, r, 1.0), r);
}

// Barrier over the CTAs of a thread-block cluster, with release / acquire
// semantics at cluster scope (orders the global tensor slab between phases).
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// The CTAs of a cluster (a.cs of them, consecutive blockIdx.x) share one
// subdomain at a time and one tensor slab: CTA `rank` takes a contiguous
// share of the z-planes in phases 1 and 3 and of the z-lines in phase 2, with
// a cluster barrier between the phases.  Every line is contracted by exactly
// the same instructions whatever a.cs is, so the result does not depend on
// it.  a.cs = 1 is a plain (non-cluster) launch.
template <int N>
__global__ void __launch_bounds__(kLargeThreads, 2) patch_smooth_large_kernel(LargeArgs a) {
  using S = LargeShape<N>;
  constexpr int N1 = S::N1, NLOC1 = S::NLOC1, NN = N * N;
  extern __shared__ double sm_large[];
  double* Zs = sm_large;          // [3][N*N]
  double* lam = Zs + 3 * NN;      // [3][N]
  double* pl = lam + 3 * N;       // [PLANES][PS]
  const int cs = a.cs;
  const int rank = blockIdx.x % cs;
  const int cluster = blockIdx.x / cs, nclusters = gridDim.x / cs;
  double* G = a.scratch + (size_t)cluster * NN * N;
  const int tid = threadIdx.x;
  // this CTA's share of the planes and of the z-lines
  const int ppc = (N + cs - 1) / cs, lpc = (NN + cs - 1) / cs;
  const int z_lo = min(N, rank * ppc), z_hi = min(N, z_lo + ppc);
  const int l_lo = min(NN, rank * lpc), l_hi = min(NN, l_lo + lpc);
  auto sync_all = [&]() {
    if (cs > 1) cluster_barrier();
    else __syncthreads();
  };
  const int64_t items = (int64_t)a.count * a.nrhs;
  for (int64_t item = cluster; item < items; item += nclusters) {
    const int q = (int)(item % a.count);
    const int64_t vbase = (item / a.count) * a.ndofs;
    const int packed = a.list[q];
    const int px = unpack_x(packed), py = unpack_y(packed), pz = unpack_z(packed);
    sync_all();   // the previous item is done with Zs, lam, the planes and G in every CTA
    for (int e = tid; e < 3 * NN; e += kLargeThreads) {
      const int t = e / NN;
      const int p = t == 0 ? px : (t == 1 ? py : pz);
      Zs[e] = a.Z[t][(size_t)p * NN + e % NN];
    }
    for (int e = tid; e < 3 * N; e += kLargeThreads) {
      const int t = e / N;
      const int p = t == 0 ? px : (t == 1 ? py : pz);
      lam[e] = a.lam[t][(size_t)p * N + e % N];
    }
    // phase 1: gather R_j r plane by plane, Z^T along x and y, park in G
    for (int z0 = z_lo; z0 < z_hi; z0 += S::PLANES) {
      const int np = min(S::PLANES, z_hi - z0);
      __syncthreads();
      for (int e = tid; e < np * NN; e += kLargeThreads) {
        const int p = e / NN, rem = e % NN;
        const int x = rem % N, y = rem / N, z = z0 + p;
        const int64_t gcell =
            (px + x / N1) + (int64_t)a.nc0 * ((py + y / N1) + (int64_t)a.nc1 * (pz + z / N1));
        pl[p * S::PS + y * S::LS + x] = a.r[vbase + gcell * NLOC1 + (x % N1) + N1 * ((y % N1) + N1 * (z % N1))];
      }
      __syncthreads();
      if (tid < np * N) contract_line_large<N, false>(pl, Zs, (tid / N) * S::PS + (tid % N) * S::LS, 1);
      __syncthreads();
      if (tid < np * N) contract_line_large<N, false>(pl, Zs + NN, (tid / N) * S::PS + tid % N, S::LS);
      __syncthreads();
      for (int e = tid; e < np * NN; e += kLargeThreads) {
        const int p = e / NN, rem = e % NN;
        G[(size_t)(z0 + p) * NN + rem] = pl[p * S::PS + (rem / N) * S::LS + rem % N];
      }
    }
    sync_all();   // G holds every plane
    // phase 2: lines along z, Z^T -> Lambda^{-1} -> Z in registers
    {
      const double* W = Zs + 2 * NN;
      for (int line = l_lo + tid; line < l_hi; line += kLargeThreads) {
        double acc[N];
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = 0.0;
#pragma unroll 2
        for (int m = 0; m < N; ++m) {
          const double v = G[(size_t)m * NN + line];
#pragma unroll
          for (int i = 0; i < N; ++i) acc[i] = fma(W[m * N + i], v, acc[i]);
        }
        const double s0 = lam[line % N] + lam[N + line / N];
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] *= recip_newton(s0 + lam[2 * N + i]);
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
          double s = 0.0;
#pragma unroll
          for (int m = 0; m < N; ++m) s = fma(W[i * N + m], acc[m], s);
          G[(size_t)i * NN + line] = s;
        }
      }
    }
    sync_all();   // every z-line is done
    // phase 3: Z along y and x plane by plane, scatter x += omega R_j^T u
    for (int z0 = z_lo; z0 < z_hi; z0 += S::PLANES) {
      const int np = min(S::PLANES, z_hi - z0);
      __syncthreads();
      for (int e = tid; e < np * NN; e += kLargeThreads) {
        const int p = e / NN, rem = e % NN;
        pl[p * S::PS + (rem / N) * S::LS + rem % N] = G[(size_t)(z0 + p) * NN + rem];
      }
      __syncthreads();
      if (tid < np * N) contract_line_large<N, true>(pl, Zs + NN, (tid / N) * S::PS + tid % N, S::LS);
      __syncthreads();
      if (tid < np * N) contract_line_large<N, true>(pl, Zs, (tid / N) * S::PS + (tid % N) * S::LS, 1);
      __syncthreads();
      for (int e = tid; e < np * NN; e += kLargeThreads) {
        const int p = e / NN, rem = e % NN;
        const int x = rem % N, y = rem / N, z = z0 + p;
        const int64_t gcell =
            (px + x / N1) + (int64_t)a.nc0 * ((py + y / N1) + (int64_t)a.nc1 * (pz + z / N1));
        const int64_t gi = vbase + gcell * NLOC1 + (x % N1) + N1 * ((y % N1) + N1 * (z % N1));
        const double u = pl[p * S::PS + y * S::LS + x];
        a.x[gi] = fma(a.omega, u, a.x[gi]);
        if (a.d != nullptr) {
          a.d[gi] = a.omega * u;
          a.rw[gi] *= 1.0 - a.omega;
        }
      }
    }
  }
}

constexpr int kLargeClusterSizes[4] = {1, 2, 4, 8};

// Resident CTAs of the large-patch kernel (plain launch) and co-resident
// clusters for each cluster size, queried once per subdomain size.
template <int N>
struct LargeOccupancy {
  int per_sm = 0;
  int clusters[4] = {0, 0, 0, 0};
};

template <int N>
static tpss_status large_prepare(int num_sms, LargeOccupancy<N>** out) {
  static LargeOccupancy<N> occ;
  if (occ.per_sm == 0) {
    auto kern = patch_smooth_large_kernel<N>;
    TPSS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LargeShape<N>::SMEM));
    int per_sm = 0;
    TPSS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLargeThreads, LargeShape<N>::SMEM));
    if (per_sm < 1) {
      set_error("smoother: large-patch kernel cannot be resident");
      return TPSS_ECUDA;
    }
    occ.clusters[0] = per_sm * num_sms;
    for (int i = 1; i < 4; ++i) {
      const int cs = kLargeClusterSizes[i];
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs * 64);
      cfg.blockDim = dim3(kLargeThreads);
      cfg.dynamicSmemBytes = LargeShape<N>::SMEM;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = cs;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nc = 0;   // this cluster size is not available: not chosen
      }
      occ.clusters[i] = nc;
    }
    occ.per_sm = per_sm;
  }
  *out = &occ;
  return TPSS_OK;
}

// Cluster size for `items` subdomain solves: the one that keeps the most
// SMs busy over the whole launch (items x cs CTA-shares spread over
// ceil(items / clusters) rounds), the smaller on ties.
template <int N>
static int large_pick_cluster(const LargeOccupancy<N>& occ, int64_t items) {
  int best = 0;
  double best_util = 0.0;
  for (int i = 0; i < 4; ++i) {
    const int nc = occ.clusters[i];
    if (nc < 1 || kLargeClusterSizes[i] > N / 2) continue;
    const int64_t rounds = (items + nc - 1) / nc;
    const double util = (double)items * kLargeClusterSizes[i] / ((double)rounds * occ.clusters[0]);
    if (util > best_util * 1.02) {
      best_util = util;
      best = i;
    }
  }
  return best;
}

template <int N>
static tpss_status large_launch(tpss_patches* P, const int* list, int count, double omega, int nrhs,
                                const double* r, double* x, cudaStream_t s, double* d) {
  if (count <= 0) return TPSS_OK;
  LargeOccupancy<N>* occ = nullptr;
  TPSS_TRY(large_prepare<N>(P->ctx->num_sms, &occ));
  const Level& L = P->ctx->levels[P->level];
  LargeArgs a{};
  for (int t = 0; t < 3; ++t) {
    a.Z[t] = P->d_Z[t];
    a.lam[t] = P->d_lam[t];
  }
  a.list = list;
  a.count = count;
  a.nrhs = nrhs;
  a.r = r;
  a.x = x;
  a.d = d;
  a.rw = const_cast<double*>(r);
  a.omega = omega;
  a.nc0 = L.nc[0];
  a.nc1 = L.nc[1];
  a.ndofs = L.ndofs;
  a.scratch = P->d_scratch;
  const int64_t items = (int64_t)count * nrhs;
  int ci = large_pick_cluster<N>(*occ, items);
  if (P->large_cluster > 0) {   // forced (tuning / tests)
    ci = -1;
    for (int i = 0; i < 4; ++i)
      if (kLargeClusterSizes[i] == P->large_cluster && occ->clusters[i] > 0) ci = i;
    if (ci < 0) {
      set_error("smoother: requested cluster size not available for this kernel");
      return TPSS_EINVAL;
    }
  }
  const int cs = kLargeClusterSizes[ci];
  // slabs: one per cluster, never more than were allocated
  const int64_t nclusters = std::min<int64_t>({items, (int64_t)occ->clusters[ci], (int64_t)P->scratch_ctas});
  a.cs = cs;
  if (cs == 1) {
    patch_smooth_large_kernel<N><<<(unsigned)nclusters, kLargeThreads, LargeShape<N>::SMEM, s>>>(a);
    TPSS_CHECK_LAUNCH();
    return TPSS_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * cs));
  cfg.blockDim = dim3(kLargeThreads);
  cfg.dynamicSmemBytes = LargeShape<N>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = cs;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  TPSS_CHECK_CUDA(cudaLaunchKernelEx(&cfg, patch_smooth_large_kernel<N>, a));
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

// Number of resident CTAs of the large-patch kernel for subdomain size n
// (scratch slabs to allocate: at least one per cluster for any cluster
// size), or an error for sizes it does not cover.
template <int N>
static tpss_status large_ctas(int num_sms, int* max_ctas) {
  LargeOccupancy<N>* occ = nullptr;
  TPSS_TRY(large_prepare<N>(num_sms, &occ));
  *max_ctas = occ->clusters[0];
  return TPSS_OK;
}

tpss_status patch_large_ctas(int n, int num_sms, int* max_ctas) {
  switch (n) {
    case 18: return large_ctas<18>(num_sms, max_ctas);
    case 20: return large_ctas<20>(num_sms, max_ctas);
    case 22: return large_ctas<22>(num_sms, max_ctas);
    case 24: return large_ctas<24>(num_sms, max_ctas);
    case 26: return large_ctas<26>(num_sms, max_ctas);
    case 28: return large_ctas<28>(num_sms, max_ctas);
    case 30: return large_ctas<30>(num_sms, max_ctas);
    case 32: return large_ctas<32>(num_sms, max_ctas);
    default:
      set_error("smoother: no large-patch kernel for this subdomain size");
      return TPSS_EINVAL;
  }
}

tpss_status patch_pass_large(tpss_patches* P, const int* list, int count, double omega, int nrhs,
                             const double* r, double* x, cudaStream_t s, double* d) {
  if (P->d_scratch == nullptr || P->scratch_ctas < 1) {
    set_error("smoother: large-patch scratch missing");
    return TPSS_EINVAL;
  }
  switch (P->n) {
    case 18: return large_launch<18>(P, list, count, omega, nrhs, r, x, s, d);
    case 20: return large_launch<20>(P, list, count, omega, nrhs, r, x, s, d);
    case 22: return large_launch<22>(P, list, count, omega, nrhs, r, x, s, d);
    case 24: return large_launch<24>(P, list, count, omega, nrhs, r, x, s, d);
    case 26: return large_launch<26>(P, list, count, omega, nrhs, r, x, s, d);
    case 28: return large_launch<28>(P, list, count, omega, nrhs, r, x, s, d);
    case 30: return large_launch<30>(P, list, count, omega, nrhs, r, x, s, d);
    case 32: return large_launch<32>(P, list, count, omega, nrhs, r, x, s, d);
    default:
      set_error("smoother: no large-patch kernel for this subdomain size");
      return TPSS_EINVAL;
  }
}

}  // namespace tpss
