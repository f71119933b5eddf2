// Matrix-free SIPG operator (eq. bfsipg) on Cartesian tensor grids.
//
// On a Cartesian grid the global SIPG matrix is the Kronecker sum of 1D DG
// matrices (Sec. 3.2, eq. KDseparable applied to the whole grid):
//   A = sum_t M_g x ... x A_g^(t) x ... x M_g,
// where M_g is block diagonal (cell mass matrices M_t(c)) and A_g^(t) is block
// tridiagonal: the cell blocks A_t(c) of eq. 1Dsipg plus the interface
// couplings of eq. 1DsipgVP, which in the Gauss-Lobatto nodal basis touch only
// the end value and the end derivative of the neighbour's line (rank 2).
// Sum factorization (Sec. 3.1) is applied in three passes (two in 2D):
//   pass x:  a = A_x u,            b = M_x u
//   pass y:  p = M_y a + A_y b,    q = M_y b           (3D only)
//   pass z:  y = M_z p + A_z q                          (y = M_y a + A_y b in 2D)
// so y = M_z M_y A_x u + M_z A_y M_x u + A_z M_y M_x u, 7 (k+1)^4 FMAs per cell
// in 3D plus O((k+1)^3) for faces.  Each pass runs one thread per
// (right-hand side, cell, line along the pass direction); the neighbour
// coupling of a pass reads the neighbour's line of the pass's "A" operand.
// The last pass optionally fuses the residual r = rhs - y.
#include "tpss_internal.cuh"

namespace tpss {

enum PassKind { kPassFirst = 0, kPassMid = 1, kPassLast = 2 };

template <typename T>
struct PassArgs {
  const T* inA;      // operand of the M_t product (u for the first pass)
  const T* inB;      // operand of the A_t product (u for the first pass)
  T* outA;           // first pass: a (= A_x u); mid: p; last: y or r
  T* outB;           // first pass: b (= M_x u); mid: q
  const T* rhs;      // last pass: residual right-hand side (nullptr = plain y)
  const T* M;        // M_t(c), [nc_t][n1*n1]
  const T* A;        // A_t(c)
  const T* F;        // face coefficients [nc_t][kFaceCoef]
  const T* d0;
  const T* d1;
  int nc0, nc1, nc2;
  int64_t ncells;
  int64_t ndofs;
  int nrhs;
};

// local offset of element m of line `line` in direction t (cell data, x fastest)
template <int DIM, int N1, int DIR>
__device__ __forceinline__ int line_base(int line) {
  if (DIR == 0) return line * N1;
  if (DIM == 2) return line;           // DIR == 1 in 2D
  if (DIR == 1) return (line % N1) + N1 * N1 * (line / N1);
  return line;                         // DIR == 2
}
template <int DIM, int N1, int DIR>
__device__ __forceinline__ constexpr int line_stride() {
  return DIR == 0 ? 1 : (DIR == 1 ? N1 : N1 * N1);
}

template <int DIM, int N1, int DIR, int KIND, typename T>
__global__ void __launch_bounds__(256) op_pass_kernel(PassArgs<T> P) {
  constexpr int LINES = DIM == 3 ? N1 * N1 : N1;
  constexpr int NLOC = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
  constexpr int S = line_stride<DIM, N1, DIR>();
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = P.ncells * LINES * P.nrhs;
  if (tid >= total) return;
  const int line = (int)(tid % LINES);
  const int64_t cr = tid / LINES;           // rhs * ncells + cell
  const int64_t cell = cr % P.ncells;
  const int64_t rhs = cr / P.ncells;
  int cpos, ncdir;
  int64_t cstride;
  if (DIR == 0) {
    cpos = (int)(cell % P.nc0); ncdir = P.nc0; cstride = 1;
  } else if (DIR == 1) {
    cpos = (int)((cell / P.nc0) % P.nc1); ncdir = P.nc1; cstride = P.nc0;
  } else {
    cpos = (int)(cell / ((int64_t)P.nc0 * P.nc1)); ncdir = P.nc2; cstride = (int64_t)P.nc0 * P.nc1;
  }
  const int64_t vbase = rhs * P.ndofs;
  const int64_t off = vbase + cell * NLOC + line_base<DIM, N1, DIR>(line);
  const T* Mc = P.M + (size_t)cpos * N1 * N1;
  const T* Ac = P.A + (size_t)cpos * N1 * N1;

  T vb[N1];  // operand of A_t
#pragma unroll
  for (int m = 0; m < N1; ++m) vb[m] = P.inB[off + m * S];
  T outa[N1], outb[N1];
  if (KIND == kPassFirst) {
    // a = A u, b = M u  (inA == inB == u)
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      T sa = 0, sb = 0;
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        sa = fma(__ldg(Ac + i * N1 + j), vb[j], sa);
        sb = fma(__ldg(Mc + i * N1 + j), vb[j], sb);
      }
      outa[i] = sa;
      outb[i] = sb;
    }
  } else {
    T va[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) va[m] = P.inA[off + m * S];
    // outa = M va + A vb ; outb = M vb (mid pass only)
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      T sa = 0, sb = 0;
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        const T mij = __ldg(Mc + i * N1 + j);
        sa = fma(mij, va[j], sa);
        sa = fma(__ldg(Ac + i * N1 + j), vb[j], sa);
        if (KIND == kPassMid) sb = fma(mij, vb[j], sb);
      }
      outa[i] = sa;
      if (KIND == kPassMid) outb[i] = sb;
    }
  }
  // face couplings of A_t to the neighbours' lines of the same operand
  const T* f = P.F + (size_t)cpos * kFaceCoef;
  if (cpos + 1 < ncdir) {
    const int64_t noff = off + cstride * NLOC;
    T s1 = 0;
#pragma unroll
    for (int j = 0; j < N1; ++j) s1 = fma(__ldg(P.d0 + j), P.inB[noff + j * S], s1);
    const T s0 = P.inB[noff];
    outa[N1 - 1] += __ldg(f + 0) * s0 + __ldg(f + 1) * s1;
    const T c = __ldg(f + 2) * s0;
#pragma unroll
    for (int i = 0; i < N1; ++i) outa[i] = fma(__ldg(P.d1 + i), c, outa[i]);
  }
  if (cpos > 0) {
    const int64_t noff = off - cstride * NLOC;
    T t1 = 0;
#pragma unroll
    for (int j = 0; j < N1; ++j) t1 = fma(__ldg(P.d1 + j), P.inB[noff + j * S], t1);
    const T t0 = P.inB[noff + (N1 - 1) * S];
    outa[0] += __ldg(f + 3) * t0 + __ldg(f + 4) * t1;
    const T c = __ldg(f + 5) * t0;
#pragma unroll
    for (int i = 0; i < N1; ++i) outa[i] = fma(__ldg(P.d0 + i), c, outa[i]);
  }
  if (KIND == kPassLast && P.rhs != nullptr) {
#pragma unroll
    for (int i = 0; i < N1; ++i) P.outA[off + i * S] = P.rhs[off + i * S] - outa[i];
  } else {
#pragma unroll
    for (int i = 0; i < N1; ++i) P.outA[off + i * S] = outa[i];
  }
  if (KIND != kPassLast) {
#pragma unroll
    for (int i = 0; i < N1; ++i) P.outB[off + i * S] = outb[i];
  }
}

template <int DIM, int N1, int DIR, int KIND, typename T>
static tpss_status launch_pass(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int LINES = DIM == 3 ? N1 * N1 : N1;
  const int64_t total = a.ncells * LINES * a.nrhs;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 0x7fffffff) {
    set_error("operator: grid too large");
    return TPSS_EINVAL;
  }
  op_pass_kernel<DIM, N1, DIR, KIND, T><<<(unsigned)blocks, threads, 0, s>>>(a);
  TPSS_CHECK_LAUNCH();
  return TPSS_OK;
}

template <int DIM, int N1, typename T>
static tpss_status apply_n(tpss_ctx* ctx, Level& L, const LevelOps<T>& op, T* const* tmp, int nrhs,
                           const T* u, T* out, const T* rhs) {
  PassArgs<T> a{};
  a.d0 = op.d0;
  a.d1 = op.d1;
  a.nc0 = L.nc[0];
  a.nc1 = L.nc[1];
  a.nc2 = DIM == 3 ? L.nc[2] : 1;
  a.ncells = L.ncells;
  a.ndofs = L.ndofs;
  a.nrhs = nrhs;
  // pass x: a = A_x u -> tmp0, b = M_x u -> tmp1
  a.inA = u; a.inB = u; a.outA = tmp[0]; a.outB = tmp[1]; a.rhs = nullptr;
  a.M = op.M[0]; a.A = op.A[0]; a.F = op.F[0];
  TPSS_TRY((launch_pass<DIM, N1, 0, kPassFirst, T>(a, ctx->stream)));
  if (DIM == 3) {
    // pass y: p = M_y a + A_y b -> tmp2, q = M_y b -> tmp3
    a.inA = tmp[0]; a.inB = tmp[1]; a.outA = tmp[2]; a.outB = tmp[3];
    a.M = op.M[1]; a.A = op.A[1]; a.F = op.F[1];
    TPSS_TRY((launch_pass<DIM, N1, 1, kPassMid, T>(a, ctx->stream)));
    // pass z: y = M_z p + A_z q
    a.inA = tmp[2]; a.inB = tmp[3]; a.outA = out; a.outB = nullptr; a.rhs = rhs;
    a.M = op.M[2]; a.A = op.A[2]; a.F = op.F[2];
    TPSS_TRY((launch_pass<DIM, N1, 2, kPassLast, T>(a, ctx->stream)));
  } else {
    a.inA = tmp[0]; a.inB = tmp[1]; a.outA = out; a.outB = nullptr; a.rhs = rhs;
    a.M = op.M[1]; a.A = op.A[1]; a.F = op.F[1];
    TPSS_TRY((launch_pass<DIM, N1, 1, kPassLast, T>(a, ctx->stream)));
  }
  return TPSS_OK;
}

template <typename T>
static const LevelOps<T>& ops_of(const Level& L);
template <>
const LevelOps<double>& ops_of<double>(const Level& L) { return L.op64; }
template <>
const LevelOps<float>& ops_of<float>(const Level& L) { return L.op32; }
template <typename T>
static T* const* tmp_of(const Level& L);
template <>
double* const* tmp_of<double>(const Level& L) { return L.t64; }
template <>
float* const* tmp_of<float>(const Level& L) { return L.t32; }

template <typename T>
tpss_status apply_operator_t(tpss_ctx* ctx, int level, int nrhs, const T* u, T* out, const T* rhs) {
  if (ctx->mapped) return mapped_apply_t<T>(ctx, level, nrhs, u, out, rhs);
  TPSS_TRY(ensure_level_scratch(ctx, level, nrhs));
  Level& L = ctx->levels[level];
  const LevelOps<T>& op = ops_of<T>(L);
  T* const* tmp = tmp_of<T>(L);
#define TPSS_OP_CASE(D, N)                                                  \
  if (ctx->dim == D && ctx->n1 == N) return apply_n<D, N, T>(ctx, L, op, tmp, nrhs, u, out, rhs);
  TPSS_OP_CASE(3, 2) TPSS_OP_CASE(3, 3) TPSS_OP_CASE(3, 4) TPSS_OP_CASE(3, 5)
  TPSS_OP_CASE(3, 6) TPSS_OP_CASE(3, 7) TPSS_OP_CASE(3, 8)
  TPSS_OP_CASE(2, 2) TPSS_OP_CASE(2, 3) TPSS_OP_CASE(2, 4) TPSS_OP_CASE(2, 5)
  TPSS_OP_CASE(2, 6) TPSS_OP_CASE(2, 7) TPSS_OP_CASE(2, 8)
  if constexpr (sizeof(T) == sizeof(double)) {   // degrees 8..15: FP64 only
    TPSS_OP_CASE(3, 9) TPSS_OP_CASE(3, 10) TPSS_OP_CASE(3, 11) TPSS_OP_CASE(3, 12)
    TPSS_OP_CASE(3, 13) TPSS_OP_CASE(3, 14) TPSS_OP_CASE(3, 15) TPSS_OP_CASE(3, 16)
    TPSS_OP_CASE(2, 9) TPSS_OP_CASE(2, 10) TPSS_OP_CASE(2, 11) TPSS_OP_CASE(2, 12)
    TPSS_OP_CASE(2, 13) TPSS_OP_CASE(2, 14) TPSS_OP_CASE(2, 15) TPSS_OP_CASE(2, 16)
  }
#undef TPSS_OP_CASE
  set_error(sizeof(T) == sizeof(double) ? "operator: unsupported degree"
                                        : "operator: FP32 operators support degrees up to 7");
  return TPSS_EINVAL;
}


// The operator with caller-provided intermediates (four vectors of
// ndofs * nrhs doubles); used by the allocation-free entry point.
tpss_status apply_operator_into(tpss_ctx* ctx, int level, int nrhs, const double* u, double* out,
                                double* const* tmp) {
  if (ctx->mapped) return mapped_apply_t<double>(ctx, level, nrhs, u, out, nullptr);
  Level& L = ctx->levels[level];
  const LevelOps<double>& op = L.op64;
#define TPSS_OPI_CASE(D, N)                                                  \
  if (ctx->dim == D && ctx->n1 == N) return apply_n<D, N, double>(ctx, L, op, tmp, nrhs, u, out, nullptr);
  TPSS_OPI_CASE(3, 2) TPSS_OPI_CASE(3, 3) TPSS_OPI_CASE(3, 4) TPSS_OPI_CASE(3, 5)
  TPSS_OPI_CASE(3, 6) TPSS_OPI_CASE(3, 7) TPSS_OPI_CASE(3, 8)
  TPSS_OPI_CASE(2, 2) TPSS_OPI_CASE(2, 3) TPSS_OPI_CASE(2, 4) TPSS_OPI_CASE(2, 5)
  TPSS_OPI_CASE(2, 6) TPSS_OPI_CASE(2, 7) TPSS_OPI_CASE(2, 8)
  TPSS_OPI_CASE(3, 9) TPSS_OPI_CASE(3, 10) TPSS_OPI_CASE(3, 11) TPSS_OPI_CASE(3, 12)
  TPSS_OPI_CASE(3, 13) TPSS_OPI_CASE(3, 14) TPSS_OPI_CASE(3, 15) TPSS_OPI_CASE(3, 16)
  TPSS_OPI_CASE(2, 9) TPSS_OPI_CASE(2, 10) TPSS_OPI_CASE(2, 11) TPSS_OPI_CASE(2, 12)
  TPSS_OPI_CASE(2, 13) TPSS_OPI_CASE(2, 14) TPSS_OPI_CASE(2, 15) TPSS_OPI_CASE(2, 16)
#undef TPSS_OPI_CASE
  set_error("operator: unsupported degree");
  return TPSS_EINVAL;
}

template tpss_status apply_operator_t<double>(tpss_ctx*, int, int, const double*, double*, const double*);
template tpss_status apply_operator_t<float>(tpss_ctx*, int, int, const float*, float*, const float*);

}  // namespace tpss

using namespace tpss;

extern "C" tpss_status tpss_apply_operator(tpss_ctx* ctx, int level, int nrhs, const double* u, double* Au) {
  clear_error();
  TPSS_REQUIRE(ctx && u && Au, "tpss_apply_operator: null argument");
  TPSS_REQUIRE(level >= 0 && level < ctx->nlevels, "tpss_apply_operator: level out of range");
  TPSS_REQUIRE(nrhs >= 1, "tpss_apply_operator: nrhs must be >= 1");
  TPSS_REQUIRE(u != Au, "tpss_apply_operator: u and Au must not alias");
  return apply_operator_t<double>(ctx, level, nrhs, u, Au, nullptr);
}

extern "C" tpss_status tpss_apply_operator_f32(tpss_ctx* ctx, int level, int nrhs, const float* u, float* Au) {
  clear_error();
  TPSS_REQUIRE(ctx && u && Au, "tpss_apply_operator_f32: null argument");
  TPSS_REQUIRE(level >= 0 && level < ctx->nlevels, "tpss_apply_operator_f32: level out of range");
  TPSS_REQUIRE(nrhs >= 1, "tpss_apply_operator_f32: nrhs must be >= 1");
  TPSS_REQUIRE(u != Au, "tpss_apply_operator_f32: u and Au must not alias");
  return apply_operator_t<float>(ctx, level, nrhs, u, Au, nullptr);
}

extern "C" tpss_status tpss_residual(tpss_ctx* ctx, int level, int nrhs, const double* b, const double* x,
                                     double* r) {
  clear_error();
  TPSS_REQUIRE(ctx && b && x && r, "tpss_residual: null argument");
  TPSS_REQUIRE(level >= 0 && level < ctx->nlevels, "tpss_residual: level out of range");
  TPSS_REQUIRE(nrhs >= 1, "tpss_residual: nrhs must be >= 1");
  TPSS_REQUIRE(r != x, "tpss_residual: r must not alias x");
  return apply_operator_t<double>(ctx, level, nrhs, x, r, b);
}
