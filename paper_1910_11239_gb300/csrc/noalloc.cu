// Allocation-free variant of the matrix-free operator.
//
// tpss_apply_operator keeps its three-pass intermediates in per-level scratch
// that the library allocates with cudaMalloc the first time a level is used
// with a given number of right-hand sides (and grows later, with a stream
// synchronization).  Some callers cannot have that happen: code whose device
// memory is entirely reserved by another allocator (for example a framework's
// caching allocator), or latency-critical loops in which an allocation and
// the device synchronization it implies are not acceptable.  For them,
// tpss_apply_operator_noalloc runs the same kernels with the intermediates in
// one fixed, statically allocated device array instead.
//
// The array holds kNoAllocMaxEntries * 4 doubles (16 MiB) and is reserved on
// every GPU that loads this library for as long as the process lives.  All
// calls share it: each pass overwrites what it uses, so nothing has to be
// cleared between calls, but two calls that overlap on the GPU (for example
// on two streams) would overwrite each other's intermediates.
#include <mutex>

#include "tpss_internal.cuh"

namespace tpss {

tpss_status apply_operator_into(tpss_ctx* ctx, int level, int nrhs, const double* u, double* out,
                                double* const* tmp);

namespace {

constexpr int64_t kNoAllocMaxEntries = int64_t(1) << 19;  // ndofs * nrhs per call
constexpr int kNoAllocVectors = 4;                        // a, b, p, q of the three passes

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocVectors * kNoAllocMaxEntries];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device; the host-side symbol is only a stand-in, never a device address).
tpss_status scratch_address(double** out) {
  int dev = 0;
  TPSS_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("tpss_apply_operator_noalloc: device index out of range");
    return TPSS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    TPSS_CHECK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TPSS_OK;
}

}  // namespace
}  // namespace tpss

using namespace tpss;

extern "C" tpss_status tpss_apply_operator_noalloc(tpss_ctx* ctx, int level, int nrhs, const double* u,
                                                   double* Au) {
  clear_error();
  TPSS_REQUIRE(ctx && u && Au, "tpss_apply_operator_noalloc: null argument");
  TPSS_REQUIRE(level >= 0 && level < ctx->nlevels, "tpss_apply_operator_noalloc: level out of range");
  TPSS_REQUIRE(nrhs >= 1, "tpss_apply_operator_noalloc: nrhs must be >= 1");
  TPSS_REQUIRE(u != Au, "tpss_apply_operator_noalloc: u and Au must not alias");
  // A mesh of quadrilaterals / hexahedra uses a single-pass operator with no
  // intermediates at all: no scratch, hence no size limit.
  if (ctx->mapped) return apply_operator_into(ctx, level, nrhs, u, Au, nullptr);
  const int64_t entries = ctx->levels[level].ndofs * (int64_t)nrhs;
  if (entries > kNoAllocMaxEntries) {
    set_error("tpss_apply_operator_noalloc: ndofs * nrhs = " + std::to_string(entries) +
              " exceeds the fixed scratch limit of " + std::to_string(kNoAllocMaxEntries));
    return TPSS_EINVAL;
  }
  double* base = nullptr;
  TPSS_TRY(scratch_address(&base));
  double* tmp[kNoAllocVectors];
  for (int i = 0; i < kNoAllocVectors; ++i) tmp[i] = base + (int64_t)i * entries;
  return apply_operator_into(ctx, level, nrhs, u, Au, tmp);
}
