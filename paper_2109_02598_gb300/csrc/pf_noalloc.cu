// pf_reduce_noalloc: the mass / free-energy reduction of pf_reduce for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that has already reserved all of
// the device's memory for its own allocator (so any allocation from this library would
// fail or fragment its pool), or a latency-critical loop where cudaMalloc's implicit
// device-wide synchronisation is not acceptable.  This entry point runs the same two
// reduction kernels as pf_reduce, on a field the caller owns, writing the result to a
// device double the caller owns; the only other memory it touches is a fixed scratch
// array of kReduceBlocks (512) FP64 partial sums (4 KiB) defined below, which exists on
// every GPU that loads the library until the process exits.
//
// The scratch is a file-scope __device__ array.  In host code its name only stands in
// for the symbol; its device address is fetched once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on that device,
// and cached.  Make that first call before any stream capture.  Under CUDA's lazy module
// loading (the default) that first call is also where the library's modules are loaded on
// the device, which allocates device memory for their code and for this array and may
// synchronise; a warm-up call before the caller's allocator takes the device avoids that.
// The cached address belongs to the device's primary context: after cudaDeviceReset it no
// longer exists, so this entry point must not be called again in that process.
//
// Every call on a device shares the one array.  Each call writes all 512 partials before
// reading any of them, so no stale contents from the previous call are used and nothing
// needs clearing; but two calls whose kernels overlap on the GPU (e.g. on two streams
// without ordering) race on the array and may return wrong sums.
#include <cmath>
#include <mutex>

#include "pf_internal.h"

namespace pf {
int invalid(const char* fmt, ...);
}

namespace {

static __device__ __align__(256) double g_noalloc_partials[pf::kReduceBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pf::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return pf::invalid("device ordinal %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return pf::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return PF_OK;
}

}  // namespace

extern "C" int pf_reduce_noalloc(int what, int dim, const int64_t* n, int64_t pitch,
                                 const float* field, double h, double c1, double c2,
                                 double* out_dev, void* stream) {
  using namespace pf;
  if (what != PF_REDUCE_MASS && what != PF_REDUCE_ENERGY)
    return invalid("pf_reduce_noalloc: unknown reduction %d", what);
  if (dim != 2 && dim != 3) return invalid("pf_reduce_noalloc: dim must be 2 or 3 (got %d)", dim);
  if (n == nullptr || field == nullptr || out_dev == nullptr)
    return invalid("pf_reduce_noalloc: n, field and out_dev must not be NULL");
  const int64_t nz = dim == 3 ? n[2] : 1;
  const int64_t lim = (int64_t)1 << 30;
  if (n[0] < 1 || n[1] < 1 || nz < 1 || n[0] > lim || n[1] > lim || nz > lim)
    return invalid("pf_reduce_noalloc: sizes must be in [1, 2^30] (got %lld x %lld x %lld)",
                   (long long)n[0], (long long)n[1], (long long)nz);
  if (pitch < n[0]) return invalid("pf_reduce_noalloc: pitch %lld < nx %lld", (long long)pitch,
                                   (long long)n[0]);
  // pitch, ny, nz <= 2^30 each: pitch * ny fits in int64, and the plane count is compared
  // by division, so no product can overflow
  const int64_t max_elems = (int64_t)1 << 36;
  if (pitch > lim || pitch * n[1] > max_elems || nz > max_elems / (pitch * n[1]))
    return invalid("pf_reduce_noalloc: field of %lld x %lld x %lld floats exceeds the 2^36 "
                   "maximum", (long long)pitch, (long long)n[1], (long long)nz);
  if (!(h > 0.0) || !std::isfinite(h)) return invalid("pf_reduce_noalloc: h must be finite and > 0");
  double* scratch = nullptr;
  if (int rc = scratch_for_current_device(&scratch)) return rc;
  Geom g{};
  g.dim = dim;
  g.nx = (int)n[0];
  g.ny = (int)n[1];
  g.nz = (int)nz;
  g.pitch = pitch;
  g.plane = pitch * n[1];
  PF_CUDA_TRY(launch_reduce(what, g, field, c1, c2, h, scratch, out_dev, (cudaStream_t)stream));
  return PF_OK;
}
