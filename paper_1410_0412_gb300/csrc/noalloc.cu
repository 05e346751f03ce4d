// lbm_macroscopic_noalloc: the macroscopic read-back and FP64 global sums of
// lbm_macroscopic, for callers that cannot allocate device memory.
//
// lbm_macroscopic needs a caller-provided device workspace for its per-block
// partial sums.  Some callers cannot obtain one: a host application that has
// handed all device memory to its own pool allocator, or a tight loop in which
// a cudaMalloc (which may synchronise the device) is not allowed.  This entry
// point instead keeps the partial sums in a fixed array that lives in the
// library's own device memory for as long as the library is loaded.
//
// Limits and behaviour:
//  - at most kNoAllocMaxNodes fluid nodes (the array holds one 4-double
//    partial per 128-node block: 4 MiB on every GPU that loads the library);
//    larger lattices are rejected with LBM_ERR_ARG;
//  - the first call on a device looks up the array's device address (with that
//    device current) and caches it; make that first call before any stream
//    capture.  The cache assumes the device's primary context lives as long
//    as the process: after cudaDeviceReset (or anything else that destroys
//    that context) the cached address is stale, so do not call this entry
//    point across a reset;
//  - every call shares the one array: calls whose kernels overlap on the GPU
//    (e.g. on two streams without ordering) race on it and may return wrong
//    sums.  Every partial a call reads is written by the same call first, so no
//    clearing is needed between calls;
//  - it allocates nothing: no cudaMalloc, cudaFree or allocating library call.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace lbm {

constexpr int64_t kNoAllocMaxNodes = int64_t(1) << 24;
constexpr int64_t kNoAllocMaxParts = kNoAllocMaxNodes / 128;

namespace {

static __device__ __align__(256) double g_partials[kNoAllocMaxParts * 4];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_partials_addr[kMaxDevices] = {nullptr};

// Device address of g_partials on the current device (looked up once per device).
int partials_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(LBM_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess || !p)
      return set_error(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_macroscopic_noalloc(const lbm_lattice* L, int prec, const lbm_params* params, const void* pdf,
                                       int layout, const float* s, double* rho, double* u, double* sums,
                                       void* stream) {
  // the same checks as lbm_macroscopic, then the size limit of the fixed array
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (int rc = check_layout(layout)) return rc;
  if (!pdf) return set_error(LBM_ERR_ARG, "pdf is NULL");
  if (L->N > kNoAllocMaxNodes)
    return set_error(LBM_ERR_ARG, "lbm_macroscopic_noalloc handles at most 16777216 fluid nodes; "
                                  "use lbm_macroscopic with a workspace");
  if (int rc = layout_tables(L, layout)) return rc;
  double* partials = nullptr;
  if (int rc = partials_on_current_device(&partials)) return rc;
  const int64_t parts = reduce_parts(L);
  return LBM_DISPATCH(prec, launch_macroscopic_t, L, kp, pdf, layout, s, rho, u, sums, partials, parts, stream);
}
