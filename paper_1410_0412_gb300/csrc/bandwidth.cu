// Streaming micro-benchmarks whose access patterns match the propagation steps
// (the paper's Sect. 5.2, Table 3): they supply pattern-specific bandwidths
// for the roofline P = b / B_l.
//   CNT-kA: k arrays copied into k others with streaming (evict-first) stores,
//           the access pattern of the OS-NT step (19 reads + 19 NT stores).
//   U-kA:   k arrays updated in place (read, write back), the access pattern of
//           the AA even step.
// The arrays are [k][n] slices of one buffer, like the SoA PDF grids.
// A third kernel measures the FP64 pipe's throughput, the compute roof of the
// native FP64 step on this GPU.
#include <cuda_runtime.h>

#include "internal.h"

namespace lbm {
namespace dev {

constexpr int kBwBlock = 256;

// 16-byte vectors per thread, grid-stride over n / 4 float4 per array.
__global__ void __launch_bounds__(kBwBlock) k_bw_copy(const float4* __restrict__ src, float4* __restrict__ dst,
                                                       int64_t n4, int k) {
  for (int64_t e = blockIdx.x * int64_t(kBwBlock) + threadIdx.x; e < n4; e += int64_t(gridDim.x) * kBwBlock)
    for (int a = 0; a < k; ++a) __stcs(dst + a * n4 + e, __ldg(src + a * n4 + e));
}

__global__ void __launch_bounds__(kBwBlock) k_bw_update(float4* __restrict__ buf, int64_t n4, int k) {
  for (int64_t e = blockIdx.x * int64_t(kBwBlock) + threadIdx.x; e < n4; e += int64_t(gridDim.x) * kBwBlock)
    for (int a = 0; a < k; ++a) {
      float4 v = buf[a * n4 + e];
      v.x += 1.0f;
      v.y += 1.0f;
      v.z += 1.0f;
      v.w += 1.0f;
      buf[a * n4 + e] = v;
    }
}

// FP64 pipe throughput: kFmaChains independent DFMA chains per thread, iters
// steps each, x <- fma(x, a, b).  With a = b = 1 every chain counts up by one
// per step exactly (integers below 2^53), so the output is checkable:
// out[t] = sum over chains c of (t mod 1024 + c + iters).
constexpr int kFmaChains = 8;

__global__ void __launch_bounds__(kBwBlock) k_fp64_peak(double* __restrict__ out, double a, double b, int iters) {
  const int64_t t = blockIdx.x * int64_t(kBwBlock) + threadIdx.x;
  double x[kFmaChains];
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) x[c] = double(t % 1024) + c;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = ::fma(x[c], a, b);
  }
  double sum = 0.0;
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) sum += x[c];
  out[t] = sum;
}

}  // namespace dev
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_fp64_peak_kernel(double* out, int64_t threads, int iters, void* stream) {
  if (!out) return set_error(LBM_ERR_ARG, "out is NULL");
  if (threads < dev::kBwBlock || threads % dev::kBwBlock || threads > (int64_t(1) << 31))
    return set_error(LBM_ERR_ARG, "threads must be a positive multiple of 256, at most 2^31");
  if (iters < 1 || iters > (1 << 24)) return set_error(LBM_ERR_ARG, "iters must lie in [1, 2^24]");
  auto st = static_cast<cudaStream_t>(stream);
  dev::k_fp64_peak<<<unsigned(threads / dev::kBwBlock), dev::kBwBlock, 0, st>>>(out, 1.0, 1.0, iters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("fp64 peak kernel: ") + cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" int lbm_bandwidth_kernel(int kind, const void* src, void* dst, int64_t bytes_per_array, int arrays,
                                    void* stream) {
  if (kind != 0 && kind != 1) return set_error(LBM_ERR_ARG, "kind must be 0 (copy) or 1 (update)");
  if (arrays < 1 || bytes_per_array < 16 || bytes_per_array % 16)
    return set_error(LBM_ERR_ARG, "arrays >= 1 and bytes_per_array a positive multiple of 16");
  if (!dst || (kind == 0 && !src)) return set_error(LBM_ERR_ARG, "buffer is NULL");
  if ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) % 16)
    return set_error(LBM_ERR_ARG, "buffers must be 16-byte aligned");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n4 = bytes_per_array / 16;
  const unsigned grid = unsigned(std::max(1, sms) * 8);  // 8 CTAs of 256 threads per SM, grid-stride
  auto st = static_cast<cudaStream_t>(stream);
  if (kind == 0)
    dev::k_bw_copy<<<grid, dev::kBwBlock, 0, st>>>(static_cast<const float4*>(src), static_cast<float4*>(dst), n4,
                                                    arrays);
  else
    dev::k_bw_update<<<grid, dev::kBwBlock, 0, st>>>(static_cast<float4*>(dst), n4, arrays);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("bandwidth kernel: ") + cudaGetErrorString(e));
  return LBM_OK;
}
