// Streaming micro-benchmarks whose access patterns match the propagation steps
// (the paper's Sect. 5.2, Table 3): they supply pattern-specific bandwidths
// for the roofline P = b / B_l.
//   CNT-kA: k arrays copied into k others with streaming (evict-first) stores,
//           the access pattern of the OS-NT step (19 reads + 19 NT stores).
//   U-kA:   k arrays updated in place (read, write back), the access pattern of
//           the AA even step.
// The arrays are [k][n] slices of one buffer, like the SoA PDF grids.
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

}  // namespace dev
}  // namespace lbm

using namespace lbm;

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
