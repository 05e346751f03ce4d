// Ghost-PDF exchange between the partitions of one lattice (Sect. 6).
//
// Every step, each partition needs the PDFs its nodes pull from nodes of other
// partitions.  The exchange table lists them grouped by (receiver, owner); one
// CTA copies up to kHaloBlock of them between one pair of grids, so on a
// machine with one partition per GPU the same kernel would read the owner's
// grid through a peer mapping.  Here all grids share one GPU.
//
// Which direction array a ghost slot lives in depends on the step form:
//  * OS-NT pulls P_i from adj[i][n]: slot s of array i receives the owner's
//    post-collision P_i at node m (LBM_HALO_OSNT, before the step);
//  * the AA odd step reads A[inv i][adj[i][n]] and writes its result back
//    into the same slot, so slot s of array inv(i) is filled from the owner
//    before the odd step (LBM_HALO_AA_GATHER) and returned to it afterwards
//    (LBM_HALO_AA_SCATTER).  The AA even step touches local slots only.
// Entries of one partition have distinct (array, slot) pairs, and their
// sources are distinct (array, node) pairs of the owner (pull reciprocity), so
// neither direction of copy has two writers to one element.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace lbm {
namespace {

__device__ __forceinline__ int inv_dir(int i) { return (i & 1) ? i + 1 : i - 1; }

template <typename T, int MODE>
__global__ void __launch_bounds__(kHaloBlock) k_halo(HaloDev h, T* const* __restrict__ grids) {
  const int32_t grp = h.blk_group[blockIdx.x];
  const int64_t e = int64_t(h.blk_first[blockIdx.x]) + threadIdx.x;
  if (e >= h.grp_end[grp]) return;
  const uint32_t ds = h.e_dirslot[e];
  const int i = int(ds >> kSlotBits) + 1;  // pulled PDF, 1..18
  const int64_t slot = int64_t(ds & ((1u << kSlotBits) - 1u));
  const int p = h.grp_p[grp], q = h.grp_q[grp];
  const int a = MODE == LBM_HALO_OSNT ? i : inv_dir(i);
  T* local = grids[p] + int64_t(a) * h.npad[p] + slot;
  T* remote = grids[q] + int64_t(a) * h.npad[q] + h.e_node[e];
  if (MODE == LBM_HALO_AA_SCATTER)
    *remote = *local;
  else
    *local = *remote;
}

template <typename T>
cudaError_t launch_mode(const HaloDev& d, void* const* grids, int mode, cudaStream_t st) {
  T* const* g = reinterpret_cast<T* const*>(grids);
  const unsigned nb = unsigned(d.B);
  if (mode == LBM_HALO_OSNT)
    k_halo<T, LBM_HALO_OSNT><<<nb, kHaloBlock, 0, st>>>(d, g);
  else if (mode == LBM_HALO_AA_GATHER)
    k_halo<T, LBM_HALO_AA_GATHER><<<nb, kHaloBlock, 0, st>>>(d, g);
  else
    k_halo<T, LBM_HALO_AA_SCATTER><<<nb, kHaloBlock, 0, st>>>(d, g);
  return cudaGetLastError();
}

}  // namespace

int launch_halo(const lbm_partitioning* S, int prec, void* const* grids, int mode, void* stream) {
  const HaloDev& d = S->dev;
  if (d.B == 0) return LBM_OK;
  if (d.B > 0x7fffffff) return set_error(LBM_ERR_UNSUPPORTED, "exchange table needs too many CTAs");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (prec == LBM_F64 || prec == LBM_F64_DF)
    e = launch_mode<double>(d, grids, mode, st);
  else if (prec == LBM_F32)
    e = launch_mode<float>(d, grids, mode, st);
  else
    e = launch_mode<__half>(d, grids, mode, st);
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("halo exchange: ") + cudaGetErrorString(e));
  return LBM_OK;
}

}  // namespace lbm
