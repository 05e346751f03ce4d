// Internal declarations shared by the host lattice builder, the C ABI layer
// and the CUDA kernels of liblbm.  Not part of the public interface.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

// D3Q19 velocity set in the library's direction order (see lbm.h).
constexpr int kQ = 19;
constexpr int kCX[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int kCY[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int kCZ[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
constexpr int kInv[kQ] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};

// Node-count padding of every SoA direction array; 128 nodes keep each
// direction of an FP16 grid 256-byte aligned.
constexpr int64_t kPad = 128;
// RIA lookup granularity: one 32-bit run-head mask and one run index per 32
// consecutive nodes (a warp's worth).
constexpr int kWarpNodes = 32;

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Host threads of the table builders: LBM_HOST_THREADS (1..256) when set,
// otherwise every hardware thread, at most 64.  Read on every call, so a
// process may change it between builds; the tables do not depend on it.
int host_threads();

// Allocator whose value-less construct() leaves the element uninitialized, so
// that resize() of a large table costs no serial fill: the builders then
// write every element, in parallel.
template <class T> struct NoInitAlloc : std::allocator<T> {
  template <class U> struct rebind { using other = NoInitAlloc<U>; };
  NoInitAlloc() = default;
  template <class U> NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U> void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A> void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
using TableVec = std::vector<int32_t, NoInitAlloc<int32_t>>;

// Run slot tables (derive_run_slots): run-major, kSlotStride int32 per run
// (18 slots and 2 words of padding, 80 bytes), so that a thread fetches its
// run's 18 slots with five aligned vector loads instead of 18 scalar ones.
// With LBM_SLOT_AOS=0 they are direction-major, [18][Rpad].
#ifndef LBM_SLOT_AOS
#define LBM_SLOT_AOS 1
#endif
constexpr int kSlotStride = 20;
inline size_t run_slot_words(int64_t Rpad) { return size_t(LBM_SLOT_AOS ? kSlotStride : 18) * size_t(Rpad); }

// Device addresses of the uploaded tables (all inside one caller buffer).
struct DevTables {
  const int32_t* adj = nullptr;         // [18][Npad]
  const int32_t* run_adj = nullptr;     // [18][Rpad]   adjacency entries of each run's first node
  const uint32_t* head_bits = nullptr;  // [nwarps]     bit j of word w: node 32w+j starts a run
  const int32_t* warp_run0 = nullptr;   // [nwarps]     run holding node 32w
  const int32_t* warp_head0 = nullptr;  // [nwarps]     first node of that run
  // [Rpad][kSlotStride] the AA odd step's and the OS-NT step's slots of each
  // run's first node (see derive_run_slots), or NULL where the lattice does
  // not qualify
  const int32_t* run_slot = nullptr;
  const int32_t* run_slot_osnt = nullptr;
  int64_t Npad = 0, Rpad = 0, R = 0, nwarps = 0;
  uint32_t npad = 0, rpad = 0;          // the same strides as 32-bit values (N < 2^31)
  int pressure = 0;                     // the lattice has inlet/outlet markers
  const int32_t* et_nb = nullptr;       // [6][Npad]   Esoteric Twist neighbour locations
  const uint32_t* et_mask = nullptr;    // [Npad]      Esoteric Twist link kinds
  uint32_t spad = 0;                    // Esoteric Twist grid stride (nodes + phantoms, padded)
  // Esoteric Twist run table (the RIA coding of et_nb / et_mask), same warp-level index
  const int32_t* et_run_nb = nullptr;   // [6][et_rpad] locations of each run's first node
  const uint32_t* et_run_mask = nullptr;// [et_rpad]    its link mask
  const uint32_t* et_head_bits = nullptr;
  const int32_t* et_warp_run0 = nullptr;
  const int32_t* et_warp_head0 = nullptr;
  uint32_t et_rpad = 0;
};

// Ghost slots of a partition: local node index space [0, N_p) followed by the
// slots; slot numbers and direction share one 32-bit word on the device.
constexpr int kSlotBits = 27;
constexpr int kHaloBlock = 256;

// One ghost PDF of a partition: the pull of direction dir + 1 that lands in
// local slot `slot` comes from node `node` (local index) of partition q.
struct GhostEntry {
  int32_t q, dir, slot, node;
};

// Device addresses of the uploaded exchange table (one caller buffer).
struct HaloDev {
  const uint32_t* e_dirslot = nullptr;  // [E]  dir << kSlotBits | slot
  const int32_t* e_node = nullptr;      // [E]  source node, local to the owner
  const int32_t* grp_p = nullptr;       // [G]  receiving partition of each (receiver, owner) group
  const int32_t* grp_q = nullptr;       // [G]  owning partition
  const int32_t* grp_end = nullptr;     // [G]  one past the group's last entry
  const int32_t* blk_group = nullptr;   // [B]  group of each CTA
  const int32_t* blk_first = nullptr;   // [B]  first entry of each CTA
  const int64_t* npad = nullptr;        // [P]  grid stride of each partition
  int64_t E = 0, G = 0, B = 0;
};

}  // namespace lbm

struct lbm_lattice {
  int X = 0, Y = 0, Z = 0;
  lbm_bc bc{};
  int enumeration = 0, block_B = 1;
  int64_t N = 0, Npad = 0, R = 0, Rpad = 0, nwarps = 0;
  std::vector<int32_t> node_xyz;   // [N][3]
  lbm::TableVec adj;               // [18][Npad], padding = -1
  std::vector<int32_t> run_start;  // [R+1]
  lbm::TableVec run_adj;           // [18][Rpad], padding = -1
  std::vector<uint32_t> head_bits; // [nwarps]  run heads, one bit per node
  std::vector<int32_t> warp_run0;  // [nwarps]  run holding node 32w
  std::vector<int32_t> warp_head0; // [nwarps]  first node of that run
  int64_t hist[33] = {0};
  // The AA odd step's slots per run (derive_run_slots): -1 not derived yet,
  // 0 the lattice does not qualify, 1 run_slot holds them
  int run_slot_state = -1;
  lbm::TableVec run_slot;          // [Rpad][kSlotStride] AA odd step
  lbm::TableVec run_slot_osnt;     // [Rpad][kSlotStride] OS-NT step
  // Esoteric Twist tables, derived on first use (derive_et)
  int et_ready = 0;
  int64_t et_S = 0, et_Spad = 0;   // storage locations (nodes + phantoms) and the padded grid stride
  std::vector<int32_t> et_nb;      // [6][Npad] storage index of n + (+x, +y, +z, +x+y, +x+z, +y+z)
  std::vector<uint32_t> et_mask;   // [Npad] bit i-1: pull i meets a marker; bits 18..27: pressure faces
  std::vector<int32_t> et_phantom; // [S-N][3] coordinates of the phantom locations
  int64_t et_R = 0, et_Rpad = 0;   // runs of the ET tables (a run continues while all six locations advance by one
  std::vector<int32_t> et_run_start;   // [et_R+1]             and the mask is unchanged)
  std::vector<int32_t> et_run_nb;      // [6][et_Rpad]
  std::vector<uint32_t> et_run_mask;   // [et_Rpad]
  std::vector<uint32_t> et_head_bits;  // [nwarps]
  std::vector<int32_t> et_warp_run0;   // [nwarps]
  std::vector<int32_t> et_warp_head0;  // [nwarps]
  int uploaded = 0;                // LBM_TABLES_* bits present on the device
  int partition_local = 0;         // a partition's local lattice: entries >= N are ghost slots
  lbm::DevTables dev;
};

struct lbm_partitioning {
  int P = 0;
  int64_t N = 0;                                 // nodes of the partitioned lattice
  std::vector<int64_t> first;                    // [P+1] chunk bounds N p / P
  std::vector<lbm_lattice*> part;                // [P] local lattices (owned)
  std::vector<std::vector<lbm::GhostEntry>> ghost;  // [P] ghost entries, by owner, direction, slot
  std::vector<int64_t> ghost_slots;              // [P] slots behind the local nodes (max over directions)
  // host copy of the exchange table (the source of lbm_halo_upload)
  std::vector<uint32_t> h_dirslot;
  std::vector<int32_t> h_node, h_grp_p, h_grp_q, h_grp_end, h_blk_group, h_blk_first;
  std::vector<int64_t> h_npad;
  int uploaded = 0;
  lbm::HaloDev dev;
  // Library-owned side streams on which the chunks' steps run concurrently
  // (fork / join through events on the caller's stream); created on the
  // first partitioned run, on the device current at that time.
  std::vector<void*> side_streams, side_done;
  void* fork_event = nullptr;
  std::mutex side_mu;  // guards their creation
  lbm_partitioning() = default;
  lbm_partitioning(const lbm_partitioning&) = delete;
  lbm_partitioning& operator=(const lbm_partitioning&) = delete;
  ~lbm_partitioning();
};

namespace lbm {

// Error reporting (thread-local message, see lbm_last_error).
int set_error(int code, const std::string& msg);

// Host table construction (lattice.cpp).
int build_tables(lbm_lattice* L, const uint8_t* solid);
int build_tables_from_order(lbm_lattice* L, const uint8_t* solid, const int32_t* node_xyz, int64_t N);
int renumber_partitions(const lbm_lattice* L, int P, int32_t* out);
int partition_ghosts(const lbm_lattice* L, int P, int64_t* ghosts);
int build_partitioning(const lbm_lattice* G, int P, lbm_partitioning* out);   // partition.cpp
int validate_partitioning(const lbm_partitioning* S, const lbm_lattice* G);
int launch_halo(const lbm_partitioning* S, int prec, void* const* grids, int mode, void* stream);  // halo.cu
int derive_ria(lbm_lattice* L);
int derive_et(lbm_lattice* L);   // Esoteric Twist tables (idempotent)
int derive_run_slots(lbm_lattice* L);  // the AA odd step's run slots (idempotent)
int validate(const lbm_lattice* L);
int validate_runs(const lbm_lattice* L);  // the RIA tables alone (any index range)

// Kernel-side parameter block, computed on the host from lbm_params.
struct KParams {
  double lp, lm;        // TRT rates lambda+, lambda-
  double g[3];          // body force per unit mass
  double rho_s;         // density of the storage shift (0 when unshifted)
  double rho_in, rho_out;
  float scale, inv_scale;  // FP16 storage scale and its inverse
};

int make_kparams(const lbm_params* p, int prec, KParams* kp);

// Argument checks shared by the entry points (api.cpp): a non-NULL handle; a
// known layout; the device tables the layout's gathers need (none for
// LBM_LAYOUT_AA_EVEN, the Esoteric Twist tables for the ET layouts, any
// addressing otherwise).  Each returns LBM_OK or sets the error message.
int check_lat(const lbm_lattice* L);
int any_tables(const lbm_lattice* L, int* ria);
int check_layout(int layout);
int layout_tables(const lbm_lattice* L, int layout);

// Kernel launchers, one explicit instantiation per storage precision in
// kernels_<prec>.cu.  All return a LBM_* status.
template <int PREC>
int launch_osnt_t(const lbm_lattice* L, const KParams& kp, const void* src, void* dst, const float* s, int ria,
                  void* stream);
template <int PREC>
int launch_aa_t(const lbm_lattice* L, const KParams& kp, void* pdf, int parity, const float* s, int ria,
                void* stream);
template <int PREC>
int launch_et_t(const lbm_lattice* L, const KParams& kp, void* pdf, int parity, const float* s, int ria,
                void* stream);
template <int PREC>
int launch_init_eq_t(const lbm_lattice* L, const KParams& kp, void* pdf, int layout, double rho0, const double* u0,
                     void* stream);
template <int PREC>
int launch_load_canonical_t(const lbm_lattice* L, const KParams& kp, const double* F, void* pdf, int layout,
                            void* stream);
template <int PREC>
int launch_canonical_t(const lbm_lattice* L, const KParams& kp, const void* pdf, int layout, double* F,
                       void* stream);
template <int PREC>
int launch_macroscopic_t(const lbm_lattice* L, const KParams& kp, const void* pdf, int layout, const float* s,
                         double* rho, double* u, double* sums, double* partials, int64_t nparts, void* stream);

template <int PREC>
int launch_adjoint_t(const lbm_lattice* L, const KParams& kp, const void* G, const void* lam_next, void* lam,
                     const float* s, double* grad_s, int ria, void* stream);
template <int PREC>
int launch_objective_t(const lbm_lattice* L, const KParams& kp, const void* pdf, int layout, const float* s,
                       double* J, void* lamT, double* grad_s, double* partials, void* stream);

// Precision dispatch: call F<LBM_F64 | LBM_F32 | LBM_F16S>.  LBM_F64_DF grids
// are IEEE double grids: everything but the step kernels treats them as LBM_F64.
#define LBM_DISPATCH(prec, fn, ...)                                        \
  (((prec) == LBM_F64 || (prec) == LBM_F64_DF) ? fn<LBM_F64>(__VA_ARGS__)  \
   : (prec) == LBM_F32 ? fn<LBM_F32>(__VA_ARGS__)                          \
                       : fn<LBM_F16S>(__VA_ARGS__))
// Step kernels: the double-float arithmetic has its own instantiation.
#define LBM_DISPATCH_STEP(prec, fn, ...)                                   \
  ((prec) == LBM_F64_DF ? fn<LBM_F64_DF>(__VA_ARGS__) : LBM_DISPATCH(prec, fn, __VA_ARGS__))

// Number of per-CTA partial sums of the reductions (one per 128-node CTA).
inline int64_t reduce_parts(const lbm_lattice* L) { return std::max<int64_t>(1, (L->N + 127) / 128); }

}  // namespace lbm
