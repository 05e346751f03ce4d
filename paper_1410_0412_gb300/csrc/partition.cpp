// P-way partitioning of a lattice into local lattices plus a ghost-PDF map
// (Sect. 6, Sect. 6.1).
//
// The paper distributes the adjacency list among processes in P contiguous
// chunks of the node vector, chunk p = nodes [N p / P, N (p+1) / P), and each
// step every process receives the PDFs its nodes pull from nodes of other
// chunks.  Here each chunk becomes an ordinary lbm_lattice whose node index
// space is [0, N_p) for its own nodes, followed by ghost slots: a pull of
// direction i from a node of another chunk points at a ghost slot N_p + k,
// where k counts, in local node order, the chunk's earlier foreign pulls in
// direction i.  Slot k of direction array i receives the owner's PDF before
// the step reads it, so the unchanged step kernels run on every chunk.
//
// Numbering ghost slots in node order keeps RIA runs intact across a chunk
// face: consecutive nodes that pull from the other side get consecutive
// slots, i.e. an index advancing by one (Sect. 4.1).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <functional>
#include <new>
#include <string>
#include <thread>

#include <cuda_runtime.h>

#include "internal.h"

namespace lbm {

namespace {

void parallel_parts(int P, const std::function<void(int)>& body) {
  const int T = std::max(1, std::min(P, host_threads()));
  std::vector<std::thread> th;
  std::atomic<int> next{0};
  for (int t = 0; t < T; ++t)
    th.emplace_back([&] {
      for (int p = next++; p < P; p = next++) body(p);
    });
  for (auto& x : th) x.join();
}

}  // namespace

int build_halo_host(lbm_partitioning* S);

int build_partitioning(const lbm_lattice* G, int P, lbm_partitioning* out) {
  const int64_t N = G->N, Ng = G->Npad;
  out->P = P;
  out->N = N;
  out->first.resize(P + 1);
  for (int p = 0; p <= P; ++p) out->first[p] = N * p / P;
  out->part.assign(P, nullptr);
  out->ghost.assign(P, {});
  out->ghost_slots.assign(P, 0);
  std::vector<int> status(P, LBM_OK);
  std::vector<std::string> msg(P);
  const std::vector<int64_t>& first = out->first;
  auto owner = [&](int64_t m) {
    return int(std::upper_bound(first.begin(), first.end(), m) - first.begin()) - 1;
  };
  parallel_parts(P, [&](int p) {
    try {
      const int64_t a = first[p], b = first[p + 1], Np = b - a;
      // ghost slots per direction, in local node order
      int64_t cnt[18] = {0};
      for (int i = 0; i < 18; ++i)
        for (int64_t n = a; n < b; ++n) {
          const int32_t m = G->adj[i * Ng + n];
          cnt[i] += m >= 0 && (m < a || m >= b);
        }
      const int64_t gmax = *std::max_element(cnt, cnt + 18);
      if (Np + gmax > (int64_t(1) << kSlotBits)) {
        status[p] = LBM_ERR_UNSUPPORTED;
        msg[p] = "partition " + std::to_string(p) + " has more than 2^27 nodes plus ghost slots";
        return;
      }
      lbm_lattice* L = new lbm_lattice();
      out->part[p] = L;
      L->X = G->X;
      L->Y = G->Y;
      L->Z = G->Z;
      L->bc = G->bc;
      L->enumeration = G->enumeration;
      L->block_B = G->block_B;
      L->N = Np;
      L->partition_local = 1;
      L->Npad = round_up(std::max<int64_t>(Np + gmax, 1), kPad);
      if (int64_t(G->node_xyz.size()) == 3 * N)
        L->node_xyz.assign(G->node_xyz.begin() + 3 * a, G->node_xyz.begin() + 3 * b);
      L->adj.assign(18 * L->Npad, LBM_MARK_WALL);
      std::vector<GhostEntry>& E = out->ghost[p];
      E.reserve(std::accumulate(cnt, cnt + 18, int64_t(0)));
      for (int i = 0; i < 18; ++i) {
        int64_t k = 0;
        for (int64_t n = a; n < b; ++n) {
          const int32_t m = G->adj[i * Ng + n];
          int32_t loc;
          if (m < 0) {
            loc = m;
          } else if (m >= a && m < b) {
            loc = int32_t(m - a);
          } else {
            const int q = owner(m);
            loc = int32_t(Np + k);
            E.push_back(GhostEntry{q, i, int32_t(Np + k), int32_t(m - first[q])});
            ++k;
          }
          L->adj[i * L->Npad + (n - a)] = loc;
        }
      }
      // exchange order: by owner, then direction, then slot
      std::stable_sort(E.begin(), E.end(), [](const GhostEntry& u, const GhostEntry& v) { return u.q < v.q; });
      out->ghost_slots[p] = gmax;
      status[p] = derive_ria(L);
      if (status[p]) msg[p] = "out of host memory for the RIA table of partition " + std::to_string(p);
    } catch (const std::bad_alloc&) {
      status[p] = LBM_ERR_ALLOC;
      msg[p] = "out of host memory while building partition " + std::to_string(p);
    } catch (...) {
      status[p] = LBM_ERR_ALLOC;
      msg[p] = "host tables of partition " + std::to_string(p) + " exceed the vector size limit";
    }
  });
  for (int p = 0; p < P; ++p)
    if (status[p]) return set_error(status[p], msg[p]);
  return build_halo_host(out);
}

// Flatten the ghost lists into the device exchange table: entries grouped by
// (receiver p, owner q), each group cut into CTAs of kHaloBlock entries, so a
// CTA copies between one pair of grids.
int build_halo_host(lbm_partitioning* S) {
  int64_t E = 0;
  for (const auto& g : S->ghost) E += int64_t(g.size());
  if (E > INT32_MAX) return set_error(LBM_ERR_UNSUPPORTED, "more than 2^31 ghost PDFs");
  S->h_dirslot.clear();
  S->h_node.clear();
  S->h_grp_p.clear();
  S->h_grp_q.clear();
  S->h_grp_end.clear();
  S->h_blk_group.clear();
  S->h_blk_first.clear();
  S->h_dirslot.reserve(E);
  S->h_node.reserve(E);
  for (int p = 0; p < S->P; ++p) {
    const auto& g = S->ghost[p];
    for (size_t k = 0; k < g.size(); ++k) {
      if (k == 0 || g[k].q != g[k - 1].q) {
        if (!S->h_grp_p.empty()) S->h_grp_end.push_back(int32_t(S->h_dirslot.size()));
        S->h_grp_p.push_back(p);
        S->h_grp_q.push_back(g[k].q);
      }
      S->h_dirslot.push_back((uint32_t(g[k].dir) << kSlotBits) | uint32_t(g[k].slot));
      S->h_node.push_back(g[k].node);
    }
  }
  if (!S->h_grp_p.empty()) S->h_grp_end.push_back(int32_t(S->h_dirslot.size()));
  int64_t begin = 0;
  for (size_t grp = 0; grp < S->h_grp_p.size(); ++grp) {
    const int64_t end = S->h_grp_end[grp];
    for (int64_t f = begin; f < end; f += kHaloBlock) {
      S->h_blk_group.push_back(int32_t(grp));
      S->h_blk_first.push_back(int32_t(f));
    }
    begin = end;
  }
  S->h_npad.resize(S->P);
  for (int p = 0; p < S->P; ++p) S->h_npad[p] = S->part[p]->Npad;
  return LBM_OK;
}

int validate_partitioning(const lbm_partitioning* S, const lbm_lattice* G) {
  constexpr int64_t kUnset = -1000;  // below every marker
  if (S->N != G->N) return set_error(LBM_ERR_TABLE, "partitioning and lattice differ in N");
  const int64_t Ng = G->Npad;
  for (int p = 0; p < S->P; ++p) {
    const lbm_lattice* L = S->part[p];
    const int64_t a = S->first[p], Np = L->N;
    if (Np != S->first[p + 1] - a) return set_error(LBM_ERR_TABLE, "partition size mismatch");
    // slot -> global source, per direction
    std::vector<int64_t> slot_src(size_t(18) * size_t(L->Npad - Np), kUnset);
    for (const GhostEntry& e : S->ghost[p]) {
      if (e.q < 0 || e.q >= S->P || e.q == p || e.dir < 0 || e.dir >= 18 || e.slot < Np || e.slot >= L->Npad)
        return set_error(LBM_ERR_TABLE, "ghost entry out of range in partition " + std::to_string(p));
      const int64_t src = S->first[e.q] + e.node;
      if (e.node < 0 || src >= S->first[e.q + 1])
        return set_error(LBM_ERR_TABLE, "ghost source outside its owner in partition " + std::to_string(p));
      int64_t& cell = slot_src[size_t(e.dir) * size_t(L->Npad - Np) + size_t(e.slot - Np)];
      if (cell != kUnset) return set_error(LBM_ERR_TABLE, "ghost slot used twice in partition " + std::to_string(p));
      cell = src;
    }
    for (int i = 0; i < 18; ++i)
      for (int64_t n = 0; n < Np; ++n) {
        const int32_t loc = L->adj[i * L->Npad + n];
        int64_t want = G->adj[i * Ng + a + n], got;
        if (loc < 0)
          got = loc;
        else if (loc < Np)
          got = a + loc;
        else if (loc < L->Npad)
          got = slot_src[size_t(i) * size_t(L->Npad - Np) + size_t(loc - Np)];
        else
          got = kUnset;
        if (got != want)
          return set_error(LBM_ERR_TABLE, "partition " + std::to_string(p) + " does not decode to the lattice at node " +
                                              std::to_string(a + n));
      }
    if (int rc = validate_runs(L)) return rc;
  }
  return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

lbm_partitioning::~lbm_partitioning() {
  for (lbm_lattice* L : part) delete L;
  for (void* st : side_streams) cudaStreamDestroy(static_cast<cudaStream_t>(st));
  for (void* ev : side_done) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
  if (fork_event) cudaEventDestroy(static_cast<cudaEvent_t>(fork_event));
}

namespace {

// Up to this many chunks step at the same time.
constexpr int kSideStreams = 16;

int ensure_side_streams(lbm_partitioning* S) {
  std::lock_guard<std::mutex> lock(S->side_mu);
  if (S->fork_event) return LBM_OK;
  const int K = std::min(S->P, kSideStreams);
  cudaError_t e = cudaSuccess;
  cudaEvent_t fork;
  e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    cudaStream_t st;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    S->side_streams.push_back(st);
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    S->side_done.push_back(ev);
  }
  if (e != cudaSuccess) {
    for (void* st : S->side_streams) cudaStreamDestroy(static_cast<cudaStream_t>(st));
    for (void* ev : S->side_done) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
    S->side_streams.clear();
    S->side_done.clear();
    return set_error(LBM_ERR_CUDA, std::string("side streams: ") + cudaGetErrorString(e));
  }
  S->fork_event = fork;
  return LBM_OK;
}

// Run step(p, stream) for every chunk, chunk p on side stream p mod K, all
// after the work already queued on `stream` and before anything queued on it
// afterwards.
template <typename F>
int for_chunks(const lbm_partitioning* S, void* stream, F step) {
  cudaStream_t main = static_cast<cudaStream_t>(stream);
  cudaEvent_t fork = static_cast<cudaEvent_t>(S->fork_event);
  const int K = int(S->side_streams.size());
  cudaError_t e = cudaEventRecord(fork, main);
  for (int k = 0; k < K && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(static_cast<cudaStream_t>(S->side_streams[k]), fork, 0);
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("fork: ") + cudaGetErrorString(e));
  for (int p = 0; p < S->P; ++p)
    if (int rc = step(p, S->side_streams[p % K])) return rc;
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    e = cudaEventRecord(static_cast<cudaEvent_t>(S->side_done[k]), static_cast<cudaStream_t>(S->side_streams[k]));
    if (e == cudaSuccess) e = cudaStreamWaitEvent(main, static_cast<cudaEvent_t>(S->side_done[k]), 0);
  }
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("join: ") + cudaGetErrorString(e));
  return LBM_OK;
}

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

struct HaloLayout {
  size_t dirslot = 0, node = 0, grp_p = 0, grp_q = 0, grp_end = 0, blk_group = 0, blk_first = 0, npad = 0, total = 0;
};

HaloLayout halo_layout(const lbm_partitioning* S) {
  HaloLayout t;
  const size_t E = S->h_dirslot.size(), G = S->h_grp_p.size(), B = S->h_blk_group.size(), P = size_t(S->P);
  size_t off = 0;
  auto take = [&](size_t& at, size_t bytes) {
    at = off;
    off = al256(off + std::max<size_t>(bytes, 4));
  };
  take(t.dirslot, E * 4);
  take(t.node, E * 4);
  take(t.grp_p, G * 4);
  take(t.grp_q, G * 4);
  take(t.grp_end, G * 4);
  take(t.blk_group, B * 4);
  take(t.blk_first, B * 4);
  take(t.npad, P * 8);
  t.total = off;
  return t;
}

int check_part(const lbm_partitioning* S, int p) {
  if (!S) return set_error(LBM_ERR_ARG, "partitioning handle is NULL");
  if (p < 0 || p >= S->P) return set_error(LBM_ERR_ARG, "partition index out of range");
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_partition_build(const lbm_lattice* lat, int P, lbm_partitioning** out) {
  if (!out) return set_error(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!lat) return set_error(LBM_ERR_ARG, "lattice handle is NULL");
  if (P < 1 || P > std::max<int64_t>(lat->N, 1)) return set_error(LBM_ERR_ARG, "P must be in [1, max(N, 1)]");
  lbm_partitioning* S = new (std::nothrow) lbm_partitioning();
  if (!S) return set_error(LBM_ERR_ALLOC, "out of host memory");
  int rc;
  try {
    rc = build_partitioning(lat, P, S);
  } catch (const std::bad_alloc&) {
    rc = set_error(LBM_ERR_ALLOC, "out of host memory while partitioning");
  }
  if (rc) {
    delete S;
    return rc;
  }
  *out = S;
  return LBM_OK;
}

void lbm_free_partitioning(lbm_partitioning* part) { delete part; }

int lbm_partition_info(const lbm_partitioning* part, int p, int64_t* first_node, int64_t* N_p, int64_t* ghost_pdfs,
                       int64_t* ghost_slots) {
  if (int rc = check_part(part, p)) return rc;
  if (first_node) *first_node = part->first[p];
  if (N_p) *N_p = part->first[p + 1] - part->first[p];
  if (ghost_pdfs) *ghost_pdfs = int64_t(part->ghost[p].size());
  if (ghost_slots) *ghost_slots = part->ghost_slots[p];
  return LBM_OK;
}

int lbm_partition_local(lbm_partitioning* part, int p, lbm_lattice** local) {
  if (int rc = check_part(part, p)) return rc;
  if (!local) return set_error(LBM_ERR_ARG, "local is NULL");
  *local = part->part[p];
  return LBM_OK;
}

int lbm_partition_export_ghosts(const lbm_partitioning* part, int p, int32_t* src_part, int32_t* dir, int32_t* slot,
                                int32_t* src_node) {
  if (int rc = check_part(part, p)) return rc;
  const auto& g = part->ghost[p];
  for (size_t k = 0; k < g.size(); ++k) {
    if (src_part) src_part[k] = g[k].q;
    if (dir) dir[k] = g[k].dir + 1;
    if (slot) slot[k] = g[k].slot;
    if (src_node) src_node[k] = g[k].node;
  }
  return LBM_OK;
}

int lbm_partition_validate(const lbm_partitioning* part, const lbm_lattice* lat) {
  if (!part || !lat) return set_error(LBM_ERR_ARG, "partitioning or lattice handle is NULL");
  try {
    return validate_partitioning(part, lat);
  } catch (const std::bad_alloc&) {
    return set_error(LBM_ERR_ALLOC, "out of host memory while validating the partitioning");
  }
}

int lbm_halo_table_bytes(const lbm_partitioning* part, size_t* bytes) {
  if (!part) return set_error(LBM_ERR_ARG, "partitioning handle is NULL");
  if (!bytes) return set_error(LBM_ERR_ARG, "bytes is NULL");
  *bytes = halo_layout(part).total;
  return LBM_OK;
}

int lbm_halo_upload(lbm_partitioning* part, void* dev, size_t bytes, void* stream) {
  if (!part) return set_error(LBM_ERR_ARG, "partitioning handle is NULL");
  if (!dev) return set_error(LBM_ERR_ARG, "device table buffer is NULL");
  if (reinterpret_cast<uintptr_t>(dev) % 256) return set_error(LBM_ERR_ARG, "device table buffer not 256-byte aligned");
  const HaloLayout t = halo_layout(part);
  if (bytes < t.total) return set_error(LBM_ERR_ARG, "device table buffer too small");
  part->uploaded = 0;
  part->dev = HaloDev{};
  char* base = static_cast<char*>(dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  auto put = [&](size_t off, const void* src, size_t n) {
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, st);
  };
  put(t.dirslot, part->h_dirslot.data(), part->h_dirslot.size() * 4);
  put(t.node, part->h_node.data(), part->h_node.size() * 4);
  put(t.grp_p, part->h_grp_p.data(), part->h_grp_p.size() * 4);
  put(t.grp_q, part->h_grp_q.data(), part->h_grp_q.size() * 4);
  put(t.grp_end, part->h_grp_end.data(), part->h_grp_end.size() * 4);
  put(t.blk_group, part->h_blk_group.data(), part->h_blk_group.size() * 4);
  put(t.blk_first, part->h_blk_first.data(), part->h_blk_first.size() * 4);
  put(t.npad, part->h_npad.data(), part->h_npad.size() * 8);
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("halo upload: ") + cudaGetErrorString(e));
  HaloDev& d = part->dev;
  d.e_dirslot = reinterpret_cast<const uint32_t*>(base + t.dirslot);
  d.e_node = reinterpret_cast<const int32_t*>(base + t.node);
  d.grp_p = reinterpret_cast<const int32_t*>(base + t.grp_p);
  d.grp_q = reinterpret_cast<const int32_t*>(base + t.grp_q);
  d.grp_end = reinterpret_cast<const int32_t*>(base + t.grp_end);
  d.blk_group = reinterpret_cast<const int32_t*>(base + t.blk_group);
  d.blk_first = reinterpret_cast<const int32_t*>(base + t.blk_first);
  d.npad = reinterpret_cast<const int64_t*>(base + t.npad);
  d.E = int64_t(part->h_dirslot.size());
  d.G = int64_t(part->h_grp_p.size());
  d.B = int64_t(part->h_blk_group.size());
  part->uploaded = 1;
  return LBM_OK;
}

int lbm_halo_exchange(const lbm_partitioning* part, int prec, void* const* grids, int mode, void* stream) {
  if (!part) return set_error(LBM_ERR_ARG, "partitioning handle is NULL");
  if (!part->uploaded) return set_error(LBM_ERR_ARG, "exchange table not uploaded to the device");
  if (prec < LBM_F64 || prec > LBM_F64_DF) return set_error(LBM_ERR_ARG, "unknown precision");
  if (mode < LBM_HALO_OSNT || mode > LBM_HALO_AA_SCATTER) return set_error(LBM_ERR_ARG, "unknown exchange mode");
  if (!grids) return set_error(LBM_ERR_ARG, "grids is NULL");
  if (reinterpret_cast<uintptr_t>(grids) % 8) return set_error(LBM_ERR_ARG, "grids not 8-byte aligned");
  return launch_halo(part, prec, grids, mode, stream);
}

int lbm_partition_run_aa(const lbm_partitioning* part, int prec, const lbm_params* params, void* const* grids_host,
                         void* const* grids_dev, const float* s, int start_parity, int steps, int ria, void* stream) {
  if (!part) return set_error(LBM_ERR_ARG, "partitioning handle is NULL");
  if (!grids_host || !grids_dev) return set_error(LBM_ERR_ARG, "grids_host or grids_dev is NULL");
  if (start_parity != 0 && start_parity != 1) return set_error(LBM_ERR_ARG, "parity must be 0 or 1");
  if (steps < 0) return set_error(LBM_ERR_ARG, "steps must be >= 0");
  if (!part->uploaded) return set_error(LBM_ERR_ARG, "exchange table not uploaded to the device");
  for (int p = 0; p < part->P; ++p)
    if (!grids_host[p]) return set_error(LBM_ERR_ARG, "grids_host has a NULL grid");
  if (int rc = ensure_side_streams(const_cast<lbm_partitioning*>(part))) return rc;
  for (int k = 0; k < steps; ++k) {
    const int parity = (start_parity + k) & 1;
    if (parity == 1)
      if (int rc = lbm_halo_exchange(part, prec, grids_dev, LBM_HALO_AA_GATHER, stream)) return rc;
    if (int rc = for_chunks(part, stream, [&](int p, void* st) {
          return lbm_step_aa(part->part[p], prec, params, grids_host[p], parity, s ? s + part->first[p] : nullptr,
                             ria, st);
        }))
      return rc;
    if (parity == 1)
      if (int rc = lbm_halo_exchange(part, prec, grids_dev, LBM_HALO_AA_SCATTER, stream)) return rc;
  }
  return LBM_OK;
}

int lbm_partition_run_osnt(const lbm_partitioning* part, int prec, const lbm_params* params, void* const* grids_host,
                           void* const* grids_dev, const float* s, int steps, int ria, void* stream) {
  if (!part) return set_error(LBM_ERR_ARG, "partitioning handle is NULL");
  if (!grids_host || !grids_dev) return set_error(LBM_ERR_ARG, "grids_host or grids_dev is NULL");
  if (steps < 0) return set_error(LBM_ERR_ARG, "steps must be >= 0");
  if (!part->uploaded) return set_error(LBM_ERR_ARG, "exchange table not uploaded to the device");
  const int P = part->P;
  for (int p = 0; p < 2 * P; ++p)
    if (!grids_host[p]) return set_error(LBM_ERR_ARG, "grids_host has a NULL grid");
  if (int rc = ensure_side_streams(const_cast<lbm_partitioning*>(part))) return rc;
  for (int k = 0; k < steps; ++k) {
    const int src = (k & 1) * P, dst = P - src;
    if (int rc = lbm_halo_exchange(part, prec, grids_dev + src, LBM_HALO_OSNT, stream)) return rc;
    if (int rc = for_chunks(part, stream, [&](int p, void* st) {
          return lbm_step_osnt(part->part[p], prec, params, grids_host[src + p], grids_host[dst + p],
                               s ? s + part->first[p] : nullptr, ria, st);
        }))
      return rc;
  }
  return LBM_OK;
}

}  // extern "C"
