// Host-side construction of the sparse lattice: fluid-node enumeration,
// adjacency list and RIA run table, plus their validation.
//
// Sect. 1 and Sect. 5.6: fluid nodes are stored in one 1-D vector whose order
// is set by an enumeration function, lexicographic sorting (LS) with a
// blocking factor B or a space-filling (Hilbert) curve.  Sect. 4 "Loop
// Balance" and Fig. 2a: an adjacency list holds, per node, where each of the
// 18 moving PDFs is pulled from.  Sect. 4.1 and Fig. 2b: reduced indirect
// addressing keeps only the runs of nodes whose access pattern is the
// previous node's shifted by one, run-length coded.
//
// Everything here is O(voxels) or O(N) and multithreaded with std::thread;
// none of it is on the timed path.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <thread>

#include "internal.h"

namespace lbm {

int host_threads() {
  if (const char* e = std::getenv("LBM_HOST_THREADS")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 1 && v <= 256) return static_cast<int>(v);
  }
  const unsigned h = std::thread::hardware_concurrency();
  return h == 0 ? 4 : static_cast<int>(std::min(h, 64u));
}

namespace {

int n_threads() { return host_threads(); }

// Run body(begin, end) over [0, n) split into contiguous chunks, one per thread.
// Fewer than min_items items run on the calling thread: per-node loops keep
// the default, loops over coarse items (slabs, chunks, partitions) pass 2.
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body, int64_t min_items = 4096) {
  int T = n_threads();
  if (n < min_items || T == 1) {
    if (n > 0) body(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + T - 1) / T;
  for (int t = 0; t < T; ++t) {
    int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back(body, b, e);
  }
  for (auto& x : th) x.join();
}

// Exclusive prefix sum in place; returns the total.
int64_t exclusive_scan(std::vector<int64_t>& v) {
  int64_t acc = 0;
  for (auto& x : v) {
    int64_t c = x;
    x = acc;
    acc += c;
  }
  return acc;
}

// ---- LS with blocking factor B -------------------------------------------------
// Work unit u = (block z, block y, block x, z offset in the block); units are
// numbered in the enumeration's own order, so counting fluid voxels per unit,
// scanning, and refilling gives the node order without a sort.
int enumerate_lex(lbm_lattice* L, const uint8_t* solid, int B) {
  const int64_t X = L->X, Y = L->Y, Z = L->Z;
  const int64_t Bm = std::max<int64_t>({X, Y, Z});
  const int64_t b = (B <= 1 || B >= Bm) ? Bm : B;  // B = 1 orders like one big block
  const int64_t nbx = (X + b - 1) / b, nby = (Y + b - 1) / b, nbz = (Z + b - 1) / b;
  const int64_t units = nbz * nby * nbx * b;
  auto unit_box = [&](int64_t u, int64_t& z, int64_t& y0, int64_t& y1, int64_t& x0, int64_t& x1) {
    int64_t dz = u % b;
    int64_t blk = u / b;
    int64_t bx = blk % nbx;
    int64_t by = (blk / nbx) % nby;
    int64_t bz = blk / (nbx * nby);
    z = bz * b + dz;
    y0 = by * b;
    y1 = std::min(Y, y0 + b);
    x0 = bx * b;
    x1 = std::min(X, x0 + b);
    return z < Z;
  };
  std::vector<int64_t> cnt(units, 0);
  parallel_for(units, [&](int64_t ub, int64_t ue) {
    for (int64_t u = ub; u < ue; ++u) {
      int64_t z, y0, y1, x0, x1;
      if (!unit_box(u, z, y0, y1, x0, x1)) continue;
      int64_t c = 0;
      for (int64_t y = y0; y < y1; ++y) {
        const uint8_t* row = solid + (z * Y + y) * X;
        for (int64_t x = x0; x < x1; ++x) c += row[x] == 0;
      }
      cnt[u] = c;
    }
  }, 2);
  int64_t N = exclusive_scan(cnt);
  if (N > INT32_MAX) return set_error(LBM_ERR_ARG, "more than 2^31-1 fluid nodes");
  L->N = N;
  L->node_xyz.assign(3 * N, 0);
  parallel_for(units, [&](int64_t ub, int64_t ue) {
    for (int64_t u = ub; u < ue; ++u) {
      int64_t z, y0, y1, x0, x1;
      if (!unit_box(u, z, y0, y1, x0, x1)) continue;
      int64_t n = cnt[u];
      for (int64_t y = y0; y < y1; ++y) {
        const uint8_t* row = solid + (z * Y + y) * X;
        for (int64_t x = x0; x < x1; ++x)
          if (row[x] == 0) {
            L->node_xyz[3 * n + 0] = static_cast<int32_t>(x);
            L->node_xyz[3 * n + 1] = static_cast<int32_t>(y);
            L->node_xyz[3 * n + 2] = static_cast<int32_t>(z);
            ++n;
          }
      }
    }
  }, 2);
  return LBM_OK;
}

// ---- Hilbert curve ----------------------------------------------------------------
// Bit i of v moved to bit 3i (v < 2^21).
inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// Index of (x, y, z) on the Hilbert curve of the 2^bits cube, after J. Skilling,
// "Programming the Hilbert curve" (AIP Conf. Proc. 707, 2004): undo the
// per-level rotations/reflections from the top bit down, Gray-code across the
// three axes, then read the transposed bits out level by level (x first).
// Branch-free: each level's "bit set" choice is a mask, so the per-voxel
// loop does not mispredict on the coordinates' bits.
uint64_t hilbert_index(uint32_t x, uint32_t y, uint32_t z, int bits) {
  if (bits == 0) return 0;
  uint32_t a0 = x, a1 = y, a2 = z;
  for (int l = bits - 1; l >= 1; --l) {
    const uint32_t low = (1u << l) - 1u;
    // axis 0: bit set -> invert its low bits (the exchange with itself is a no-op)
    a0 ^= low & (0u - ((a0 >> l) & 1u));
    // axes 1, 2: bit set -> invert axis 0's low bits, else exchange them with axis 0's
    {
      const uint32_t m = 0u - ((a1 >> l) & 1u);
      const uint32_t t = (a0 ^ a1) & low & ~m;
      a0 ^= (low & m) | t;
      a1 ^= t;
    }
    {
      const uint32_t m = 0u - ((a2 >> l) & 1u);
      const uint32_t t = (a0 ^ a2) & low & ~m;
      a0 ^= (low & m) | t;
      a2 ^= t;
    }
  }
  a1 ^= a0;  // Gray code across the axes
  a2 ^= a1;
  uint32_t fix = 0;
  for (int l = bits - 1; l >= 1; --l) fix ^= ((1u << l) - 1u) & (0u - ((a2 >> l) & 1u));
  a0 ^= fix;
  a1 ^= fix;
  a2 ^= fix;
  // read the transposed bits out level by level, axis 0 first
  const uint32_t mask = (1u << bits) - 1u;
  return (spread3(a0 & mask) << 2) | (spread3(a1 & mask) << 1) | spread3(a2 & mask);
}

int enumerate_hilbert(lbm_lattice* L, const uint8_t* solid) {
  const int64_t X = L->X, Y = L->Y, Z = L->Z;
  int bits = 0;
  while ((int64_t(1) << bits) < std::max<int64_t>({X, Y, Z})) ++bits;
  if (3 * bits > 33)
    return set_error(LBM_ERR_UNSUPPORTED, "Hilbert enumeration limited to boxes up to 2048 per axis");
  // Raster list of fluid voxels (count per z-slab, scan, fill).
  std::vector<int64_t> cnt(Z, 0);
  parallel_for(Z, [&](int64_t zb, int64_t ze) {
    for (int64_t z = zb; z < ze; ++z) {
      int64_t c = 0;
      const uint8_t* sl = solid + z * X * Y;
      for (int64_t k = 0; k < X * Y; ++k) c += sl[k] == 0;
      cnt[z] = c;
    }
  }, 2);
  const int64_t N = exclusive_scan(cnt);
  if (N > INT32_MAX) return set_error(LBM_ERR_ARG, "more than 2^31-1 fluid nodes");
  // Sort keys: the voxel's Hilbert index above its raster rank (31 bits).  The
  // indices are unique, so sorting the keys sorts the voxels along the curve;
  // the cost follows N, not the 8^bits cells of the enclosing cube.
  using KeyVec = std::vector<uint64_t, NoInitAlloc<uint64_t>>;
  KeyVec kv, tmp;
  std::vector<int32_t, NoInitAlloc<int32_t>> raster;
  try {
    kv.resize(N);
    tmp.resize(N);
    raster.resize(3 * N);
  } catch (...) {
    return set_error(LBM_ERR_ALLOC, "out of host memory for the Hilbert sort");
  }
  parallel_for(Z, [&](int64_t zb, int64_t ze) {
    for (int64_t z = zb; z < ze; ++z) {
      int64_t n = cnt[z];
      for (int64_t y = 0; y < Y; ++y)
        for (int64_t x = 0; x < X; ++x)
          if (solid[(z * Y + y) * X + x] == 0) {
            raster[3 * n] = int32_t(x);
            raster[3 * n + 1] = int32_t(y);
            raster[3 * n + 2] = int32_t(z);
            kv[n] = (hilbert_index(uint32_t(x), uint32_t(y), uint32_t(z), bits) << 31) | uint64_t(n);
            ++n;
          }
    }
  }, 2);
  // One most-significant-digit pass on the top SB key bits (per-thread
  // histograms, scatter), then each bucket sorted on its own.
  const int kb = 3 * bits + 31;  // significant key bits
  const int SB = std::min(16, kb);
  const int shift = kb - SB;
  const int64_t NB = int64_t(1) << SB;
  const int T = n_threads();
  const int64_t chunk = std::max<int64_t>(1, (N + T - 1) / T);
  std::vector<int64_t> hist(size_t(T) * NB, 0), start(NB + 1, 0);
  parallel_for(T, [&](int64_t tb, int64_t te) {
    for (int64_t t = tb; t < te; ++t)
      for (int64_t k = t * chunk; k < std::min(N, (t + 1) * chunk); ++k) ++hist[t * NB + int64_t(kv[k] >> shift)];
  }, 2);
  int64_t acc = 0;
  for (int64_t b = 0; b < NB; ++b) {
    start[b] = acc;
    for (int t = 0; t < T; ++t) {
      const int64_t c = hist[t * NB + b];
      hist[t * NB + b] = acc;
      acc += c;
    }
  }
  start[NB] = acc;
  parallel_for(T, [&](int64_t tb, int64_t te) {
    for (int64_t t = tb; t < te; ++t)
      for (int64_t k = t * chunk; k < std::min(N, (t + 1) * chunk); ++k) tmp[hist[t * NB + int64_t(kv[k] >> shift)]++] = kv[k];
  }, 2);
  parallel_for(NB, [&](int64_t bb, int64_t be) {
    for (int64_t b = bb; b < be; ++b) std::sort(tmp.begin() + start[b], tmp.begin() + start[b + 1]);
  }, 2);
  L->N = N;
  L->node_xyz.resize(3 * N);
  parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t k = b; k < e; ++k)
      std::memcpy(&L->node_xyz[3 * k], &raster[3 * int64_t(tmp[k] & 0x7fffffffu)], 3 * sizeof(int32_t));
  });
  return LBM_OK;
}

// ---- adjacency list -------------------------------------------------------------------
int fill_adjacency(lbm_lattice* L) {
  const int64_t X = L->X, Y = L->Y, Z = L->Z, N = L->N, Np = L->Npad;
  TableVec v2n;
  try {
    v2n.resize(X * Y * Z);  // uninitialized: filled below
    L->adj.resize(18 * Np);
  } catch (...) {
    return set_error(LBM_ERR_ALLOC, "out of host memory for the adjacency list");
  }
  parallel_for(Z, [&](int64_t zb, int64_t ze) {
    std::fill(v2n.begin() + zb * X * Y, v2n.begin() + ze * X * Y, -1);
  }, 2);
  for (int i = 0; i < 18; ++i) std::fill(L->adj.begin() + i * Np + N, L->adj.begin() + (i + 1) * Np, LBM_MARK_WALL);
  parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t n = b; n < e; ++n) {
      const int32_t* p = &L->node_xyz[3 * n];
      v2n[(int64_t(p[2]) * Y + p[1]) * X + p[0]] = int32_t(n);
    }
  });
  const int64_t dim[3] = {X, Y, Z};
  const int* per = L->bc.periodic;
  const int xp = L->bc.x_pressure;
  parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t n = b; n < e; ++n) {
      const int32_t* p = &L->node_xyz[3 * n];
      for (int i = 1; i < kQ; ++i) {
        int64_t s[3] = {p[0] - kCX[i], p[1] - kCY[i], p[2] - kCZ[i]};
        bool wall = false;
        int press = 0;
        for (int a = 0; a < 3; ++a) {
          if (s[a] >= 0 && s[a] < dim[a]) continue;
          if (per[a]) {
            s[a] = (s[a] + dim[a]) % dim[a];
          } else if (a == 0 && xp) {
            press = s[a] < 0 ? LBM_MARK_INLET : LBM_MARK_OUTLET;
          } else {
            wall = true;
          }
        }
        int32_t v;
        if (wall)
          v = LBM_MARK_WALL;
        else if (press)
          v = press;
        else
          v = v2n[(s[2] * Y + s[1]) * X + s[0]];  // -1 when solid
        L->adj[(i - 1) * Np + n] = v;
      }
    }
  });
  return LBM_OK;
}

// Node n (>= 1) continues the run of node n-1 (Sect. 4.1): for every direction
// both pull from fluid nodes with source index advanced by exactly one, or both
// carry the same marker (their own-node source also advances by one).
inline bool continues(const int32_t* adj, int64_t Np, int64_t n) {
  for (int i = 0; i < 18; ++i) {
    int32_t a = adj[i * Np + n - 1], c = adj[i * Np + n];
    bool ok = (a >= 0 && c >= 0) ? (int64_t(c) == int64_t(a) + 1) : (a < 0 && c < 0 && a == c);
    if (!ok) return false;
  }
  return true;
}

}  // namespace

int derive_ria(lbm_lattice* L) {
  const int64_t N = L->N, Np = L->Npad;
  const int T = n_threads();
  const int64_t chunk = std::max<int64_t>(1, (N + T - 1) / T);
  const int64_t nchunks = N == 0 ? 0 : (N + chunk - 1) / chunk;
  std::vector<int64_t> heads(nchunks, 0);
  parallel_for(nchunks, [&](int64_t cb, int64_t ce) {
    for (int64_t c = cb; c < ce; ++c) {
      int64_t h = 0;
      for (int64_t n = c * chunk; n < std::min(N, (c + 1) * chunk); ++n)
        h += (n == 0 || !continues(L->adj.data(), Np, n));
      heads[c] = h;
    }
  }, 2);
  const int64_t R = exclusive_scan(heads);
  L->R = R;
  L->Rpad = round_up(std::max<int64_t>(R, 1), kPad);
  try {
    L->run_start.assign(R + 1, 0);
    L->run_adj.resize(18 * L->Rpad);  // rows [0, R) are filled below
  } catch (...) {
    return set_error(LBM_ERR_ALLOC, "out of host memory for the RIA table");
  }
  for (int i = 0; i < 18; ++i)
    std::fill(L->run_adj.begin() + i * L->Rpad + R, L->run_adj.begin() + (i + 1) * L->Rpad, LBM_MARK_WALL);
  parallel_for(nchunks, [&](int64_t cb, int64_t ce) {
    for (int64_t c = cb; c < ce; ++c) {
      int64_t r = heads[c];
      for (int64_t n = c * chunk; n < std::min(N, (c + 1) * chunk); ++n)
        if (n == 0 || !continues(L->adj.data(), Np, n)) {
          L->run_start[r] = int32_t(n);
          for (int i = 0; i < 18; ++i) L->run_adj[i * L->Rpad + r] = L->adj[i * Np + n];
          ++r;
        }
    }
  }, 2);
  L->run_start[R] = int32_t(N);
  // Warp-level run index: a head bit per node, and for every 32-node group the
  // run holding its first node and that run's first node.
  L->nwarps = (N + kWarpNodes - 1) / kWarpNodes;
  L->head_bits.assign(L->nwarps, 0u);
  L->warp_run0.assign(L->nwarps, 0);
  L->warp_head0.assign(L->nwarps, 0);
  for (int64_t r = 0; r < R; ++r) {
    const int64_t h = L->run_start[r];
    L->head_bits[h / kWarpNodes] |= 1u << (h % kWarpNodes);
  }
  parallel_for(L->nwarps, [&](int64_t wb, int64_t we) {
    for (int64_t w = wb; w < we; ++w) {
      const int32_t first = int32_t(w * kWarpNodes);
      auto it = std::upper_bound(L->run_start.begin(), L->run_start.begin() + R, first);
      const int32_t r = int32_t((it - L->run_start.begin()) - 1);
      L->warp_run0[w] = r;
      L->warp_head0[w] = L->run_start[r];
    }
  });
  std::memset(L->hist, 0, sizeof(L->hist));
  for (int64_t r = 0; r < R; ++r) {
    int64_t len = int64_t(L->run_start[r + 1]) - L->run_start[r];
    int b = 0;
    while ((int64_t(2) << b) <= len) ++b;
    L->hist[b]++;
  }
  return LBM_OK;
}

int build_tables_from_order(lbm_lattice* L, const uint8_t* solid, const int32_t* node_xyz, int64_t N) {
  const int64_t X = L->X, Y = L->Y, Z = L->Z;
  // every fluid voxel exactly once, nothing else
  std::vector<uint8_t> seen(X * Y * Z, 0);
  int64_t fluid = 0;
  for (int64_t v = 0; v < X * Y * Z; ++v) fluid += solid[v] == 0;
  if (fluid != N) return set_error(LBM_ERR_ARG, "node list length differs from the number of fluid voxels");
  for (int64_t n = 0; n < N; ++n) {
    const int32_t x = node_xyz[3 * n], y = node_xyz[3 * n + 1], z = node_xyz[3 * n + 2];
    if (x < 0 || x >= X || y < 0 || y >= Y || z < 0 || z >= Z)
      return set_error(LBM_ERR_ARG, "node outside the box at position " + std::to_string(n));
    const int64_t v = (int64_t(z) * Y + y) * X + x;
    if (solid[v] || seen[v]) return set_error(LBM_ERR_ARG, "node list repeats a voxel or names a solid one");
    seen[v] = 1;
  }
  L->N = N;
  L->node_xyz.assign(node_xyz, node_xyz + 3 * N);
  L->Npad = round_up(std::max<int64_t>(L->N, 1), kPad);
  if (int rc = fill_adjacency(L)) return rc;
  return derive_ria(L);
}

int renumber_partitions(const lbm_lattice* L, int P, int32_t* out) {
  const int64_t N = L->N;
  const int64_t Xs = L->X, Ys = L->Y;
  std::vector<int64_t> idx(N);
  for (int64_t n = 0; n < N; ++n) idx[n] = n;
  auto key = [&](int64_t n) {
    const int32_t* p = &L->node_xyz[3 * n];
    return (int64_t(p[2]) * Ys + p[1]) * Xs + p[0];
  };
  parallel_for(P, [&](int64_t pb, int64_t pe) {
    for (int64_t p = pb; p < pe; ++p) {
      const int64_t a = N * p / P, b = N * (p + 1) / P;
      std::sort(idx.begin() + a, idx.begin() + b, [&](int64_t u, int64_t v) { return key(u) < key(v); });
    }
  }, 2);
  for (int64_t n = 0; n < N; ++n) std::memcpy(out + 3 * n, &L->node_xyz[3 * idx[n]], 3 * sizeof(int32_t));
  return LBM_OK;
}

int partition_ghosts(const lbm_lattice* L, int P, int64_t* ghosts) {
  const int64_t N = L->N, Np = L->Npad;
  parallel_for(P, [&](int64_t pb, int64_t pe) {
    for (int64_t p = pb; p < pe; ++p) {
      const int64_t a = N * p / P, b = N * (p + 1) / P;
      int64_t g = 0;
      for (int i = 0; i < 18; ++i)
        for (int64_t n = a; n < b; ++n) {
          const int32_t m = L->adj[i * Np + n];
          g += m >= 0 && (m < a || m >= b);
        }
      ghosts[p] = g;
    }
  }, 2);
  return LBM_OK;
}

// Esoteric Twist tables.  The six locations n + (+x, +y, +z, +x+y, +x+z,
// +y+z) are the pull sources of directions 2, 4, 6, 8, 12 and 16, so a
// non-negative adjacency entry already names the fluid node there; every
// other location gets a phantom storage index N + rank, ranks in
// lexicographic order of the (wrapped) coordinates, x fastest.
int derive_et_tables(lbm_lattice* L);

// The AA odd step's slots per run.  With RIA, node n = head + off of run r
// reads f_i from slot (inv i, run_adj[i][r] + off) when the head pulls from a
// fluid node, and from its own slot (i, head + off) through a bounce-back
// marker; as a flat index of the [19][Npad] grid this is
// run_slot(i, r) + off in both cases, with
//   run_slot[i][r] = inv(i) Npad + run_adj[i][r]   (fluid source)
//                  = i Npad + run_start[r]          (bounce-back).
// The step also writes P_i to the slot f_inv(i) came from, so the same entries
// give its stores.  The OS-NT step pulls post-collision P_i from slot
// (i, run_adj[i][r] + off) of the source grid, or P_inv(i) from the node's own
// slot (inv i, head + off) through a marker: run_slot_osnt[i][r] =
// i Npad + run_adj[i][r] or inv(i) Npad + run_start[r].  This pre-resolves the
// table (the same 4 bytes per run and direction as run_adj) so the kernel
// spends one add per access.  Lattices
// with pressure markers (whose anti-bounce-back needs the marker kind) or a
// grid of 2^31 or more slots do not qualify: run_slot_state = 0.
int derive_run_slots(lbm_lattice* L) {
  if (L->run_slot_state >= 0) return LBM_OK;
  if (int64_t(19) * L->Npad >= (int64_t(1) << 31) || L->bc.x_pressure) {
    L->run_slot_state = 0;
    return LBM_OK;
  }
  try {
    std::atomic<bool> marker{false};
    parallel_for(int64_t(L->run_adj.size()), [&](int64_t b, int64_t e) {
      for (int64_t k = b; k < e; ++k)
        if (L->run_adj[size_t(k)] < LBM_MARK_WALL) {
          marker = true;
          return;
        }
    });
    if (marker) {
      L->run_slot_state = 0;
      return LBM_OK;
    }
    L->run_slot.resize(run_slot_words(L->Rpad));
    L->run_slot_osnt.resize(run_slot_words(L->Rpad));
    // element (i, r): run-major r * kSlotStride + i - 1, or direction-major (i - 1) * Rpad + r
    const size_t rs_r = LBM_SLOT_AOS ? kSlotStride : 1, rs_i = LBM_SLOT_AOS ? 1 : size_t(L->Rpad);
    parallel_for(L->Rpad, [&](int64_t rb, int64_t re) {
      for (int64_t r = rb; r < re; ++r) {
        for (int i = 1; i <= 18; ++i) {
          const size_t k = size_t(r) * rs_r + size_t(i - 1) * rs_i;
          if (r >= L->R) {
            L->run_slot[k] = L->run_slot_osnt[k] = 0;  // padding
          } else {
            const int32_t a = L->run_adj[size_t(i - 1) * L->Rpad + size_t(r)];
            const int64_t head = L->run_start[size_t(r)];
            L->run_slot[k] = a >= 0 ? int32_t(int64_t(kInv[i]) * L->Npad + a) : int32_t(int64_t(i) * L->Npad + head);
            L->run_slot_osnt[k] =
                a >= 0 ? int32_t(int64_t(i) * L->Npad + a) : int32_t(int64_t(kInv[i]) * L->Npad + head);
          }
        }
        if (LBM_SLOT_AOS)
          for (int w = 18; w < kSlotStride; ++w)
            L->run_slot[size_t(r) * kSlotStride + w] = L->run_slot_osnt[size_t(r) * kSlotStride + w] = 0;
      }
    });
  } catch (const std::bad_alloc&) {
    L->run_slot.clear();
    L->run_slot_osnt.clear();
    return set_error(LBM_ERR_ALLOC, "out of host memory for the run slot table");
  }
  L->run_slot_state = 1;
  return LBM_OK;
}

int derive_et(lbm_lattice* L) {
  if (L->et_ready) return LBM_OK;
  try {
    return derive_et_tables(L);
  } catch (const std::bad_alloc&) {
    return set_error(LBM_ERR_ALLOC, "out of host memory for the Esoteric Twist tables");
  }
}

int derive_et_tables(lbm_lattice* L) {
  if (L->partition_local)
    return set_error(LBM_ERR_UNSUPPORTED, "Esoteric Twist tables need a whole lattice, not a partition's local one");
  static const int kSrcDir[6] = {2, 4, 6, 8, 12, 16};
  static const int kOff[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  const int64_t N = L->N, Np = L->Npad;
  const bool have_xyz = int64_t(L->node_xyz.size()) == 3 * N;
  const int64_t X = L->X, Y = L->Y;
  const int64_t dim[3] = {L->X, L->Y, L->Z};
  std::vector<int32_t> nb(size_t(6) * Np, -1);
  std::vector<uint32_t> mask(Np, 0u);
  // Locations that are no fluid node's: candidates (location key, k * Np + n),
  // counted per chunk of nodes, then filled in chunk order.
  const int T = n_threads();
  const int64_t chunk = std::max<int64_t>(1, (N + T - 1) / T);
  const int64_t nchunks = N == 0 ? 0 : (N + chunk - 1) / chunk;
  std::vector<int64_t> ccount(nchunks, 0);
  parallel_for(nchunks, [&](int64_t cb, int64_t ce) {
    for (int64_t c = cb; c < ce; ++c) {
      int64_t cnt = 0;
      for (int k = 0; k < 6; ++k)
        for (int64_t n = c * chunk; n < std::min(N, (c + 1) * chunk); ++n) {
          const int32_t m = L->adj[(kSrcDir[k] - 1) * Np + n];
          if (m >= 0)
            nb[k * Np + n] = m;
          else
            ++cnt;
        }
      ccount[c] = cnt;
    }
  }, 2);
  const int64_t ncand = exclusive_scan(ccount);
  if (ncand > 0 && !have_xyz)
    return set_error(LBM_ERR_UNSUPPORTED, "Esoteric Twist phantom locations need node coordinates");
  std::vector<uint64_t> ckey(ncand);
  std::vector<int64_t> cslot(ncand);
  parallel_for(nchunks, [&](int64_t cb, int64_t ce) {
    for (int64_t c = cb; c < ce; ++c) {
      int64_t w = ccount[c];
      for (int k = 0; k < 6; ++k)
        for (int64_t n = c * chunk; n < std::min(N, (c + 1) * chunk); ++n) {
          if (L->adj[(kSrcDir[k] - 1) * Np + n] >= 0) continue;
          int64_t p[3];
          for (int a = 0; a < 3; ++a) {
            p[a] = L->node_xyz[3 * n + a] + kOff[k][a];
            if (L->bc.periodic[a] && p[a] == dim[a]) p[a] = 0;
          }
          ckey[w] = uint64_t((p[2] * (Y + 1) + p[1]) * (X + 1) + p[0]);
          cslot[w] = k * Np + n;
          ++w;
        }
    }
  }, 2);
  std::vector<uint64_t> keys(ckey);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  const int64_t M = int64_t(keys.size());
  if (N + M > INT32_MAX) return set_error(LBM_ERR_UNSUPPORTED, "too many Esoteric Twist storage locations");
  parallel_for(ncand, [&](int64_t b, int64_t e) {
    for (int64_t c = b; c < e; ++c)
      nb[cslot[c]] = int32_t(N + (std::lower_bound(keys.begin(), keys.end(), ckey[c]) - keys.begin()));
  });
  std::vector<int32_t> ph(size_t(3) * M);
  parallel_for(M, [&](int64_t b, int64_t e) {
    for (int64_t r = b; r < e; ++r) {
      ph[3 * r] = int32_t(keys[r] % uint64_t(X + 1));
      ph[3 * r + 1] = int32_t((keys[r] / uint64_t(X + 1)) % uint64_t(Y + 1));
      ph[3 * r + 2] = int32_t(keys[r] / uint64_t((X + 1) * (Y + 1)));
    }
  });
  parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t n = b; n < e; ++n) {
      uint32_t mk = 0u;
      for (int i = 1; i < kQ; ++i) {
        const int32_t m = L->adj[(i - 1) * Np + n];
        if (m < 0) mk |= 1u << (i - 1);
        if (kCX[i] != 0 && m <= LBM_MARK_INLET) mk |= 1u << (i <= 2 ? 17 + i : 13 + i);
      }
      mask[n] = mk;
    }
  });
  // run-length coding (Sect. 4.1's idea on these tables): node n continues
  // n-1's run when all six locations advance by one and the mask is equal
  auto continues_et = [&](int64_t n) {
    for (int k = 0; k < 6; ++k)
      if (int64_t(nb[k * Np + n]) != int64_t(nb[k * Np + n - 1]) + 1) return false;
    return mask[n] == mask[n - 1];
  };
  std::vector<int64_t> hcount(nchunks, 0);
  parallel_for(nchunks, [&](int64_t cb, int64_t ce) {
    for (int64_t c = cb; c < ce; ++c) {
      int64_t h = 0;
      for (int64_t n = c * chunk; n < std::min(N, (c + 1) * chunk); ++n) h += (n == 0 || !continues_et(n));
      hcount[c] = h;
    }
  }, 2);
  const int64_t R = exclusive_scan(hcount);
  std::vector<int32_t> rs(R + 1);
  parallel_for(nchunks, [&](int64_t cb, int64_t ce) {
    for (int64_t c = cb; c < ce; ++c) {
      int64_t r = hcount[c];
      for (int64_t n = c * chunk; n < std::min(N, (c + 1) * chunk); ++n)
        if (n == 0 || !continues_et(n)) rs[r++] = int32_t(n);
    }
  }, 2);
  rs[R] = int32_t(N);
  const int64_t Rpad = round_up(std::max<int64_t>(R, 1), kPad);
  std::vector<int32_t> rnb(size_t(6) * Rpad, -1);
  std::vector<uint32_t> rmask(Rpad, 0u);
  parallel_for(R, [&](int64_t b, int64_t e) {
    for (int64_t r = b; r < e; ++r) {
      for (int k = 0; k < 6; ++k) rnb[k * Rpad + r] = nb[k * Np + rs[r]];
      rmask[r] = mask[rs[r]];
    }
  });
  const int64_t nw = (N + kWarpNodes - 1) / kWarpNodes;
  std::vector<uint32_t> hb(nw, 0u);
  std::vector<int32_t> wr(nw, 0), wh(nw, 0);
  for (int64_t r = 0; r < R; ++r) hb[rs[r] / kWarpNodes] |= 1u << (rs[r] % kWarpNodes);
  for (int64_t w = 0, r = 0; w < nw; ++w) {
    while (r + 1 < R && rs[r + 1] <= w * kWarpNodes) ++r;
    wr[w] = int32_t(r);
    wh[w] = rs[r];
  }
  L->et_nb.swap(nb);
  L->et_mask.swap(mask);
  L->et_phantom.swap(ph);
  L->et_run_start.swap(rs);
  L->et_run_nb.swap(rnb);
  L->et_run_mask.swap(rmask);
  L->et_head_bits.swap(hb);
  L->et_warp_run0.swap(wr);
  L->et_warp_head0.swap(wh);
  L->et_R = R;
  L->et_Rpad = Rpad;
  L->et_S = N + M;
  L->et_Spad = round_up(std::max<int64_t>(N + M, 1), kPad);
  L->et_ready = 1;
  return LBM_OK;
}

int build_tables(lbm_lattice* L, const uint8_t* solid) {
  int rc = (L->enumeration == LBM_ENUM_HILBERT) ? enumerate_hilbert(L, solid)
                                                 : enumerate_lex(L, solid, L->block_B);
  if (rc) return rc;
  L->Npad = round_up(std::max<int64_t>(L->N, 1), kPad);
  if ((rc = fill_adjacency(L))) return rc;
  return derive_ria(L);
}

int validate(const lbm_lattice* L) {
  const int64_t N = L->N, Np = L->Npad;
  if (L->partition_local) {
    // a partition's local lattice: entries may point at ghost slots in
    // [N, Npad), so only ranges and the run table are checked here (the ghost
    // map itself is checked against the whole lattice by partition validation)
    for (int64_t k = 0; k < 18 * Np; ++k)
      if (L->adj[k] < LBM_MARK_OUTLET || L->adj[k] >= Np)
        return set_error(LBM_ERR_TABLE, "adjacency entry out of range at node " + std::to_string(k % Np));
    return validate_runs(L);
  }
  const int32_t* adj = L->adj.data();
  std::atomic<int64_t> bad{-1};
  std::atomic<int> kind{0};
  auto flag = [&](int64_t n, int k) {
    int64_t cur = -1;
    if (bad.compare_exchange_strong(cur, n)) kind = k;
  };
  parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t n = b; n < e && bad < 0; ++n)
      for (int i = 1; i < kQ; ++i) {
        int32_t m = adj[(i - 1) * Np + n];
        if (m >= 0) {
          if (m >= N) {
            flag(n, 1);
            break;
          }
          if (adj[(kInv[i] - 1) * Np + m] != n) {
            flag(n, 2);
            break;
          }
        } else if (m < LBM_MARK_OUTLET) {
          flag(n, 1);
          break;
        }
      }
  });
  if (bad >= 0)
    return set_error(LBM_ERR_TABLE, std::string(kind == 1 ? "adjacency entry out of range"
                                                          : "adjacency not reciprocal") +
                                        " at node " + std::to_string(int64_t(bad)));
  return validate_runs(L);
}

int validate_runs(const lbm_lattice* L) {
  const int64_t N = L->N, Np = L->Npad, R = L->R;
  const int32_t* adj = L->adj.data();
  std::atomic<int64_t> bad{-1};
  std::atomic<int> kind{0};
  auto flag = [&](int64_t n, int k) {
    int64_t cur = -1;
    if (bad.compare_exchange_strong(cur, n)) kind = k;
  };
  if (int64_t(L->run_start.size()) != R + 1 || L->run_start[0] != 0 || L->run_start[R] != N)
    return set_error(LBM_ERR_TABLE, "run table does not cover [0, N)");
  for (int64_t r = 0; r < R; ++r)
    if (L->run_start[r + 1] <= L->run_start[r])
      return set_error(LBM_ERR_TABLE, "run starts not strictly increasing at run " + std::to_string(r));
  parallel_for(R, [&](int64_t b, int64_t e) {
    for (int64_t r = b; r < e && bad < 0; ++r) {
      const int64_t h = L->run_start[r];
      if (h > 0 && continues(adj, Np, h)) {
        flag(r, 3);
        break;
      }
      for (int64_t n = h; n < L->run_start[r + 1]; ++n)
        for (int i = 0; i < 18; ++i) {
          int32_t a = L->run_adj[i * L->Rpad + r];
          int64_t want = a >= 0 ? int64_t(a) + (n - h) : a;
          if (want != adj[i * Np + n]) {
            flag(r, 4);
            n = L->run_start[r + 1];
            break;
          }
        }
    }
  });
  if (bad >= 0)
    return set_error(LBM_ERR_TABLE, std::string(kind == 3 ? "run is not maximal"
                                                          : "run table does not decode to the adjacency list") +
                                        " at run " + std::to_string(int64_t(bad)));
  // warp-level run index: recompute it by walking the runs once and compare
  if (int64_t(L->head_bits.size()) != L->nwarps || int64_t(L->warp_run0.size()) != L->nwarps ||
      int64_t(L->warp_head0.size()) != L->nwarps || L->nwarps != (N + kWarpNodes - 1) / kWarpNodes)
    return set_error(LBM_ERR_TABLE, "warp run index has the wrong size");
  std::vector<uint32_t> bits(L->nwarps, 0u);
  for (int64_t r = 0; r < R; ++r) bits[L->run_start[r] / kWarpNodes] |= 1u << (L->run_start[r] % kWarpNodes);
  int64_t r = 0;
  for (int64_t w = 0; w < L->nwarps; ++w) {
    while (r + 1 < R && L->run_start[r + 1] <= w * kWarpNodes) ++r;
    if (L->head_bits[w] != bits[w] || L->warp_run0[w] != r || L->warp_head0[w] != L->run_start[r])
      return set_error(LBM_ERR_TABLE, "warp run index inconsistent at node group " + std::to_string(w));
  }
  return LBM_OK;
}

}  // namespace lbm
