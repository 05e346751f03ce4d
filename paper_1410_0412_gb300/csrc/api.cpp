// C ABI of liblbm: argument checking, the opaque lattice handle, device table
// upload, and dispatch to the CUDA kernels.  See include/lbm.h for the
// contract of every entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "exact64.cuh"
#include "internal.h"

namespace lbm {

namespace {
thread_local std::string g_last_error;
}

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int make_kparams(const lbm_params* p, int prec, KParams* kp) {
  if (!p) return set_error(LBM_ERR_ARG, "params is NULL");
  if (!(p->omega_plus > 0.0 && p->omega_plus < 2.0))
    return set_error(LBM_ERR_ARG, "omega_plus must lie in (0, 2)");
  if (!(p->magic > 0.0) || !std::isfinite(p->magic)) return set_error(LBM_ERR_ARG, "magic must be > 0");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->g[a])) return set_error(LBM_ERR_ARG, "g must be finite");
  if (!std::isfinite(p->rho0) || !std::isfinite(p->rho_in) || !std::isfinite(p->rho_out))
    return set_error(LBM_ERR_ARG, "densities must be finite");
  if (prec < LBM_F64 || prec > LBM_F64_DF) return set_error(LBM_ERR_ARG, "unknown precision");
  if (prec == LBM_F16S && !p->shifted)
    return set_error(LBM_ERR_ARG, "LBM_F16S stores shifted values: set params.shifted");
  if (prec == LBM_F16S && !(p->f16_scale > 0.0 && std::isfinite(p->f16_scale)))
    return set_error(LBM_ERR_ARG, "f16_scale must be > 0");
  // Lambda = (1/l+ - 1/2)(1/l- - 1/2)  =>  1/l- = Lambda / (1/l+ - 1/2) + 1/2
  const double ep = 1.0 / p->omega_plus - 0.5;
  kp->lp = p->omega_plus;
  kp->lm = 1.0 / (p->magic / ep + 0.5);
  for (int a = 0; a < 3; ++a) kp->g[a] = p->g[a];
  kp->rho_s = p->shifted ? p->rho0 : 0.0;
  kp->rho_in = p->rho_in;
  kp->rho_out = p->rho_out;
  kp->scale = prec == LBM_F16S ? float(p->f16_scale) : 1.0f;
  kp->inv_scale = prec == LBM_F16S ? float(1.0 / p->f16_scale) : 1.0f;
  return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

namespace lbm {

int check_lat(const lbm_lattice* L) {
  if (!L) return set_error(LBM_ERR_ARG, "lattice handle is NULL");
  return LBM_OK;
}

// Any uploaded addressing (adjacency preferred) for gathers that need one.
int any_tables(const lbm_lattice* L, int* ria) {
  if (L->uploaded & LBM_TABLES_ADJ) {
    *ria = 0;
    return LBM_OK;
  }
  if (L->uploaded & LBM_TABLES_RIA) {
    *ria = 1;
    return LBM_OK;
  }
  return set_error(LBM_ERR_ARG, "no device tables uploaded");
}

int check_layout(int layout) {
  if (layout < LBM_LAYOUT_OSNT || layout > LBM_LAYOUT_ET_ODD) return set_error(LBM_ERR_ARG, "unknown layout");
  return LBM_OK;
}

// The device tables a layout's gathers need: none for AA_EVEN, the Esoteric
// Twist tables for the ET layouts, any addressing for the others.
int layout_tables(const lbm_lattice* L, int layout) {
  if (L->N == 0 || layout == LBM_LAYOUT_AA_EVEN) return LBM_OK;
  if (layout >= LBM_LAYOUT_ET_EVEN) {
    if (!(L->uploaded & LBM_TABLES_ET)) return set_error(LBM_ERR_ARG, "Esoteric Twist tables not uploaded to the device");
    return LBM_OK;
  }
  int ria;
  return any_tables(L, &ria);
}

}  // namespace lbm

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct TableLayout {
  size_t adj = 0, run_adj = 0, head_bits = 0, warp_run0 = 0, warp_head0 = 0, et_nb = 0, et_mask = 0;
  size_t et_run_nb = 0, et_run_mask = 0, et_head_bits = 0, et_warp_run0 = 0, et_warp_head0 = 0, total = 0;
  size_t run_slot = 0, run_slot_osnt = 0;
  bool has_run_slot = false;
};

TableLayout table_layout(const lbm_lattice* L, int which) {
  TableLayout t;
  size_t off = 0;
  if (which & LBM_TABLES_ADJ) {
    t.adj = off;
    off = align256(off + size_t(18) * L->Npad * 4);
  }
  if (which & LBM_TABLES_RIA) {
    t.run_adj = off;
    off = align256(off + size_t(18) * L->Rpad * 4);
    t.head_bits = off;
    off = align256(off + size_t(std::max<int64_t>(L->nwarps, 1)) * 4);
    t.warp_run0 = off;
    off = align256(off + size_t(std::max<int64_t>(L->nwarps, 1)) * 4);
    t.warp_head0 = off;
    off = align256(off + size_t(std::max<int64_t>(L->nwarps, 1)) * 4);
    if (L->run_slot_state == 1) {
      t.run_slot = off;
      t.has_run_slot = true;
      off = align256(off + run_slot_words(L->Rpad) * 4);
      t.run_slot_osnt = off;
      off = align256(off + run_slot_words(L->Rpad) * 4);
    }
  }
  if (which & LBM_TABLES_ET) {
    t.et_nb = off;
    off = align256(off + size_t(6) * L->Npad * 4);
    t.et_mask = off;
    off = align256(off + size_t(L->Npad) * 4);
    t.et_run_nb = off;
    off = align256(off + size_t(6) * L->et_Rpad * 4);
    t.et_run_mask = off;
    off = align256(off + size_t(L->et_Rpad) * 4);
    const size_t nw = size_t(std::max<int64_t>(int64_t(L->et_head_bits.size()), 1));
    t.et_head_bits = off;
    off = align256(off + nw * 4);
    t.et_warp_run0 = off;
    off = align256(off + nw * 4);
    t.et_warp_head0 = off;
    off = align256(off + nw * 4);
  }
  t.total = off;
  return t;
}

int check_tables(const lbm_lattice* L, int ria) {
  int need = ria ? LBM_TABLES_RIA : LBM_TABLES_ADJ;
  if (!(L->uploaded & need))
    return set_error(LBM_ERR_ARG, ria ? "RIA tables not uploaded to the device"
                                      : "adjacency list not uploaded to the device");
  return LBM_OK;
}

// Whole-lattice operations that a partition's local lattice cannot do alone
// (its ghost slots are not nodes).
int check_whole(const lbm_lattice* L, const char* what) {
  if (L->partition_local)
    return set_error(LBM_ERR_UNSUPPORTED, std::string(what) + " needs a whole lattice, not a partition's local lattice");
  return LBM_OK;
}

constexpr int kAllTables = LBM_TABLES_ADJ | LBM_TABLES_RIA | LBM_TABLES_ET;

}  // namespace

extern "C" {

const char* lbm_last_error(void) { return g_last_error.c_str(); }

int lbm_build_lattice(const uint8_t* solid, int X, int Y, int Z, const lbm_bc* bc, int enumeration,
                      int block_B, lbm_lattice** out) {
  if (!out) return set_error(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!solid || !bc) return set_error(LBM_ERR_ARG, "solid or bc is NULL");
  if (X < 1 || Y < 1 || Z < 1) return set_error(LBM_ERR_ARG, "box dimensions must be >= 1");
  if (int64_t(X) * Y * Z >= (int64_t(1) << 40)) return set_error(LBM_ERR_ARG, "box too large");
  if (enumeration != LBM_ENUM_LEX && enumeration != LBM_ENUM_HILBERT)
    return set_error(LBM_ERR_ARG, "unknown enumeration");
  if (enumeration == LBM_ENUM_LEX && block_B < 1) return set_error(LBM_ERR_ARG, "block_B must be >= 1");
  if (bc->x_pressure && bc->periodic[0]) return set_error(LBM_ERR_ARG, "x cannot be periodic and a pressure axis");
  lbm_lattice* L = new (std::nothrow) lbm_lattice();
  if (!L) return set_error(LBM_ERR_ALLOC, "out of host memory");
  L->X = X;
  L->Y = Y;
  L->Z = Z;
  L->bc = *bc;
  for (int a = 0; a < 3; ++a) L->bc.periodic[a] = bc->periodic[a] ? 1 : 0;
  L->bc.x_pressure = bc->x_pressure ? 1 : 0;
  L->enumeration = enumeration;
  L->block_B = block_B;
  int rc;
  try {
    rc = build_tables(L, solid);
  } catch (const std::bad_alloc&) {
    rc = set_error(LBM_ERR_ALLOC, "out of host memory while building tables");
  }
  if (rc) {
    delete L;
    return rc;
  }
  *out = L;
  return LBM_OK;
}

int lbm_build_lattice_ordered(const uint8_t* solid, int X, int Y, int Z, const lbm_bc* bc, const int32_t* node_xyz,
                              int64_t N, lbm_lattice** out) {
  if (!out) return set_error(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!solid || !bc || (N > 0 && !node_xyz)) return set_error(LBM_ERR_ARG, "solid, bc or node_xyz is NULL");
  if (X < 1 || Y < 1 || Z < 1) return set_error(LBM_ERR_ARG, "box dimensions must be >= 1");
  if (int64_t(X) * Y * Z >= (int64_t(1) << 40)) return set_error(LBM_ERR_ARG, "box too large");
  if (N < 0 || N > INT32_MAX) return set_error(LBM_ERR_ARG, "N out of range");
  if (bc->x_pressure && bc->periodic[0]) return set_error(LBM_ERR_ARG, "x cannot be periodic and a pressure axis");
  lbm_lattice* L = new (std::nothrow) lbm_lattice();
  if (!L) return set_error(LBM_ERR_ALLOC, "out of host memory");
  L->X = X;
  L->Y = Y;
  L->Z = Z;
  for (int a = 0; a < 3; ++a) L->bc.periodic[a] = bc->periodic[a] ? 1 : 0;
  L->bc.x_pressure = bc->x_pressure ? 1 : 0;
  L->enumeration = -1;
  int rc;
  try {
    rc = build_tables_from_order(L, solid, node_xyz, N);
  } catch (const std::bad_alloc&) {
    rc = set_error(LBM_ERR_ALLOC, "out of host memory while building tables");
  }
  if (rc) {
    delete L;
    return rc;
  }
  *out = L;
  return LBM_OK;
}

int lbm_renumber_partitions(const lbm_lattice* L, int P, int32_t* node_xyz_out) {
  if (int rc = check_lat(L)) return rc;
  if (P < 1 || P > L->N) return set_error(LBM_ERR_ARG, "P must be in [1, N]");
  if (!node_xyz_out) return set_error(LBM_ERR_ARG, "node_xyz_out is NULL");
  if (int64_t(L->node_xyz.size()) != 3 * L->N) return set_error(LBM_ERR_ARG, "lattice has no node coordinates");
  try {
    return renumber_partitions(L, P, node_xyz_out);
  } catch (const std::bad_alloc&) {
    return set_error(LBM_ERR_ALLOC, "out of host memory while renumbering");
  }
}

int lbm_partition_ghosts(const lbm_lattice* L, int P, int64_t* ghost_pdfs) {
  if (int rc = check_lat(L)) return rc;
  if (P < 1 || P > std::max<int64_t>(L->N, 1)) return set_error(LBM_ERR_ARG, "P must be in [1, N]");
  if (!ghost_pdfs) return set_error(LBM_ERR_ARG, "ghost_pdfs is NULL");
  return partition_ghosts(L, P, ghost_pdfs);
}

int lbm_lattice_from_adjacency(int64_t N, const int32_t* adj, const int32_t* node_xyz, lbm_lattice** out) {
  if (!out) return set_error(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (N < 0 || N > INT32_MAX) return set_error(LBM_ERR_ARG, "N out of range");
  if (N > 0 && !adj) return set_error(LBM_ERR_ARG, "adj is NULL");
  lbm_lattice* L = new (std::nothrow) lbm_lattice();
  if (!L) return set_error(LBM_ERR_ALLOC, "out of host memory");
  int rc = LBM_OK;
  try {
    L->N = N;
    L->Npad = round_up(std::max<int64_t>(N, 1), kPad);
    L->adj.assign(18 * L->Npad, LBM_MARK_WALL);
    for (int i = 0; i < 18; ++i) std::memcpy(&L->adj[i * L->Npad], adj + i * N, size_t(N) * 4);
    if (node_xyz) L->node_xyz.assign(node_xyz, node_xyz + 3 * N);
    rc = derive_ria(L);
  } catch (const std::bad_alloc&) {
    rc = set_error(LBM_ERR_ALLOC, "out of host memory");
  }
  if (rc) {
    delete L;
    return rc;
  }
  *out = L;
  return LBM_OK;
}

void lbm_free_lattice(lbm_lattice* lat) { delete lat; }

int lbm_lattice_info(const lbm_lattice* L, int64_t* N, int64_t* Npad, int64_t* R, int64_t* run_hist) {
  if (int rc = check_lat(L)) return rc;
  if (N) *N = L->N;
  if (Npad) *Npad = L->Npad;
  if (R) *R = L->R;
  if (run_hist) std::memcpy(run_hist, L->hist, sizeof(L->hist));
  return LBM_OK;
}

int lbm_export_tables(const lbm_lattice* L, int32_t* node_xyz, int32_t* adj, int32_t* run_start,
                      int32_t* run_adj) {
  if (int rc = check_lat(L)) return rc;
  if (node_xyz) {
    if (int64_t(L->node_xyz.size()) != 3 * L->N)
      return set_error(LBM_ERR_ARG, "lattice has no node coordinates");
    std::memcpy(node_xyz, L->node_xyz.data(), size_t(3 * L->N) * 4);
  }
  if (adj)
    for (int i = 0; i < 18; ++i) std::memcpy(adj + i * L->N, &L->adj[i * L->Npad], size_t(L->N) * 4);
  if (run_start) std::memcpy(run_start, L->run_start.data(), size_t(L->R + 1) * 4);
  if (run_adj)
    for (int i = 0; i < 18; ++i) std::memcpy(run_adj + i * L->R, &L->run_adj[i * L->Rpad], size_t(L->R) * 4);
  return LBM_OK;
}

int lbm_export_adjacency_rows(const lbm_lattice* L, const int64_t* nodes, int64_t count, int32_t* out) {
  if (int rc = check_lat(L)) return rc;
  if (count < 0 || (count > 0 && (!nodes || !out))) return set_error(LBM_ERR_ARG, "nodes or out is NULL");
  for (int64_t k = 0; k < count; ++k)
    if (nodes[k] < 0 || nodes[k] >= L->N) return set_error(LBM_ERR_ARG, "node index out of range");
  for (int i = 0; i < 18; ++i)
    for (int64_t k = 0; k < count; ++k) out[i * count + k] = L->adj[i * L->Npad + nodes[k]];
  return LBM_OK;
}

int lbm_check_finite(const double* values, int64_t count, void* stream) {
  if (count < 0 || (count > 0 && !values)) return set_error(LBM_ERR_ARG, "values is NULL");
  if (count == 0) return LBM_OK;
  std::vector<double> h;
  try {
    h.assign(size_t(count), 0.0);
  } catch (const std::bad_alloc&) {
    return set_error(LBM_ERR_ALLOC, "out of host memory for the check");
  }
  auto st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(h.data(), values, size_t(count) * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("check_finite: ") + cudaGetErrorString(e));
  for (int64_t k = 0; k < count; ++k)
    if (!std::isfinite(h[size_t(k)]))
      return set_error(LBM_ERR_NONFINITE, "non-finite value at index " + std::to_string(k));
  return LBM_OK;
}

int lbm_exact_moments_host(const double* d, int64_t n, double* out) {
  if (n < 0 || (n > 0 && (!d || !out))) return set_error(LBM_ERR_ARG, "d or out is NULL, or n < 0");
  for (int64_t k = 0; k < n; ++k) {
    double f[19], sa[10], da[10], drho, jx, jy, jz;
    std::memcpy(f, d + 19 * k, sizeof f);
    dev::exact_moments<true>(f, sa, da, drho, jx, jy, jz);
    double* o = out + 22 * k;
    o[0] = drho;
    o[1] = jx;
    o[2] = jy;
    o[3] = jz;
    for (int p = 1; p <= 9; ++p) {
      o[3 + p] = sa[p];
      o[12 + p] = da[p];
    }
  }
  return LBM_OK;
}

int lbm_fx_pairs_host(const double* d, const double* terms, int64_t n, double qm, double qp, int flags,
                      double* out, int* ok) {
  const int lp1 = flags & 1, general = flags & 2;
  if (n < 0 || (n > 0 && (!d || !terms || !out || !ok)))
    return set_error(LBM_ERR_ARG, "d, terms, out or ok is NULL, or n < 0");
  if (!(std::fabs(qm) < 0.5) || !(std::fabs(qp) < 0.5) || (lp1 && qp != 0.0))
    return set_error(LBM_ERR_ARG, "qm and qp must lie in (-1/2, 1/2), and qp = 0 when lp1");
  const int64_t qm_fx = dev::q64_of(qm), qp_fx = dev::q64_of(qp);
  for (int64_t k = 0; k < n; ++k) {
    double f[19], p[19];
    std::memcpy(f, d + 19 * k, sizeof f);
    const double* t = terms + 10 * k;
    int64_t Sk[10], D[10], S, Jx, Jy, Jz;
    int emax_fast;
    const bool near = dev::fx_pos_near(f, emax_fast);
    const int emax = !general && near ? dev::fx_moments<true, true>(f, Sk, D, S, Jx, Jy, Jz, emax_fast)
                                      : dev::fx_moments<true>(f, Sk, D, S, Jx, Jy, Jz);
    double* o = out + 19 * k;
    ok[k] = dev::fx_class_ok(emax, t[0], t[1], t[2], t[3], t[4], t[5], t[6], t[7], t[8], t[9]) ? 1 : 0;
    if (!ok[k]) {
      for (int i = 0; i < 19; ++i) o[i] = 0.0;
      continue;
    }
    const int kx = lp1 ? 4 : 2;
    const dev::FxClass q = dev::fx_class(emax - kx, t[0], t[1], t[2], t[3], t[4], t[5], t[6], t[7], t[8], t[9]);
    if (lp1)
      general ? dev::fx_pairs<true, 4, true>(q, D, Sk, qm_fx, qp_fx, emax - kx, p)
              : dev::fx_pairs<true, 4>(q, D, Sk, qm_fx, qp_fx, emax - kx, p);
    else
      general ? dev::fx_pairs<false, 2, true>(q, D, Sk, qm_fx, qp_fx, emax - kx, p)
              : dev::fx_pairs<false, 2>(q, D, Sk, qm_fx, qp_fx, emax - kx, p);
    o[0] = static_cast<double>(emax - kx);  // the pair scale es: units of 2^(es - 1080)
    for (int i = 1; i < 19; ++i) o[i] = p[i];
  }
  return LBM_OK;
}

int lbm_validate_tables(const lbm_lattice* L) {
  if (int rc = check_lat(L)) return rc;
  try {
    return validate(L);
  } catch (const std::bad_alloc&) {
    return set_error(LBM_ERR_ALLOC, "out of host memory while validating");
  }
}

int lbm_device_table_bytes(const lbm_lattice* L, int which, size_t* bytes) {
  if (int rc = check_lat(L)) return rc;
  if (!bytes) return set_error(LBM_ERR_ARG, "bytes is NULL");
  if (which <= 0 || which > kAllTables) return set_error(LBM_ERR_ARG, "bad table selection");
  if (which & LBM_TABLES_ET)
    if (int rc = derive_et(const_cast<lbm_lattice*>(L))) return rc;
  if (which & LBM_TABLES_RIA)
    if (int rc = derive_run_slots(const_cast<lbm_lattice*>(L))) return rc;
  *bytes = table_layout(L, which).total;
  return LBM_OK;
}

int lbm_lattice_upload(lbm_lattice* L, int which, void* dev, size_t bytes, void* stream) {
  if (int rc = check_lat(L)) return rc;
  if (which <= 0 || which > kAllTables) return set_error(LBM_ERR_ARG, "bad table selection");
  if (which & LBM_TABLES_ET)
    if (int rc = derive_et(L)) return rc;
  if (which & LBM_TABLES_RIA)
    if (int rc = derive_run_slots(L)) return rc;
  TableLayout t = table_layout(L, which);
  if (!dev) return set_error(LBM_ERR_ARG, "device table buffer is NULL");
  if (reinterpret_cast<uintptr_t>(dev) % 256) return set_error(LBM_ERR_ARG, "device table buffer not 256-byte aligned");
  if (bytes < t.total) return set_error(LBM_ERR_ARG, "device table buffer too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(dev);
  cudaError_t e = cudaSuccess;
  L->dev = DevTables{};
  L->uploaded = 0;
  if (which & LBM_TABLES_ADJ) {
    e = cudaMemcpyAsync(base + t.adj, L->adj.data(), L->adj.size() * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    L->dev.adj = reinterpret_cast<const int32_t*>(base + t.adj);
  }
  if (which & LBM_TABLES_RIA) {
    e = cudaMemcpyAsync(base + t.run_adj, L->run_adj.data(), L->run_adj.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && L->nwarps > 0)
      e = cudaMemcpyAsync(base + t.head_bits, L->head_bits.data(), L->head_bits.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && L->nwarps > 0)
      e = cudaMemcpyAsync(base + t.warp_run0, L->warp_run0.data(), L->warp_run0.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && L->nwarps > 0)
      e = cudaMemcpyAsync(base + t.warp_head0, L->warp_head0.data(), L->warp_head0.size() * 4, cudaMemcpyHostToDevice,
                          st);
    if (e == cudaSuccess && t.has_run_slot)
      e = cudaMemcpyAsync(base + t.run_slot, L->run_slot.data(), L->run_slot.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && t.has_run_slot)
      e = cudaMemcpyAsync(base + t.run_slot_osnt, L->run_slot_osnt.data(), L->run_slot_osnt.size() * 4,
                          cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    L->dev.run_adj = reinterpret_cast<const int32_t*>(base + t.run_adj);
    L->dev.run_slot = t.has_run_slot ? reinterpret_cast<const int32_t*>(base + t.run_slot) : nullptr;
    L->dev.run_slot_osnt = t.has_run_slot ? reinterpret_cast<const int32_t*>(base + t.run_slot_osnt) : nullptr;
    L->dev.head_bits = reinterpret_cast<const uint32_t*>(base + t.head_bits);
    L->dev.warp_run0 = reinterpret_cast<const int32_t*>(base + t.warp_run0);
    L->dev.warp_head0 = reinterpret_cast<const int32_t*>(base + t.warp_head0);
  }
  if (which & LBM_TABLES_ET) {
    e = cudaMemcpyAsync(base + t.et_nb, L->et_nb.data(), L->et_nb.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + t.et_mask, L->et_mask.data(), L->et_mask.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + t.et_run_nb, L->et_run_nb.data(), L->et_run_nb.size() * 4, cudaMemcpyHostToDevice,
                          st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + t.et_run_mask, L->et_run_mask.data(), L->et_run_mask.size() * 4,
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !L->et_head_bits.empty())
      e = cudaMemcpyAsync(base + t.et_head_bits, L->et_head_bits.data(), L->et_head_bits.size() * 4,
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !L->et_warp_run0.empty())
      e = cudaMemcpyAsync(base + t.et_warp_run0, L->et_warp_run0.data(), L->et_warp_run0.size() * 4,
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !L->et_warp_head0.empty())
      e = cudaMemcpyAsync(base + t.et_warp_head0, L->et_warp_head0.data(), L->et_warp_head0.size() * 4,
                          cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    L->dev.et_nb = reinterpret_cast<const int32_t*>(base + t.et_nb);
    L->dev.et_mask = reinterpret_cast<const uint32_t*>(base + t.et_mask);
    L->dev.spad = uint32_t(L->et_Spad);
    L->dev.et_run_nb = reinterpret_cast<const int32_t*>(base + t.et_run_nb);
    L->dev.et_run_mask = reinterpret_cast<const uint32_t*>(base + t.et_run_mask);
    L->dev.et_head_bits = reinterpret_cast<const uint32_t*>(base + t.et_head_bits);
    L->dev.et_warp_run0 = reinterpret_cast<const int32_t*>(base + t.et_warp_run0);
    L->dev.et_warp_head0 = reinterpret_cast<const int32_t*>(base + t.et_warp_head0);
    L->dev.et_rpad = uint32_t(L->et_Rpad);
  }
  L->dev.Npad = L->Npad;
  L->dev.Rpad = L->Rpad;
  L->dev.R = L->R;
  L->dev.nwarps = L->nwarps;
  L->dev.npad = uint32_t(L->Npad);
  L->dev.rpad = uint32_t(L->Rpad);
  L->dev.pressure = L->bc.x_pressure ? 1 : 0;
  if (!L->bc.x_pressure)  // lattices from a raw adjacency list: look for markers
    for (size_t k = 0; k < L->adj.size() && !L->dev.pressure; ++k) L->dev.pressure = L->adj[k] < LBM_MARK_WALL;
  L->uploaded = which;
  return LBM_OK;
}

int lbm_pdf_bytes(const lbm_lattice* L, int prec, size_t* bytes) {
  if (int rc = check_lat(L)) return rc;
  if (!bytes) return set_error(LBM_ERR_ARG, "bytes is NULL");
  size_t el = (prec == LBM_F64 || prec == LBM_F64_DF) ? 8 : prec == LBM_F32 ? 4 : prec == LBM_F16S ? 2 : 0;
  if (!el) return set_error(LBM_ERR_ARG, "unknown precision");
  *bytes = size_t(19) * L->Npad * el;
  return LBM_OK;
}

int lbm_init_equilibrium(const lbm_lattice* L, int prec, const lbm_params* params, void* pdf, int layout,
                         double rho0, const double u0[3], void* stream) {
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (int rc = check_layout(layout)) return rc;
  if (!pdf || !u0) return set_error(LBM_ERR_ARG, "pdf or u0 is NULL");
  if (!(rho0 > 0.0) || !std::isfinite(rho0)) return set_error(LBM_ERR_ARG, "rho0 must be > 0");
  if (int rc = layout_tables(L, layout)) return rc;
  return LBM_DISPATCH(prec, launch_init_eq_t, L, kp, pdf, layout, rho0, u0, stream);
}

int lbm_load_canonical(const lbm_lattice* L, int prec, const lbm_params* params, const double* F, void* pdf,
                       int layout, void* stream) {
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (int rc = check_layout(layout)) return rc;
  if (layout != LBM_LAYOUT_AA_EVEN)
    if (int rc = check_whole(L, "loading a pulled layout")) return rc;
  if (!pdf || (!F && L->N > 0)) return set_error(LBM_ERR_ARG, "pdf or F is NULL");
  if (int rc = layout_tables(L, layout)) return rc;
  return LBM_DISPATCH(prec, launch_load_canonical_t, L, kp, F, pdf, layout, stream);
}

int lbm_canonical_pdfs(const lbm_lattice* L, int prec, const lbm_params* params, const void* pdf, int layout,
                       double* F, void* stream) {
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (int rc = check_layout(layout)) return rc;
  if (!pdf || (!F && L->N > 0)) return set_error(LBM_ERR_ARG, "pdf or F is NULL");
  if (int rc = layout_tables(L, layout)) return rc;
  return LBM_DISPATCH(prec, launch_canonical_t, L, kp, pdf, layout, F, stream);
}

int lbm_step_osnt(const lbm_lattice* L, int prec, const lbm_params* params, const void* src, void* dst,
                  const float* s, int ria, void* stream) {
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (!src || !dst) return set_error(LBM_ERR_ARG, "src or dst is NULL");
  if (src == dst) return set_error(LBM_ERR_ARG, "OS-NT needs two distinct grids");
  if (L->N == 0) return LBM_OK;
  if (int rc = check_tables(L, ria)) return rc;
  return LBM_DISPATCH_STEP(prec, launch_osnt_t, L, kp, src, dst, s, ria ? 1 : 0, stream);
}

int lbm_step_aa(const lbm_lattice* L, int prec, const lbm_params* params, void* pdf, int parity, const float* s,
                int ria, void* stream) {
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (!pdf) return set_error(LBM_ERR_ARG, "pdf is NULL");
  if (parity != 0 && parity != 1) return set_error(LBM_ERR_ARG, "parity must be 0 or 1");
  if (L->N == 0) return LBM_OK;
  if (parity == 1)
    if (int rc = check_tables(L, ria)) return rc;
  return LBM_DISPATCH_STEP(prec, launch_aa_t, L, kp, pdf, parity, s, ria ? 1 : 0, stream);
}

int lbm_run_aa(const lbm_lattice* L, int prec, const lbm_params* params, void* pdf, int start_parity, int steps,
               const float* s, int ria, void* stream) {
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (!pdf) return set_error(LBM_ERR_ARG, "pdf is NULL");
  if (start_parity != 0 && start_parity != 1) return set_error(LBM_ERR_ARG, "parity must be 0 or 1");
  if (steps < 0) return set_error(LBM_ERR_ARG, "steps must be >= 0");
  if (L->N == 0 || steps == 0) return LBM_OK;
  if (steps > 1 || start_parity == 1)
    if (int rc = check_tables(L, ria)) return rc;
  for (int t = 0; t < steps; ++t)
    if (int rc = LBM_DISPATCH_STEP(prec, launch_aa_t, L, kp, pdf, (start_parity + t) & 1, s, ria ? 1 : 0, stream))
      return rc;
  return LBM_OK;
}

int lbm_et_info(lbm_lattice* L, int64_t* S, int64_t* Spad, int32_t* phantom_xyz) {
  if (int rc = check_lat(L)) return rc;
  if (int rc = derive_et(L)) return rc;
  if (S) *S = L->et_S;
  if (Spad) *Spad = L->et_Spad;
  if (phantom_xyz && !L->et_phantom.empty())
    std::memcpy(phantom_xyz, L->et_phantom.data(), L->et_phantom.size() * sizeof(int32_t));
  return LBM_OK;
}

int lbm_export_et_tables(lbm_lattice* L, int32_t* nb, uint32_t* mask) {
  if (int rc = check_lat(L)) return rc;
  if (int rc = derive_et(L)) return rc;
  if (nb)
    for (int k = 0; k < 6; ++k) std::memcpy(nb + k * L->N, &L->et_nb[k * L->Npad], size_t(L->N) * 4);
  if (mask) std::memcpy(mask, L->et_mask.data(), size_t(L->N) * 4);
  return LBM_OK;
}

int lbm_run_et(const lbm_lattice* L, int prec, const lbm_params* params, void* pdf, int start_parity, int steps,
               const float* s, int ria, void* stream) {
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (!pdf) return set_error(LBM_ERR_ARG, "pdf is NULL");
  if (start_parity != 0 && start_parity != 1) return set_error(LBM_ERR_ARG, "parity must be 0 or 1");
  if (steps < 0) return set_error(LBM_ERR_ARG, "steps must be >= 0");
  if (L->N == 0 || steps == 0) return LBM_OK;
  if (!(L->uploaded & LBM_TABLES_ET)) return set_error(LBM_ERR_ARG, "Esoteric Twist tables not uploaded to the device");
  for (int t = 0; t < steps; ++t)
    if (int rc = LBM_DISPATCH_STEP(prec, launch_et_t, L, kp, pdf, (start_parity + t) & 1, s, ria ? 1 : 0, stream))
      return rc;
  return LBM_OK;
}

int lbm_step_et(const lbm_lattice* L, int prec, const lbm_params* params, void* pdf, int parity, const float* s,
                int ria, void* stream) {
  return lbm_run_et(L, prec, params, pdf, parity, 1, s, ria, stream);
}

int lbm_export_et_runs(lbm_lattice* L, int64_t* R, int32_t* run_start, int32_t* run_nb, uint32_t* run_mask) {
  if (int rc = check_lat(L)) return rc;
  if (int rc = derive_et(L)) return rc;
  if (R) *R = L->et_R;
  if (run_start) std::memcpy(run_start, L->et_run_start.data(), size_t(L->et_R + 1) * 4);
  if (run_nb)
    for (int k = 0; k < 6; ++k) std::memcpy(run_nb + k * L->et_R, &L->et_run_nb[k * L->et_Rpad], size_t(L->et_R) * 4);
  if (run_mask) std::memcpy(run_mask, L->et_run_mask.data(), size_t(L->et_R) * 4);
  return LBM_OK;
}

int lbm_export_run_slots(lbm_lattice* L, int kind, int32_t* out, int* available) {
  if (int rc = check_lat(L)) return rc;
  if (kind != 0 && kind != 1) return set_error(LBM_ERR_ARG, "kind must be 0 (AA odd) or 1 (OS-NT)");
  if (!available) return set_error(LBM_ERR_ARG, "available is NULL");
  if (int rc = derive_run_slots(L)) return rc;
  *available = L->run_slot_state == 1 ? 1 : 0;
  if (!out || !*available) return LBM_OK;
  const TableVec& t = kind == 0 ? L->run_slot : L->run_slot_osnt;
  for (int64_t r = 0; r < L->R; ++r)
    for (int j = 0; j < 18; ++j)
      out[r * 18 + j] = LBM_SLOT_AOS ? t[size_t(r) * kSlotStride + j] : t[size_t(j) * L->Rpad + size_t(r)];
  return LBM_OK;
}

int lbm_reduce_workspace_bytes(const lbm_lattice* L, size_t* bytes) {
  if (int rc = check_lat(L)) return rc;
  if (!bytes) return set_error(LBM_ERR_ARG, "bytes is NULL");
  *bytes = size_t(reduce_parts(L)) * 4 * sizeof(double);
  return LBM_OK;
}

int lbm_macroscopic(const lbm_lattice* L, int prec, const lbm_params* params, const void* pdf, int layout,
                    const float* s, double* rho, double* u, double* sums, void* workspace, size_t ws_bytes,
                    void* stream) {
  if (int rc = check_lat(L)) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (int rc = check_layout(layout)) return rc;
  if (!pdf) return set_error(LBM_ERR_ARG, "pdf is NULL");
  const int64_t parts = reduce_parts(L);
  if (sums && (!workspace || ws_bytes < size_t(parts) * 4 * sizeof(double)))
    return set_error(LBM_ERR_ARG, "reduction workspace missing or too small");
  if (reinterpret_cast<uintptr_t>(workspace) % 8) return set_error(LBM_ERR_ARG, "workspace not 8-byte aligned");
  if (int rc = layout_tables(L, layout)) return rc;
  return LBM_DISPATCH(prec, launch_macroscopic_t, L, kp, pdf, layout, s, rho, u, sums,
                      static_cast<double*>(workspace), parts, stream);
}


int lbm_objective_flux(const lbm_lattice* L, int prec, const lbm_params* params, const void* pdf, int layout,
                       const float* s, double* J, void* lambda_T, double* grad_s, void* workspace, size_t ws_bytes,
                       void* stream) {
  if (int rc = check_lat(L)) return rc;
  if (int rc = check_whole(L, "the objective")) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (int rc = check_layout(layout)) return rc;
  if (!pdf || !J) return set_error(LBM_ERR_ARG, "pdf or J is NULL");
  const int64_t parts = reduce_parts(L);
  if (!workspace || ws_bytes < size_t(parts) * 4 * sizeof(double))
    return set_error(LBM_ERR_ARG, "reduction workspace missing or too small");
  if (int rc = layout_tables(L, layout)) return rc;
  return LBM_DISPATCH(prec, launch_objective_t, L, kp, pdf, layout, s, J, lambda_T, grad_s,
                      static_cast<double*>(workspace), stream);
}

int lbm_adjoint_step(const lbm_lattice* L, int prec, const lbm_params* params, const void* G_n,
                     const void* lambda_next, void* lambda_n, const float* s, double* grad_s, int ria,
                     void* stream) {
  if (int rc = check_lat(L)) return rc;
  if (int rc = check_whole(L, "the adjoint step")) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  if (!G_n || !lambda_next || !lambda_n) return set_error(LBM_ERR_ARG, "G_n, lambda_next or lambda_n is NULL");
  if (lambda_next == lambda_n) return set_error(LBM_ERR_ARG, "lambda_next and lambda_n must differ");
  if (L->N == 0) return LBM_OK;
  if (int rc = check_tables(L, ria)) return rc;
  return LBM_DISPATCH_STEP(prec, launch_adjoint_t, L, kp, G_n, lambda_next, lambda_n, s, grad_s, ria ? 1 : 0,
                           stream);
}

}  // extern "C"

namespace {

struct CkptLayout {
  size_t grid = 0, lam = 0;
  int nck = 0, nseg = 0;
  size_t ck = 0, gT = 0, seg = 0, lamA = 0, lamB = 0, red = 0, total = 0;
};

CkptLayout ckpt_layout(const lbm_lattice* L, int prec, int T, int K) {
  CkptLayout c;
  const bool f64 = prec == LBM_F64 || prec == LBM_F64_DF;
  const size_t el = f64 ? 8 : prec == LBM_F32 ? 4 : 2;
  const size_t lel = f64 ? 8 : 4;
  c.grid = align256(size_t(19) * L->Npad * el);
  c.lam = align256(size_t(19) * L->Npad * lel);
  c.nck = T > 0 ? (T + K - 1) / K : 1;
  c.nseg = std::max(2, K - 1);
  size_t off = 0;
  c.ck = off;
  off += c.grid * c.nck;
  c.gT = off;
  off += c.grid;
  c.seg = off;
  off += c.grid * c.nseg;
  c.lamA = off;
  off += c.lam;
  c.lamB = off;
  off += c.lam;
  c.red = off;
  off += align256(size_t(reduce_parts(L)) * 4 * sizeof(double));
  c.total = off;
  return c;
}

int check_ckpt_args(const lbm_lattice* L, int prec, int T, int K, void* ws, size_t ws_bytes, CkptLayout* out) {
  if (T < 0) return set_error(LBM_ERR_ARG, "T must be >= 0");
  if (K < 1) return set_error(LBM_ERR_ARG, "K must be >= 1");
  if (prec < LBM_F64 || prec > LBM_F64_DF) return set_error(LBM_ERR_ARG, "unknown precision");
  *out = ckpt_layout(L, prec, T, K);
  if (!ws || ws_bytes < out->total) return set_error(LBM_ERR_ARG, "checkpoint workspace missing or too small");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return set_error(LBM_ERR_ARG, "workspace not 256-byte aligned");
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_ckpt_workspace_bytes(const lbm_lattice* L, int prec, int T, int K, size_t* bytes) {
  if (int rc = check_lat(L)) return rc;
  if (int rc = check_whole(L, "the checkpointed gradient")) return rc;
  if (!bytes) return set_error(LBM_ERR_ARG, "bytes is NULL");
  if (T < 0 || K < 1) return set_error(LBM_ERR_ARG, "T must be >= 0 and K >= 1");
  if (prec < LBM_F64 || prec > LBM_F64_DF) return set_error(LBM_ERR_ARG, "unknown precision");
  *bytes = ckpt_layout(L, prec, T, K).total;
  return LBM_OK;
}

int lbm_flux_forward(const lbm_lattice* L, int prec, const lbm_params* params, const void* G0, const float* s,
                     int T, int K, int ria, void* ws, size_t ws_bytes, double* J, void* stream) {
  if (int rc = check_lat(L)) return rc;
  if (int rc = check_whole(L, "the checkpointed gradient")) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  CkptLayout c;
  if (int rc = check_ckpt_args(L, prec, T, K, ws, ws_bytes, &c)) return rc;
  if (!G0 || !J) return set_error(LBM_ERR_ARG, "G0 or J is NULL");
  if (L->N > 0)
    if (int rc = check_tables(L, ria)) return rc;
  char* base = static_cast<char*>(ws);
  auto st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(base + c.ck, G0, c.grid, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
  const void* cur = base + c.ck;
  for (int t = 0; t < T && L->N > 0; ++t) {
    void* dst;
    if (t + 1 == T)
      dst = base + c.gT;
    else if ((t + 1) % K == 0)
      dst = base + c.ck + c.grid * ((t + 1) / K);
    else
      dst = base + c.seg + c.grid * ((t + 1) % 2);
    if (int rc = LBM_DISPATCH_STEP(prec, launch_osnt_t, L, kp, cur, dst, s, ria ? 1 : 0, stream)) return rc;
    cur = dst;
  }
  if (T == 0) {
    e = cudaMemcpyAsync(base + c.gT, G0, c.grid, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
  }
  return LBM_DISPATCH(prec, launch_objective_t, L, kp, base + c.gT, LBM_LAYOUT_OSNT, s, J, nullptr, nullptr,
                      reinterpret_cast<double*>(base + c.red), stream);
}

int lbm_flux_backward(const lbm_lattice* L, int prec, const lbm_params* params, const float* s, int T, int K,
                      int ria, void* ws, size_t ws_bytes, double* grad_s, void* lambda_0, void* stream) {
  if (int rc = check_lat(L)) return rc;
  if (int rc = check_whole(L, "the checkpointed gradient")) return rc;
  KParams kp;
  if (int rc = make_kparams(params, prec, &kp)) return rc;
  CkptLayout c;
  if (int rc = check_ckpt_args(L, prec, T, K, ws, ws_bytes, &c)) return rc;
  if (!grad_s && L->N > 0) return set_error(LBM_ERR_ARG, "grad_s is NULL");
  if (L->N == 0) return LBM_OK;
  if (int rc = check_tables(L, ria)) return rc;
  char* base = static_cast<char*>(ws);
  auto st = static_cast<cudaStream_t>(stream);
  void* lamA = base + c.lamA;
  void* lamB = base + c.lamB;
  double* J = reinterpret_cast<double*>(base + c.red);  // scratch: the objective's J lands in the partials area
  // lambda_T = dJ/dF_T and the direct dJ/ds term (overwrites grad_s)
  if (int rc = LBM_DISPATCH(prec, launch_objective_t, L, kp, base + c.gT, LBM_LAYOUT_OSNT, s,
                            J + 4 * reduce_parts(L) - 1, lamA, grad_s, J, stream))
    return rc;
  for (int ck = c.nck - 1; ck >= 0 && T > 0; --ck) {
    const int t0 = ck * K, t1 = std::min(T, t0 + K);
    auto state = [&](int t) -> const void* {
      return t == t0 ? static_cast<const void*>(base + c.ck + c.grid * ck)
                     : static_cast<const void*>(base + c.seg + c.grid * (t - t0 - 1));
    };
    for (int t = t0; t + 1 < t1; ++t)
      if (int rc = LBM_DISPATCH_STEP(prec, launch_osnt_t, L, kp, state(t), const_cast<void*>(state(t + 1)), s,
                                     ria ? 1 : 0, stream))
        return rc;
    for (int t = t1 - 1; t >= t0; --t) {
      if (int rc = LBM_DISPATCH_STEP(prec, launch_adjoint_t, L, kp, state(t), lamA, lamB, s, grad_s, ria ? 1 : 0,
                                     stream))
        return rc;
      std::swap(lamA, lamB);
    }
  }
  if (lambda_0) {
    cudaError_t e = cudaMemcpyAsync(lambda_0, lamA, size_t(19) * L->Npad * ((prec == LBM_F64 || prec == LBM_F64_DF) ? 8 : 4),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
  }
  return LBM_OK;
}

}  // extern "C"
