// Device code of liblbm: storage traits, neighbour addressing (adjacency
// list or RIA runs), the TRT collision, and the stream-collide kernels of the
// OS-NT and AA forms.  Each kernels_<prec>.cu instantiates these templates for
// one storage precision; nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "df32.cuh"
#include "exact64.cuh"
#include "internal.h"

namespace lbm {
namespace dev {

// ---- D3Q19 (device copies; the direction order of lbm.h) ---------------------------
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1 : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1 : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1 : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int inv(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
constexpr bool same_as_host_table(int i) {
  return i == kQ || (cx(i) == kCX[i] && cy(i) == kCY[i] && cz(i) == kCZ[i] && inv(i) == kInv[i] && same_as_host_table(i + 1));
}
static_assert(same_as_host_table(0), "device and host direction tables differ");
// weight class: 0 rest, 1 axis (1/18), 2 face diagonal (1/36)
__host__ __device__ constexpr int wclass(int i) { return i == 0 ? 0 : (i <= 6 ? 1 : 2); }
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

constexpr int kBlock = 128;  // nodes per CTA of the step kernels (one node per thread)
// The resident-CTA counts below are for 128-thread CTAs; a kernel launched
// with B threads per CTA takes ctas(n, B) to keep the same threads per SM.
constexpr int ctas(int n128, int b = kBlock) { return n128 * 128 / b > 0 ? n128 * 128 / b : 1; }
// CTA size of the FP16S OS-NT step with RIA.  Sweeps on the 256^3 bed:
// 128 / 192 / 256 / 512 threads gave 44.1 / 47.0 / 49.6 / 47.5 GFLUP/s (at the
// same threads per SM).  Every other step and precision was flat or slower
// above 128 (Esoteric Twist at 256: -1.7 % to +3 %).
#ifndef LBM_OSNT_BLOCK_F16R
#define LBM_OSNT_BLOCK_F16R 256
#endif
// Minimum resident CTAs per SM of the step kernels (caps registers at
// 65536 / (128 * n)), from sweeps on GB300.  The indirect steps are
// latency-bound (index words, then gathers, then scattered stores): with RIA
// FP32 is fastest at 10 CTAs (<= 51 registers), FP16 at 12 (<= 42; 16 spills
// and loses 7 %; OS-NT-R FP16 on the paper's channel 49.1 -> 51.5 GFLUP/s from
// 10 to 12), with the adjacency list at 8 (AA odd) or 5 (OS-NT).  The
// double-float path takes 8 (AA odd) and 6 (others).  Native FP64: the AA
// steps fit 64 registers without spills and are fastest at 8 CTAs (AA-R on the
// 256^3 bed 12.8 / 13.6 / 14.2 / 14.6 GFLUP/s at 5 / 6 / 7 / 8); OS-NT and
// the Esoteric Twist step spill at 7 and take 6.
#ifndef LBM_MIN_CTAS_F64
#define LBM_MIN_CTAS_F64 6
#endif
#ifndef LBM_MIN_CTAS_F64_AA
#define LBM_MIN_CTAS_F64_AA 8
#endif
#ifndef LBM_MIN_CTAS_OSNT_RIA_F16
#define LBM_MIN_CTAS_OSNT_RIA_F16 12
#endif
template <int PREC, bool RIA> struct MinCtasOsnt { static constexpr int value = RIA ? 10 : 5; };
template <bool RIA> struct MinCtasOsnt<LBM_F16S, RIA> { static constexpr int value = RIA ? LBM_MIN_CTAS_OSNT_RIA_F16 : 5; };
template <bool RIA> struct MinCtasOsnt<LBM_F64, RIA> { static constexpr int value = LBM_MIN_CTAS_F64; };
template <bool RIA> struct MinCtasOsnt<LBM_F64_DF, RIA> { static constexpr int value = 6; };
template <int PREC> struct MinCtasEven { static constexpr int value = 5; };
template <> struct MinCtasEven<LBM_F64> { static constexpr int value = LBM_MIN_CTAS_F64_AA; };
template <> struct MinCtasEven<LBM_F64_DF> { static constexpr int value = 6; };
#ifndef LBM_MIN_CTAS_ODD_RIA
#define LBM_MIN_CTAS_ODD_RIA 10
#endif
#ifndef LBM_MIN_CTAS_ODD_RIA_F16
#define LBM_MIN_CTAS_ODD_RIA_F16 12
#endif
template <int PREC, bool RIA> struct MinCtasOdd { static constexpr int value = RIA ? LBM_MIN_CTAS_ODD_RIA : 8; };
template <bool RIA> struct MinCtasOdd<LBM_F16S, RIA> { static constexpr int value = RIA ? LBM_MIN_CTAS_ODD_RIA_F16 : 8; };
template <bool RIA> struct MinCtasOdd<LBM_F64, RIA> { static constexpr int value = LBM_MIN_CTAS_F64_AA; };
template <bool RIA> struct MinCtasOdd<LBM_F64_DF, RIA> { static constexpr int value = 8; };
// The Esoteric Twist step: every step is indirect, and a sweep of 6/8/10/12
// on GB300 put FP32 and FP16 at 10 CTAs (<= 51 registers; +3-5 % over 8),
// double-float at 8 (+3 % over 6); native FP64 takes 6 (see above).
template <int PREC> struct MinCtasEt { static constexpr int value = 10; };
template <> struct MinCtasEt<LBM_F64_DF> { static constexpr int value = 8; };
template <> struct MinCtasEt<LBM_F64> { static constexpr int value = LBM_MIN_CTAS_F64; };
static_assert(kBlock % kWarpNodes == 0, "a warp must cover one run-index group");

// ---- storage traits -----------------------------------------------------------------
// Value stored for PDF i: f_i - w_i rho_s (rho_s = 0 when unshifted), in the
// storage type; LBM_F16S additionally multiplies by the scale.
template <int PREC> struct St;

template <> struct St<LBM_F64> {
  using T = double;
  using R = double;
  static __device__ __forceinline__ R ld(const T* p, float) { return __ldg(p); }
  static __device__ __forceinline__ void st(T* p, R v, float) { *p = v; }
  static __device__ __forceinline__ void st_stream(T* p, R v, float) { __stcs(p, v); }
};

// IEEE double storage, double-float (FP32-pair) arithmetic.
template <> struct St<LBM_F64_DF> {
  using T = double;
  using R = df;
  static __device__ __forceinline__ R ld(const T* p, float) { return df_from_double(__ldg(p)); }
  static __device__ __forceinline__ void st(T* p, R v, float) { *p = double_from_df(v); }
  static __device__ __forceinline__ void st_stream(T* p, R v, float) { __stcs(p, double_from_df(v)); }
};

template <> struct St<LBM_F32> {
  using T = float;
  using R = float;
  static __device__ __forceinline__ R ld(const T* p, float) { return __ldg(p); }
  static __device__ __forceinline__ void st(T* p, R v, float) { *p = v; }
  static __device__ __forceinline__ void st_stream(T* p, R v, float) { __stcs(p, v); }
};

template <> struct St<LBM_F16S> {
  using T = __half;
  using R = float;
  static __device__ __forceinline__ R ld(const T* p, float inv_scale) {
    return __half2float(__ldg(p)) * inv_scale;
  }
  static __device__ __forceinline__ void st(T* p, R v, float scale) { *p = __float2half_rn(v * scale); }
  static __device__ __forceinline__ void st_stream(T* p, R v, float scale) {
    __stcs(p, __float2half_rn(v * scale));
  }
};

// Element (dir, node) of a [19][npad] array: 32x32 -> 64-bit multiply-add.
__device__ __forceinline__ size_t at(int dir, uint32_t npad, int node) {
  return static_cast<unsigned long long>(static_cast<unsigned>(dir)) * npad + static_cast<unsigned>(node);
}

// ---- L2 eviction priority of the index tables ------------------------------------------
// The index tables (run words, run slots, adjacency runs) are read again every
// step, while the PDF grids stream through L2 once per step and do not fit in
// it.  Index loads carry an evict-last hint, so the tables stay in L2 across
// steps as far as it holds them.  Measured on the 256^3 bed (GFLUP/s, no hint
// -> hint): FP16S OS-NT-R 41.2 -> 44.1, AA-R 56.1 -> 56.9; FP32 OS-NT-R 34.7
// -> 35.2, AA-R 37.7 -> 37.9; FP64 unchanged.  An evict-first hint on the PDF
// loads as well was slower in every form (AA-R FP16S 40.4, FP32 29.1): the AA
// steps write back to the lines they read.  The plain adjacency list (785 MB
// on the bed) and the Esoteric Twist tables gained nothing from the hint
// (within +-0.7 %) and load without it.
#ifndef LBM_L2_HINTS
#define LBM_L2_HINTS 1
#endif
__device__ __forceinline__ unsigned long long l2_keep() {
  // volatile: one policy per load instead of a 64-bit value held live across
  // the kernel (which made the FP16 / FP32 odd steps spill)
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int ldg_keep(const int* p) {
  int v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(l2_keep()));
  return v;
}
__device__ __forceinline__ unsigned ldg_keep(const unsigned* p) {
  unsigned v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(l2_keep()));
  return v;
}
__device__ __forceinline__ int4 ldg_keep(const int4* p) {
  int4 v;
  asm("ld.global.nc.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(l2_keep()));
  return v;
}
__device__ __forceinline__ int2 ldg_keep(const int2* p) {
  int2 v;
  asm("ld.global.nc.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(l2_keep()));
  return v;
}

// an index-table word (KEEP = false: a plain load; the double-float OS-NT
// step with RIA ran at 5.5 instead of 12.8 GFLUP/s on the bed with the hint)
template <bool KEEP = true, class T> __device__ __forceinline__ T ld_idx(const T* p) {
  if constexpr (LBM_L2_HINTS != 0 && KEEP)
    return ldg_keep(p);
  else
    return __ldg(p);
}
template <int PREC> constexpr bool kKeepIdx = PREC != LBM_F64_DF;

// The 18 slots of run r of a run slot table (derive_run_slots), each plus
// off: sl[j] belongs to direction j + 1.  Run-major tables take four 16-byte
// and one 8-byte load (the row is 80-byte aligned: the table starts on a
// 256-byte boundary).  With a stash column (the AA odd step's [18][kBlock]
// shared array at this thread's lane), each slot is also parked there as soon
// as it is formed; parking all 18 after the loads made the FP16 step spill
// 152 instead of 64 bytes and lose the gain.
template <bool KEEP>
__device__ __forceinline__ void run_slots(const int32_t* tbl, uint32_t rpad, int r, int off, unsigned (&sl)[18],
                                          int* stash = nullptr) {
#if LBM_SLOT_AOS
  const int4* p = reinterpret_cast<const int4*>(tbl + static_cast<size_t>(static_cast<unsigned>(r)) * kSlotStride);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    int w[4];
    if (q < 4) {
      const int4 v = ld_idx<KEEP>(p + q);
      w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
    } else {
      const int2 v = ld_idx<KEEP>(reinterpret_cast<const int2*>(p + 4));
      w[0] = v.x, w[1] = v.y, w[2] = w[3] = 0;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = 4 * q + k;
      if (j < 18) {
        sl[j] = static_cast<unsigned>(w[k] + off);
        if (stash) stash[j * kBlock] = static_cast<int>(sl[j]);
      }
    }
  }
#else
#pragma unroll
  for (int j = 0; j < 18; ++j) {
    sl[j] = static_cast<unsigned>(ld_idx<KEEP>(tbl + at(j, rpad, r)) + off);
    if (stash) stash[j * kBlock] = static_cast<int>(sl[j]);
  }
#endif
}

// ---- neighbour addressing --------------------------------------------------------------
// m[i-1] for i = 1..18: the adjacency entry of node n (node index or marker).
// Plain form: one coalesced int32 load per direction (D_idx = 72 B/node).
__device__ __forceinline__ void nbr_adj(const DevTables& t, int n, int (&m)[18]) {
#pragma unroll
  for (int i = 0; i < 18; ++i) m[i] = __ldg(t.adj + at(i, t.npad, n));
}

// RIA form (Sect. 4.1), warp-level: the run-length coding is held as one run
// head bit per node plus, per 32 nodes, the run holding the first of them and
// that run's first node.  A lane counts the heads at or below it in its warp's
// mask (popc) to get its run, and the highest such head (clz) gives the run's
// first node; every lane of a run then rebuilds its 18 entries from the head's
// (a + offset for fluid sources, the marker itself otherwise).  Lanes of one
// run read the same head entry, so only runs cost index bytes.
struct RiaCursor {
  int r;     // run of this thread's node
  int off;   // node - first node of the run
};

template <bool KEEP = true>
__device__ __forceinline__ RiaCursor ria_locate_in(const uint32_t* head_bits, const int32_t* warp_run0,
                                                   const int32_t* warp_head0, int n) {
  const int w = n >> 5;
  const unsigned lane = unsigned(n) & 31u;
  const unsigned bits = ld_idx<KEEP>(head_bits + w);
  const unsigned le = bits & (0xffffffffu >> (31u - lane));  // heads at lanes 0..lane
  RiaCursor c;
  c.r = ld_idx<KEEP>(warp_run0 + w) + __popc(le) - int(bits & 1u);
  const int head = le ? (w << 5) + (31 - __clz(le)) : ld_idx<KEEP>(warp_head0 + w);
  c.off = n - head;
  return c;
}

template <bool KEEP = true> __device__ __forceinline__ RiaCursor ria_locate(const DevTables& t, int n) {
  return ria_locate_in<KEEP>(t.head_bits, t.warp_run0, t.warp_head0, n);
}

template <bool KEEP = true> __device__ __forceinline__ void nbr_ria(const DevTables& t, RiaCursor c, int (&m)[18]) {
#pragma unroll
  for (int i = 0; i < 18; ++i) {
    const int a = ld_idx<KEEP>(t.run_adj + at(i, t.rpad, c.r));
    m[i] = a >= 0 ? a + c.off : a;
  }
}

// ---- TRT collision (Sect. 2) in pair form ------------------------------------------------
// Operates on deviations d_i = f_i - w_i rho_s and returns post-collision
// deviations.  With l+ / l- the TRT rates, a+- = 1 - l+-/2, the even and odd
// parts of each opposite pair (a, b = inv a) relax separately:
//   p_a = (1-l+)/2 (d_a+d_b) + (1-l-)/2 (d_a-d_b) + e + o
//   p_b = (1-l+)/2 (d_a+d_b) - (1-l-)/2 (d_a-d_b) + e - o
// e = l+ (feq+ - w rho_s) + a+ S+,  o = l- feq- + a- S-  (Guo forcing),
// which is f* = f - l+(f+ - feq+) - l-(f- - feq-) + a+ S+ + a- S- rewritten.
template <class R> struct CollConst {
  R lp;       // lambda+
  R qp, qm;   // (1 - l+)/2, (1 - l-)/2
  R hg[3];    // g / 2
  R g[3];
  R k0a, k0b; // l+/18, 3 a+/18 (K0 of the axis class: k0a*base - k0b*uF)
  R k0a15;    // 3/2 k0a
  R k1;       // 4.5 l+ / 18 = l+/4 (K1 of the axis class, times rho)
  R k2;       // 3 l- / 18 = l-/6   (K2 of the axis class, times rho)
  R fs;       // 9 a+ / 18 = a+/2   (axis-class scale of F in S+)
  R fo;       // 3 a- / 18 = a-/6   (axis-class scale of F in S-)
  R omlp;     // 1 - l+
  R gsv[3], gov[3];  // axis-class S+ / S- force scales times g: fs g, fo g
  R rho_s;
  R abb_in[2], abb_out[2];  // 2 w (rho_bc - rho_s) for w = 1/18 and 1/36
  double abb64_in[2], abb64_out[2];  // the same in double (the double-float odd step's FP64 gather)
  R inv_s;                  // 1 / storage scale of the scaled collision (see make_coll_step)
  long long qm_fx, qp_fx;   // qm and qp as Q64 fractions (the FP64 fixed-point pair update)
  bool gx;                  // the body force points along x (g_y = g_z = 0)
};

template <class R> inline CollConst<R> make_coll(const KParams& kp) {
  CollConst<R> c;
  const double ap = 1.0 - kp.lp / 2, am = 1.0 - kp.lm / 2;
  c.lp = R(kp.lp);
  c.qp = R((1.0 - kp.lp) / 2);
  c.qm = R((1.0 - kp.lm) / 2);
  for (int a = 0; a < 3; ++a) {
    c.g[a] = R(kp.g[a]);
    c.hg[a] = R(kp.g[a] / 2);
  }
  c.k0a = R(kp.lp / 18.0);
  c.k0b = R(3.0 * ap / 18.0);
  c.k1 = R(kp.lp / 4.0);
  c.k2 = R(kp.lm / 6.0);
  c.fs = R(ap / 2.0);
  c.fo = R(am / 6.0);
  c.omlp = R(1.0 - kp.lp);
  c.k0a15 = R(1.5 * kp.lp / 18.0);
  for (int a = 0; a < 3; ++a) {
    c.gsv[a] = R((ap / 2.0) * kp.g[a]);
    c.gov[a] = R((am / 6.0) * kp.g[a]);
  }
  c.rho_s = R(kp.rho_s);
  c.inv_s = R(1.0f);
  c.qm_fx = q64_of((1.0 - kp.lm) / 2);
  c.qp_fx = q64_of((1.0 - kp.lp) / 2);
  c.gx = kp.g[1] == 0.0 && kp.g[2] == 0.0;
  for (int k = 0; k < 2; ++k) {
    const double w = k == 0 ? 1.0 / 18.0 : 1.0 / 36.0;
    c.abb_in[k] = R(2.0 * w * (kp.rho_in - kp.rho_s));
    c.abb_out[k] = R(2.0 * w * (kp.rho_out - kp.rho_s));
    c.abb64_in[k] = 2.0 * w * (kp.rho_in - kp.rho_s);
    c.abb64_out[k] = 2.0 * w * (kp.rho_out - kp.rho_s);
  }
  return c;
}

// The step kernels of LBM_F16S work in storage units, s (f - w rho_s) with s
// the storage scale: every constant of the collision that its output is
// linear in is multiplied by s (make_coll_step), and only rho and j are taken
// back to physical units (four multiplies by 1/s), which saves a multiply per
// PDF load and per PDF store.  With a power-of-two scale (the default 2^10)
// every intermediate is exactly s times the unscaled one, so the stored
// values are the same bits.
template <int PREC> constexpr bool kScaled = PREC == LBM_F16S;

template <int PREC> inline CollConst<typename St<PREC>::R> make_coll_step(const KParams& kp) {
  using R = typename St<PREC>::R;
  CollConst<R> c = make_coll<R>(kp);
  if (kScaled<PREC>) {
    const R sc = R(kp.scale);
    c.k0a = c.k0a * sc;
    c.k0b = c.k0b * sc;
    c.k0a15 = c.k0a15 * sc;
    c.k1 = c.k1 * sc;
    c.k2 = c.k2 * sc;
    c.fs = c.fs * sc;
    c.fo = c.fo * sc;
    for (int a = 0; a < 3; ++a) {
      c.gsv[a] = c.gsv[a] * sc;
      c.gov[a] = c.gov[a] * sc;
    }
    for (int k = 0; k < 2; ++k) {
      c.abb_in[k] = c.abb_in[k] * sc;
      c.abb_out[k] = c.abb_out[k] * sc;
    }
    c.inv_s = R(kp.inv_scale);
  }
  return c;
}

// PDF loads and stores of the step kernels: storage units for LBM_F16S
// (no scale), the storage traits otherwise.
template <int PREC>
__device__ __forceinline__ typename St<PREC>::R ld_step(const typename St<PREC>::T* p, float inv_scale) {
  if constexpr (kScaled<PREC>)
    return __half2float(__ldg(p));
  else
    return St<PREC>::ld(p, inv_scale);
}
template <int PREC>
__device__ __forceinline__ void st_step(typename St<PREC>::T* p, typename St<PREC>::R v, float scale) {
  if constexpr (kScaled<PREC>)
    *p = __float2half_rn(v);
  else
    St<PREC>::st(p, v, scale);
}
template <int PREC>
__device__ __forceinline__ void st_stream_step(typename St<PREC>::T* p, typename St<PREC>::R v, float scale) {
  if constexpr (kScaled<PREC>)
    __stcs(p, __float2half_rn(v));
  else
    St<PREC>::st_stream(p, v, scale);
}

// c . v for a lattice direction with components in {-1, 0, 1}; folds at compile time.
template <class R, int X, int Y, int Z> __device__ __forceinline__ R cdot(R vx, R vy, R vz) {
  R acc = R(0);
  bool first = true;
  if (X != 0) { acc = X > 0 ? vx : -vx; first = false; }
  if (Y != 0) { acc = first ? (Y > 0 ? vy : -vy) : (Y > 0 ? acc + vy : acc - vy); first = false; }
  if (Z != 0) { acc = first ? (Z > 0 ? vz : -vz) : (Z > 0 ? acc + vz : acc - vz); }
  return acc;
}

// Pair k (first direction a = 2k-1, b = inv a) from its class's vectors
// T = K1 u + F+ and O = K2 u + F- (F+- the class's scaled forces): the even
// part is e = K0 + (c_a.u)(c_a.T), the odd part o = c_a.O.  The diagonal class
// passes K0, T and O halved.
template <class R, int K, bool LP1>
__device__ __forceinline__ void coll_pair(R (&d)[kQ], const R sa, const R da, const R ux, const R uy, const R uz,
                                          const R K0, const R Tx, const R Ty, const R Tz, const R Ox, const R Oy,
                                          const R Oz, const R qp, const R qm) {
  using ::fma;
  constexpr int a = 2 * K - 1, b = 2 * K;
  const R cu = cdot<R, cx(a), cy(a), cz(a)>(ux, uy, uz);
  const R ct = cdot<R, cx(a), cy(a), cz(a)>(Tx, Ty, Tz);
  const R co = cdot<R, cx(a), cy(a), cz(a)>(Ox, Oy, Oz);
  const R e = fma(cu, ct, K0);
  const R Ep = LP1 ? e : fma(qp, sa, e);
  const R Op = fma(qm, da, co);
  d[a] = Ep + Op;
  d[b] = Ep - Op;
}

// Pair sums sa_k = d_a + d_b and differences da_k = d_a - d_b, the density
// deviation and the momentum.  FP64 takes them exactly on the integer pipe
// (exact64.cuh), with sa converted only when the caller needs it (l+ != 1).
template <class R, bool NEED_SA, bool IEEE = false>
__device__ __forceinline__ void moments(const R (&d)[kQ], R (&sa)[10], R (&da)[10], R& drho, R& jx, R& jy, R& jz) {
  if constexpr (std::is_same<R, double>::value && !IEEE) {
    exact_moments<NEED_SA>(d, sa, da, drho, jx, jy, jz);
  } else {
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      sa[k] = d[2 * k - 1] + d[2 * k];
      da[k] = d[2 * k - 1] - d[2 * k];
    }
    drho = d[0];
#pragma unroll
    for (int k = 1; k <= 9; ++k) drho += sa[k];
    jx = da[1] + da[4] + da[5] + da[6] + da[7];
    jy = da[2] + da[4] - da[5] + da[8] + da[9];
    jz = da[3] + da[6] - da[7] + da[8] - da[9];
  }
}

// Halving: an exponent decrement for FP64 (exact64.cuh), a multiply otherwise.
__device__ __forceinline__ double halve(double x) { return halve_exact(x); }
__device__ __forceinline__ float halve(float x) { return half(x); }
__device__ __forceinline__ df halve(df x) { return half(x); }

// The per-node terms of the collision: the velocity u and the axis-class
// even constant K0 and vectors T and O (the face diagonals use them halved).
template <class R> struct NodeTerms {
  R ux, uy, uz, K0a, Tx, Ty, Tz, Ox, Oy, Oz;
};

// s: Brinkman solid fraction of the node (DRAG only).
template <class R, bool FORCE, bool DRAG>
__device__ __forceinline__ NodeTerms<R> node_terms(const CollConst<R>& c, const R s, const R drho, const R jx,
                                                   const R jy, const R jz) {
  using ::fma;
  const R rho = c.rho_s + drho;
  const R irho = recip(rho);
  R ux = fma(jx, irho, c.hg[0]);
  R uy = fma(jy, irho, c.hg[1]);
  R uz = fma(jz, irho, c.hg[2]);
  // axis-class K0 = w (l+ (drho - 3/2 rho u.u) - 3 a+ u.F) and the vectors
  // T = K1 u + a+/2 F, O = K2 u + a-/6 F (K1 = l+ rho / 4, K2 = l- rho / 6)
  R K0a, Tx, Ty, Tz, Ox, Oy, Oz;
  if (DRAG) {
    const R kd = recip(R(1) + halve(s));
    ux *= kd;
    uy *= kd;
    uz *= kd;
    const R rs = rho * s;
    const R Fx = fma(-rs, ux, rho * c.g[0]);
    const R Fy = fma(-rs, uy, rho * c.g[1]);
    const R Fz = fma(-rs, uz, rho * c.g[2]);
    const R uu = fma(ux, ux, fma(uy, uy, uz * uz));
    const R uF = fma(ux, Fx, fma(uy, Fy, uz * Fz));
    K0a = fma(-rho, c.k0a15 * uu, fma(c.k0a, drho, -c.k0b * uF));
    const R K1a = c.k1 * rho, K2a = c.k2 * rho;
    Tx = fma(K1a, ux, c.fs * Fx);
    Ty = fma(K1a, uy, c.fs * Fy);
    Tz = fma(K1a, uz, c.fs * Fz);
    Ox = fma(K2a, ux, c.fo * Fx);
    Oy = fma(K2a, uy, c.fo * Fy);
    Oz = fma(K2a, uz, c.fo * Fz);
  } else if (FORCE) {
    // uniform body force F = rho g
    const R uu = fma(ux, ux, fma(uy, uy, uz * uz));
    if (std::is_same<R, double>::value && c.gx) {
      // the usual case of a force along the flow axis x: four FP64
      // instructions fewer (uniform branch, taken by every thread or none)
      K0a = fma(-rho, fma(c.k0a15, uu, c.k0b * (ux * c.g[0])), c.k0a * drho);
      const R K1a = c.k1 * rho, K2a = c.k2 * rho;
      Tx = rho * fma(c.k1, ux, c.gsv[0]);
      Ty = K1a * uy;
      Tz = K1a * uz;
      Ox = rho * fma(c.k2, ux, c.gov[0]);
      Oy = K2a * uy;
      Oz = K2a * uz;
    } else {
      const R ug = fma(ux, c.g[0], fma(uy, c.g[1], uz * c.g[2]));
      K0a = fma(-rho, fma(c.k0a15, uu, c.k0b * ug), c.k0a * drho);
      Tx = rho * fma(c.k1, ux, c.gsv[0]);
      Ty = rho * fma(c.k1, uy, c.gsv[1]);
      Tz = rho * fma(c.k1, uz, c.gsv[2]);
      Ox = rho * fma(c.k2, ux, c.gov[0]);
      Oy = rho * fma(c.k2, uy, c.gov[1]);
      Oz = rho * fma(c.k2, uz, c.gov[2]);
    }
  } else {
    const R uu = fma(ux, ux, fma(uy, uy, uz * uz));
    K0a = fma(-rho * c.k0a15, uu, c.k0a * drho);
    const R K1a = c.k1 * rho, K2a = c.k2 * rho;
    Tx = K1a * ux;
    Ty = K1a * uy;
    Tz = K1a * uz;
    Ox = K2a * ux;
    Oy = K2a * uy;
    Oz = K2a * uz;
  }
  return NodeTerms<R>{ux, uy, uz, K0a, Tx, Ty, Tz, Ox, Oy, Oz};
}

// The nine pairs and the rest PDF from the node terms.  LP1: the caller knows
// l+ = 1, so (1 - l+)/2 = 0 and 1 - l+ = 0: the even parts relax fully to
// equilibrium, and the ten products with those zeros are skipped
// (fma(0, x, e) = e, so the values are unchanged).  sa and d[0] are only read
// when !LP1.
template <class R, bool LP1>
__device__ __forceinline__ void pair_terms(R (&d)[kQ], const CollConst<R>& c, const NodeTerms<R>& t,
                                           const R (&sa)[10], const R (&da)[10]) {
  using ::fma;
  const R ux = t.ux, uy = t.uy, uz = t.uz, K0a = t.K0a;
  const R Tx = t.Tx, Ty = t.Ty, Tz = t.Tz, Ox = t.Ox, Oy = t.Oy, Oz = t.Oz;
  // axis pairs (weight 1/18)
  coll_pair<R, 1, LP1>(d, sa[1], da[1], ux, uy, uz, K0a, Tx, Ty, Tz, Ox, Oy, Oz, c.qp, c.qm);
  coll_pair<R, 2, LP1>(d, sa[2], da[2], ux, uy, uz, K0a, Tx, Ty, Tz, Ox, Oy, Oz, c.qp, c.qm);
  coll_pair<R, 3, LP1>(d, sa[3], da[3], ux, uy, uz, K0a, Tx, Ty, Tz, Ox, Oy, Oz, c.qp, c.qm);
  // diagonal pairs (weight 1/36): every class constant halves
  const R K0b = halve(K0a);
  const R hTx = halve(Tx), hTy = halve(Ty), hTz = halve(Tz);
  const R hOx = halve(Ox), hOy = halve(Oy), hOz = halve(Oz);
  coll_pair<R, 4, LP1>(d, sa[4], da[4], ux, uy, uz, K0b, hTx, hTy, hTz, hOx, hOy, hOz, c.qp, c.qm);
  coll_pair<R, 5, LP1>(d, sa[5], da[5], ux, uy, uz, K0b, hTx, hTy, hTz, hOx, hOy, hOz, c.qp, c.qm);
  coll_pair<R, 6, LP1>(d, sa[6], da[6], ux, uy, uz, K0b, hTx, hTy, hTz, hOx, hOy, hOz, c.qp, c.qm);
  coll_pair<R, 7, LP1>(d, sa[7], da[7], ux, uy, uz, K0b, hTx, hTy, hTz, hOx, hOy, hOz, c.qp, c.qm);
  coll_pair<R, 8, LP1>(d, sa[8], da[8], ux, uy, uz, K0b, hTx, hTy, hTz, hOx, hOy, hOz, c.qp, c.qm);
  coll_pair<R, 9, LP1>(d, sa[9], da[9], ux, uy, uz, K0b, hTx, hTy, hTz, hOx, hOy, hOz, c.qp, c.qm);
  // rest PDF: p0 = (1 - l+) d0 + w0 (l+ base - 3 a+ u.F), w0 = 6 w_axis
  d[0] = LP1 ? 6.0f * K0a : fma(c.omlp, d[0], 6.0f * K0a);
}

// collide_m: the collision from given moments.
template <class R, bool FORCE, bool DRAG, bool LP1 = false>
__device__ __forceinline__ void collide_m(R (&d)[kQ], const CollConst<R>& c, const R s, const R (&sa)[10],
                                          const R (&da)[10], const R drho, const R jx, const R jy, const R jz) {
  pair_terms<R, LP1>(d, c, node_terms<R, FORCE, DRAG>(c, s, drho, jx, jy, jz), sa, da);
}

// The FP64 collision: exact fixed-point moments (exact64.cuh), the node terms
// in FP64, and the pair update in fixed point on the integer pipe when the
// node's values are in its range (fx_class_ok; a warp-uniform branch),
// otherwise in FP64 from the moments rounded to double.  NaN or Inf PDFs
// take the FP64 branch and come out NaN.
template <bool FORCE, bool DRAG, bool LP1>
__device__ __forceinline__ void collide_f64(double (&d)[kQ], const CollConst<double>& c, const double s) {
  int64_t Sk[10], D[10], S, Jx, Jy, Jz;
  // the shorter conversions when every node of the warp has positive PDFs
  // within 5 binades of its largest (full-f storage near equilibrium)
  int emax_fast, emax;
  double drho;
  if (__all_sync(__activemask(), fx_pos_near(d, emax_fast))) {
    emax = fx_moments<!LP1, true>(d, Sk, D, S, Jx, Jy, Jz, emax_fast);
    // positive PDFs: S >= the largest one's image >= 2^57, so the short conversion applies
    drho = fx_to_double_pos(S, emax);
  } else {
    emax = fx_moments<!LP1>(d, Sk, D, S, Jx, Jy, Jz);
    drho = emax < kFxMaxExp ? fx_to_double(S, emax) : dfrom(0x7ff8000000000000ull);
  }
  const NodeTerms<double> t = node_terms<double, FORCE, DRAG>(c, s, drho, fx_to_double(Jx, emax),
                                                              fx_to_double(Jy, emax), fx_to_double(Jz, emax));
  const bool ok = fx_class_ok(emax, t.ux, t.uy, t.uz, t.K0a, t.Tx, t.Ty, t.Tz, t.Ox, t.Oy, t.Oz);
  if (__all_sync(__activemask(), ok)) {
    constexpr int kx = LP1 ? 4 : 2;
    const FxClass q = fx_class(emax - kx, t.ux, t.uy, t.uz, t.K0a, t.Tx, t.Ty, t.Tz, t.Ox, t.Oy, t.Oz);
    fx_pairs<LP1, kx>(q, D, Sk, c.qm_fx, c.qp_fx, emax - kx, d);
    d[0] = LP1 ? 6.0 * t.K0a : ::fma(c.omlp, d[0], 6.0 * t.K0a);
  } else {
    double sa[10], da[10];
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      if (!LP1) sa[k] = fx_to_double(Sk[k], emax);
      da[k] = fx_to_double(D[k], emax);
    }
    pair_terms<double, LP1>(d, c, t, sa, da);
  }
}

template <class R, bool FORCE, bool DRAG, bool LP1 = false, bool SC = false>
__device__ __forceinline__ void collide(R (&d)[kQ], const CollConst<R>& c, const R s) {
  if constexpr (std::is_same<R, double>::value) {
    collide_f64<FORCE, DRAG, LP1>(d, c, s);
    return;
  }
  R sa[10], da[10], drho, jx, jy, jz;
  moments<R, !LP1>(d, sa, da, drho, jx, jy, jz);
  if (SC) {  // storage units -> physical units for the moments
    drho = drho * c.inv_s;
    jx = jx * c.inv_s;
    jy = jy * c.inv_s;
    jz = jz * c.inv_s;
  }
  collide_m<R, FORCE, DRAG, LP1>(d, c, s, sa, da, drho, jx, jy, jz);
}

// True for every thread of the warp when any active thread has `flag`: the
// anti-bounce-back work of pressure faces becomes a warp-uniform branch that
// warps away from the faces skip, instead of predicated arithmetic that every
// node would issue.
__device__ __forceinline__ bool warp_any(bool flag) { return __any_sync(__activemask(), flag); }

// ---- PDF gathers of the storage layouts ----------------------------------------------
// Pull of f_i at node n with adjacency entry m:
//   OS-NT grid (post-collision P):   P[i][m]      | marker: P[inv i][n]
//   AA grid after an odd count:      A[inv i][m]  | marker: A[i][n]
// a pressure marker (-2 / -3) turns the bounce-back value v into
// 2 w_i (rho_bc - rho_s) - v (anti-bounce-back, in deviation form).
template <int PREC, bool AA_ODD, bool SC = false>
__device__ __forceinline__ void gather(const typename St<PREC>::T* g, uint32_t npad, int n, const int (&m)[18],
                                       typename St<PREC>::R (&d)[kQ], float inv_scale,
                                       const typename St<PREC>::R (&abb_in)[2],
                                       const typename St<PREC>::R (&abb_out)[2], int pressure) {
  d[0] = SC ? ld_step<PREC>(g + n, inv_scale) : St<PREC>::ld(g + n, inv_scale);
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const int mi = m[i - 1];
    const int dir = (mi >= 0) == AA_ODD ? inv(i) : i;
    const int node = mi >= 0 ? mi : n;
    d[i] = SC ? ld_step<PREC>(g + at(dir, npad, node), inv_scale) : St<PREC>::ld(g + at(dir, npad, node), inv_scale);
  }
  if (pressure) {  // uniform: only lattices with pressure faces pay for the check
    bool face = false;
#pragma unroll
    for (int i = 1; i < kQ; ++i) face |= m[i - 1] < -1;
    if (warp_any(face)) {
#pragma unroll
      for (int i = 1; i < kQ; ++i) {
        const int mi = m[i - 1];
        if (mi < -1) d[i] = (mi == LBM_MARK_INLET ? abb_in[wclass(i) - 1] : abb_out[wclass(i) - 1]) - d[i];
      }
    }
  }
}

// ---- kernels -----------------------------------------------------------------------------
template <int PREC, bool RIA> struct OsntBlock {
  static constexpr int value = PREC == LBM_F16S && RIA ? LBM_OSNT_BLOCK_F16R : kBlock;
};

// OS-NT step: pull (indirect) from src, collide, store locally into dst with
// evict-first stores so the write stream does not push src out of L2.
template <int PREC, bool RIA, bool FORCE, bool DRAG, bool LP1 = false>
__global__ void __launch_bounds__(OsntBlock<PREC, RIA>::value,
                                  ctas(MinCtasOsnt<PREC, RIA>::value, OsntBlock<PREC, RIA>::value))
    k_osnt(DevTables t, KParams kp, CollConst<typename St<PREC>::R> c, const typename St<PREC>::T* __restrict__ src,
           typename St<PREC>::T* __restrict__ dst, const float* __restrict__ s, int N) {
  using R = typename St<PREC>::R;
  const int n0 = blockIdx.x * OsntBlock<PREC, RIA>::value;
  const int n = n0 + threadIdx.x;
  if (RIA && t.run_slot_osnt) {
    // Pre-resolved run slots (no pressure faces; the grid below 2^31 slots):
    // P_i (or P_inv(i) through a bounce-back marker) is pulled from slot
    // run_slot_osnt(i, r) + off of the flat source grid.
    if (n >= N) return;
    const RiaCursor cur = ria_locate<kKeepIdx<PREC>>(t, n);
    unsigned sl[18];
    run_slots<kKeepIdx<PREC>>(t.run_slot_osnt, t.rpad, cur.r, cur.off, sl);
    R d[kQ];
    d[0] = ld_step<PREC>(src + n, kp.inv_scale);
#pragma unroll
    for (int i = 1; i < kQ; ++i) d[i] = ld_step<PREC>(src + sl[i - 1], kp.inv_scale);
    const R sn = DRAG ? R(__ldg(s + n)) : R(0);
    collide<R, FORCE, DRAG, LP1, kScaled<PREC>>(d, c, sn);
#pragma unroll
    for (int i = 0; i < kQ; ++i) st_stream_step<PREC>(dst + at(i, t.npad, n), d[i], kp.scale);
    return;
  }
  int m[18];
  if (RIA) {
    if (n >= N) return;
    nbr_ria<kKeepIdx<PREC>>(t, ria_locate<kKeepIdx<PREC>>(t, n), m);
  } else {
    if (n >= N) return;
    nbr_adj(t, n, m);
  }
  R d[kQ];
  gather<PREC, false, kScaled<PREC>>(src, t.npad, n, m, d, kp.inv_scale, c.abb_in, c.abb_out, t.pressure);
  const R sn = DRAG ? R(__ldg(s + n)) : R(0);
  collide<R, FORCE, DRAG, LP1, kScaled<PREC>>(d, c, sn);
#pragma unroll
  for (int i = 0; i < kQ; ++i) st_stream_step<PREC>(dst + at(i, t.npad, n), d[i], kp.scale);
}

// AA even step: direct read of the 19 local PDFs, collide, write to the
// opposite local slots (no index loads at all).
template <int PREC, bool FORCE, bool DRAG, bool LP1 = false>
__global__ void __launch_bounds__(kBlock, ctas(MinCtasEven<PREC>::value)) k_aa_even(DevTables t, KParams kp, CollConst<typename St<PREC>::R> c,
                                                    typename St<PREC>::T* __restrict__ A,
                                                    const float* __restrict__ s, int N) {
  using R = typename St<PREC>::R;
  const int n = blockIdx.x * kBlock + threadIdx.x;
  if (n >= N) return;
  R d[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) d[i] = ld_step<PREC>(A + at(i, t.npad, n), kp.inv_scale);
  const R sn = DRAG ? R(__ldg(s + n)) : R(0);
  collide<R, FORCE, DRAG, LP1, kScaled<PREC>>(d, c, sn);
#pragma unroll
  for (int i = 0; i < kQ; ++i) st_step<PREC>(A + at(inv(i), t.npad, n), d[i], kp.scale);
}

// AA even step for shifted FP16 storage, two consecutive nodes per thread: one
// 4-byte half2 access per direction and thread keeps twice the bytes in flight
// of the one-node form (Npad is a multiple of 128, so every pair is aligned;
// a pair's second node may lie past N: it is loaded and computed but not
// stored).
template <bool FORCE, bool DRAG>
__global__ void __launch_bounds__(kBlock) k_aa_even_h2(DevTables t, KParams kp, CollConst<float> c,
                                                       __half* __restrict__ A, const float* __restrict__ s,
                                                       int N) {
  const int n = 2 * (blockIdx.x * kBlock + threadIdx.x);
  if (n >= N) return;
  float d0[kQ], d1[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float2 v = __half22float2(__ldg(reinterpret_cast<const __half2*>(A + at(i, t.npad, n))));
    d0[i] = v.x;  // storage units: the scale is folded into c (make_coll_step)
    d1[i] = v.y;
  }
  const float s0 = DRAG ? __ldg(s + n) : 0.0f;
  const float s1 = DRAG ? (n + 1 < N ? __ldg(s + n + 1) : 0.0f) : 0.0f;
  collide<float, FORCE, DRAG, false, true>(d0, c, s0);
  collide<float, FORCE, DRAG, false, true>(d1, c, s1);
  // the pair's second node may lie past N (odd N): write node slots only, as
  // the slot after the last node can be a partition's ghost slot
  if (n + 1 < N) {
#pragma unroll
    for (int i = 0; i < kQ; ++i)
      *reinterpret_cast<__half2*>(A + at(inv(i), t.npad, n)) = __floats2half2_rn(d0[i], d1[i]);
  } else {
#pragma unroll
    for (int i = 0; i < kQ; ++i) A[at(inv(i), t.npad, n)] = __float2half_rn(d0[i]);
  }
}

// AA odd step: read f_i from the neighbour's opposite slot A[inv i][m_i], collide,
// write p_i to A[i][m_{inv i}] -- the same 19 slots, so in place and race-free.
template <int PREC, bool RIA, bool FORCE, bool DRAG, bool LP1 = false>
__global__ void __launch_bounds__(kBlock, ctas(MinCtasOdd<PREC, RIA>::value)) k_aa_odd(DevTables t, KParams kp,
                                                                              CollConst<typename St<PREC>::R> c,
                                                                              typename St<PREC>::T* __restrict__ A,
                                                                              const float* __restrict__ s, int N) {
  using R = typename St<PREC>::R;
  // The 18 resolved entries must survive the collision: they are parked in
  // shared memory ([18][kBlock], lane-consecutive, conflict-free) rather than
  // held in registers across it or read again from L1 after it (measured
  // faster for every precision on GB300).
  __shared__ int s_m[18][kBlock];
  const int n = blockIdx.x * kBlock + threadIdx.x;
  if (n >= N) return;
  R d[kQ];
  if (RIA && t.run_slot) {
    // Pre-resolved run slots (no pressure faces; the grid below 2^31 slots):
    // f_i is read from slot run_slot(i, r) + off of the flat grid, and P_i
    // goes back to the slot f_inv(i) came from.
    const RiaCursor cur = ria_locate<kKeepIdx<PREC>>(t, n);
    unsigned sl[18];
    run_slots<kKeepIdx<PREC>>(t.run_slot, t.rpad, cur.r, cur.off, sl, &s_m[0][threadIdx.x]);
    if constexpr (PREC == LBM_F64_DF) {
      const double* g = reinterpret_cast<const double*>(A);
      double g64[kQ];
      g64[0] = __ldg(g + n);
#pragma unroll
      for (int i = 1; i < kQ; ++i) g64[i] = __ldg(g + sl[i - 1]);
      double sa64[10], da64[10], drho64, jx64, jy64, jz64;
      moments<double, !LP1, true>(g64, sa64, da64, drho64, jx64, jy64, jz64);
      R sa[10], da[10];
#pragma unroll
      for (int k = 1; k <= 9; ++k) {
        if (!LP1) sa[k] = df_from_double(sa64[k]);
        da[k] = df_from_double(da64[k]);
      }
      if (!LP1) d[0] = df_from_double(g64[0]);
      const R sn = DRAG ? R(__ldg(s + n)) : R(0);
      collide_m<R, FORCE, DRAG, LP1>(d, c, sn, sa, da, df_from_double(drho64), df_from_double(jx64),
                                     df_from_double(jy64), df_from_double(jz64));
    } else {
      d[0] = ld_step<PREC>(A + n, kp.inv_scale);
#pragma unroll
      for (int i = 1; i < kQ; ++i) d[i] = ld_step<PREC>(A + sl[i - 1], kp.inv_scale);
      const R sn = DRAG ? R(__ldg(s + n)) : R(0);
      collide<R, FORCE, DRAG, LP1, kScaled<PREC>>(d, c, sn);
    }
    st_step<PREC>(A + n, d[0], kp.scale);
#pragma unroll
    for (int i = 1; i < kQ; ++i) st_step<PREC>(A + static_cast<unsigned>(s_m[inv(i) - 1][threadIdx.x]), d[i], kp.scale);
    return;
  }
  {
    int m[18];
    if (RIA) {
      nbr_ria<kKeepIdx<PREC>>(t, ria_locate<kKeepIdx<PREC>>(t, n), m);
    } else {
      nbr_adj(t, n, m);
    }
#pragma unroll
    for (int j = 0; j < 18; ++j) s_m[j][threadIdx.x] = m[j];
    if constexpr (PREC == LBM_F64_DF) {
      // The double-float odd step leaves its FP64 pipe mostly idle: it takes
      // the moments there, in IEEE double from the loaded doubles, and
      // converts only those 13 (or 23) values to double-float.
      double g64[kQ];
      gather<LBM_F64, true>(reinterpret_cast<const double*>(A), t.npad, n, m, g64, kp.inv_scale, c.abb64_in,
                            c.abb64_out, t.pressure);
      double sa64[10], da64[10], drho64, jx64, jy64, jz64;
      moments<double, !LP1, true>(g64, sa64, da64, drho64, jx64, jy64, jz64);
      R sa[10], da[10];
#pragma unroll
      for (int k = 1; k <= 9; ++k) {
        if (!LP1) sa[k] = df_from_double(sa64[k]);
        da[k] = df_from_double(da64[k]);
      }
      if (!LP1) d[0] = df_from_double(g64[0]);
      const R sn = DRAG ? R(__ldg(s + n)) : R(0);
      collide_m<R, FORCE, DRAG, LP1>(d, c, sn, sa, da, df_from_double(drho64), df_from_double(jx64),
                                     df_from_double(jy64), df_from_double(jz64));
    } else {
      gather<PREC, true, kScaled<PREC>>(A, t.npad, n, m, d, kp.inv_scale, c.abb_in, c.abb_out, t.pressure);
    }
  }
  if constexpr (PREC != LBM_F64_DF) {
    const R sn = DRAG ? R(__ldg(s + n)) : R(0);
    collide<R, FORCE, DRAG, LP1, kScaled<PREC>>(d, c, sn);
  }
  st_step<PREC>(A + n, d[0], kp.scale);
  // p_i goes to the slot node m_{inv i} pulls it from next (or, through a
  // marker, to this node's own opposite slot)
  int mo_[18];
#pragma unroll
  for (int j = 0; j < 18; ++j) mo_[j] = s_m[j][threadIdx.x];
  bool face = false;
  if (t.pressure) {
#pragma unroll
    for (int j = 0; j < 18; ++j) face |= mo_[j] < -1;
  }
  if (t.pressure && warp_any(face)) {
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      const int mo = mo_[inv(i) - 1];
      R v = d[i];
      if (mo < -1) v = (mo == LBM_MARK_INLET ? c.abb_in[wclass(i) - 1] : c.abb_out[wclass(i) - 1]) - v;
      const int dir = mo >= 0 ? i : inv(i);
      const int node = mo >= 0 ? mo : n;
      st_step<PREC>(A + at(dir, t.npad, node), v, kp.scale);
    }
  } else {
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      const int mo = mo_[inv(i) - 1];
      const int dir = mo >= 0 ? i : inv(i);
      const int node = mo >= 0 ? mo : n;
      st_step<PREC>(A + at(dir, t.npad, node), d[i], kp.scale);
    }
  }
}

// AA odd step with RIA through the run slot table, two nodes per thread (n
// and n + kBlock of a 2 kBlock-node CTA), for FP32 storage.  The step is bound
// by the latency of its two dependent rounds of loads (run slots, then the
// scattered PDFs), not by bytes or issue; two independent nodes per thread put
// twice the loads in flight per warp.  Same arithmetic and slots as
// k_aa_odd's slot path.  Measured on the 256^3 bed: FP32 0.354 -> 0.336 ms per
// launch at 8 CTAs per SM (0.340 at 6); FP16 is slower this way (0.260 ->
// 0.293 ms at 8, 0.276 at 6: its 12 one-node CTAs already hide the latency
// better than 8 two-node ones), so it keeps k_aa_odd.
#ifndef LBM_MIN_CTAS_ODD_X2
#define LBM_MIN_CTAS_ODD_X2 8
#endif
template <int PREC, bool FORCE, bool DRAG>
__global__ void __launch_bounds__(kBlock, ctas(LBM_MIN_CTAS_ODD_X2)) k_aa_odd_x2(DevTables t, KParams kp,
                                                                         CollConst<typename St<PREC>::R> c,
                                                                         typename St<PREC>::T* __restrict__ A,
                                                                         const float* __restrict__ s, int N) {
  using R = typename St<PREC>::R;
  static_assert(std::is_same<R, float>::value, "float-collision precisions only");
  __shared__ int s_sl[2][18][kBlock];
  const int n0 = blockIdx.x * (2 * kBlock) + threadIdx.x;
  if (n0 >= N) return;
  const int n1 = n0 + kBlock;
  const bool has1 = n1 < N;
  R d0[kQ], d1[kQ];
  {
    const RiaCursor c0 = ria_locate(t, n0);
    const RiaCursor c1 = ria_locate(t, has1 ? n1 : n0);
    unsigned sl0[18], sl1[18];
    run_slots<true>(t.run_slot, t.rpad, c0.r, c0.off, sl0);
    run_slots<true>(t.run_slot, t.rpad, c1.r, c1.off, sl1);
#pragma unroll
    for (int j = 0; j < 18; ++j) {
      s_sl[0][j][threadIdx.x] = static_cast<int>(sl0[j]);
      s_sl[1][j][threadIdx.x] = static_cast<int>(sl1[j]);
    }
    d0[0] = ld_step<PREC>(A + n0, kp.inv_scale);
    d1[0] = ld_step<PREC>(A + (has1 ? n1 : n0), kp.inv_scale);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      d0[i] = ld_step<PREC>(A + sl0[i - 1], kp.inv_scale);
      d1[i] = ld_step<PREC>(A + sl1[i - 1], kp.inv_scale);
    }
  }
  const R s0 = DRAG ? R(__ldg(s + n0)) : R(0);
  collide<R, FORCE, DRAG, false, kScaled<PREC>>(d0, c, s0);
  st_step<PREC>(A + n0, d0[0], kp.scale);
#pragma unroll
  for (int i = 1; i < kQ; ++i)
    st_step<PREC>(A + static_cast<unsigned>(s_sl[0][inv(i) - 1][threadIdx.x]), d0[i], kp.scale);
  if (has1) {
    const R s1 = DRAG ? R(__ldg(s + n1)) : R(0);
    collide<R, FORCE, DRAG, false, kScaled<PREC>>(d1, c, s1);
    st_step<PREC>(A + n1, d1[0], kp.scale);
#pragma unroll
    for (int i = 1; i < kQ; ++i)
      st_step<PREC>(A + static_cast<unsigned>(s_sl[1][inv(i) - 1][threadIdx.x]), d1[i], kp.scale);
  }
}

// ---- Esoteric Twist: one grid, in place (named in Sect. 1 and Sect. 4) ------------------
// The link between n and n + c_i keeps its two slots (one per travel
// direction) at location n + c_i^+, c^+ = componentwise max(c, 0), so a node
// touches only itself and six neighbour locations, whose storage indices are
// the table et_nb[6][Npad] (+x, +y, +z, +x+y, +x+z, +y+z; phantom locations
// past N hold the slots of links through non-fluid cells).  Even step: read
// f_i from slot i at n + c_inv(i)^+, write P_j to slot inv(j) at n + c_j^+ (the
// slot f_inv(j) came from).  Odd step: slots inv(i) and j.  A link to a wall
// or a pressure face (et_mask bit inv(j) - 1) stores the bounced value in the
// pair's other slot, the one this node reads next step.
__host__ __device__ constexpr int et_row(int i) {
  return (cx(i) > 0 ? 1 : 0) + (cy(i) > 0 ? 2 : 0) + (cz(i) > 0 ? 4 : 0) == 0   ? -1
         : (cx(i) > 0 ? 1 : 0) + (cy(i) > 0 ? 2 : 0) + (cz(i) > 0 ? 4 : 0) == 1 ? 0
         : (cx(i) > 0 ? 1 : 0) + (cy(i) > 0 ? 2 : 0) + (cz(i) > 0 ? 4 : 0) == 2 ? 1
         : (cx(i) > 0 ? 1 : 0) + (cy(i) > 0 ? 2 : 0) + (cz(i) > 0 ? 4 : 0) == 4 ? 2
         : (cx(i) > 0 ? 1 : 0) + (cy(i) > 0 ? 2 : 0) + (cz(i) > 0 ? 4 : 0) == 3 ? 3
         : (cx(i) > 0 ? 1 : 0) + (cy(i) > 0 ? 2 : 0) + (cz(i) > 0 ? 4 : 0) == 5 ? 4
                                                                                : 5;
}
// et_mask bit of "pull direction i (c_ix != 0) meets a pressure face"
__host__ __device__ constexpr int et_xbit(int i) { return i <= 2 ? 17 + i : 13 + i; }
static_assert(et_row(1) == 0 && et_row(2) == -1 && et_row(7) == 3 && et_row(9) == 0 && et_row(10) == 1 &&
                  et_row(11) == 4 && et_row(14) == 2 && et_row(15) == 5 && et_row(17) == 1 && et_row(18) == 2,
              "ET location rows");
static_assert(et_xbit(1) == 18 && et_xbit(2) == 19 && et_xbit(7) == 20 && et_xbit(14) == 27, "ET pressure bits");

__device__ __forceinline__ void et_locations(const DevTables& t, int n, int (&loc)[7]) {
  loc[0] = n;
#pragma unroll
  for (int k = 0; k < 6; ++k) loc[k + 1] = __ldg(t.et_nb + at(k, t.npad, n));
}

// The node's locations and link mask, from the plain tables (28 B per node) or
// from their run-length coding (RIA, Sect. 4.1: runs of nodes whose six
// locations advance by one and whose masks agree; found with the same
// warp-level run index as the adjacency runs).
template <bool RIA>
__device__ __forceinline__ unsigned et_locate(const DevTables& t, int n, int (&loc)[7]) {
  if (!RIA) {
    et_locations(t, n, loc);
    return __ldg(t.et_mask + n);
  }
  const RiaCursor c = ria_locate_in<false>(t.et_head_bits, t.et_warp_run0, t.et_warp_head0, n);
  loc[0] = n;
#pragma unroll
  for (int k = 0; k < 6; ++k) loc[k + 1] = __ldg(t.et_run_nb + at(k, t.et_rpad, c.r)) + c.off;
  return __ldg(t.et_run_mask + c.r);
}

template <int PREC, bool RIA, bool ODD, bool FORCE, bool DRAG, bool LP1 = false>
__global__ void __launch_bounds__(kBlock, ctas(MinCtasEt<PREC>::value)) k_et(DevTables t, KParams kp,
                                                                          CollConst<typename St<PREC>::R> c,
                                                                          typename St<PREC>::T* __restrict__ A,
                                                                          const float* __restrict__ s, int N) {
  using R = typename St<PREC>::R;
  // As in the AA odd step, the wider precisions park the six locations and
  // the mask in shared memory across the collision (lane-consecutive, no bank
  // conflicts); FP16 keeps them in registers.
  constexpr bool kStash = PREC != LBM_F16S;
  __shared__ int s_loc[kStash ? 7 : 1][kBlock];
  const int n = blockIdx.x * kBlock + threadIdx.x;
  if (n >= N) return;
  int loc[7];
  unsigned mask = et_locate<RIA>(t, n, loc);
  R d[kQ];
  d[0] = ld_step<PREC>(A + n, kp.inv_scale);
#pragma unroll
  for (int i = 1; i < kQ; ++i)
    d[i] = ld_step<PREC>(A + at(ODD ? inv(i) : i, t.spad, loc[et_row(inv(i)) + 1]), kp.inv_scale);
  if (kStash) {
#pragma unroll
    for (int k = 1; k < 7; ++k) s_loc[k - 1][threadIdx.x] = loc[k];
    s_loc[6][threadIdx.x] = int(mask);
  }
  const R sn = DRAG ? R(__ldg(s + n)) : R(0);
  collide<R, FORCE, DRAG, LP1, kScaled<PREC>>(d, c, sn);
  st_step<PREC>(A + n, d[0], kp.scale);
  if (kStash) {
#pragma unroll
    for (int k = 1; k < 7; ++k) loc[k] = s_loc[k - 1][threadIdx.x];
    mask = unsigned(s_loc[6][threadIdx.x]);
  }
  // bits 18..27 of the mask: pull directions that meet a pressure face.  The
  // FP64 path branches per warp around the anti-bounce-back arithmetic (a
  // predicated subtraction would be issued for all ten x-directions of every
  // node); the others keep one predicated loop (fewer registers, cheap
  // arithmetic).
  if constexpr (std::is_same<R, double>::value) {
    if (t.pressure && warp_any((mask >> 18) != 0u)) {
#pragma unroll
      for (int j = 1; j < kQ; ++j) {
        const int jj = inv(j);
        const bool link = !((mask >> (jj - 1)) & 1u);
        R v = d[j];
        if (cx(jj) != 0 && ((mask >> et_xbit(jj)) & 1u))
          v = (cx(jj) > 0 ? c.abb_in[wclass(j) - 1] : c.abb_out[wclass(j) - 1]) - v;
        st_step<PREC>(A + at(link != ODD ? jj : j, t.spad, loc[et_row(j) + 1]), v, kp.scale);
      }
    } else {
#pragma unroll
      for (int j = 1; j < kQ; ++j) {
        const int jj = inv(j);
        const bool link = !((mask >> (jj - 1)) & 1u);
        st_step<PREC>(A + at(link != ODD ? jj : j, t.spad, loc[et_row(j) + 1]), d[j], kp.scale);
      }
    }
  } else {
#pragma unroll
    for (int j = 1; j < kQ; ++j) {
      const int jj = inv(j);
      const bool link = !((mask >> (jj - 1)) & 1u);
      R v = d[j];
      if (cx(jj) != 0) {
        if (t.pressure && ((mask >> et_xbit(jj)) & 1u))
          v = (cx(jj) > 0 ? c.abb_in[wclass(j) - 1] : c.abb_out[wclass(j) - 1]) - v;
      }
      st_step<PREC>(A + at(link != ODD ? jj : j, t.spad, loc[et_row(j) + 1]), v, kp.scale);
    }
  }
}

}  // namespace dev
}  // namespace lbm

namespace lbm {
namespace dev {

// ---- state set-up and read-back kernels ------------------------------------------------

// Fill a grid so that its canonical state is the uniform f^eq given in feq[19]
// (FP64, unshifted).  AA_EVEN layout stores f^eq directly; the OS-NT layout
// stores the slot (j, n) as the value node adj(inv j, n) pulls from it:
// f^eq_j for a fluid puller, f^eq_{inv j} for bounce-back, and
// 2 w_j rho_bc - f^eq_{inv j} for anti-bounce-back; the AA_ODD layout holds
// that same value in slot (inv j, n).
struct Feq19 {
  double v[kQ];
};

template <int PREC, bool RIA>
__global__ void __launch_bounds__(kBlock) k_init_eq(DevTables t, KParams kp, Feq19 feq, typename St<PREC>::T* pdf,
                                                    int layout, int N) {
  using R = typename St<PREC>::R;
  const int n0 = blockIdx.x * kBlock;
  const int n = n0 + threadIdx.x;
  if (layout >= LBM_LAYOUT_ET_EVEN) {  // every slot a node reads holds its f_i directly
    if (n >= N) return;
    int loc[7];
    et_locations(t, n, loc);
    St<PREC>::st(pdf + n, R(feq.v[0] - wgt(0) * kp.rho_s), kp.scale);
#pragma unroll
    for (int i = 1; i < kQ; ++i)
      St<PREC>::st(pdf + at(layout == LBM_LAYOUT_ET_ODD ? inv(i) : i, t.spad, loc[et_row(inv(i)) + 1]),
                   R(feq.v[i] - wgt(i) * kp.rho_s), kp.scale);
    return;
  }
  int m[18];
  if (layout != LBM_LAYOUT_AA_EVEN) {
    if (RIA) {
      if (n >= N) return;
      nbr_ria(t, ria_locate(t, n), m);
    } else {
      if (n >= N) return;
      nbr_adj(t, n, m);
    }
  } else if (n >= N) {
    return;
  }
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    double v = feq.v[j];
    int slot = j;
    if (layout != LBM_LAYOUT_AA_EVEN && j > 0) {
      const int mp = m[inv(j) - 1];
      if (mp < 0) v = feq.v[inv(j)];
      if (mp < -1) v = wgt(j) * 2.0 * (mp == LBM_MARK_INLET ? kp.rho_in : kp.rho_out) - v;
      if (layout == LBM_LAYOUT_AA_ODD) slot = inv(j);
    }
    St<PREC>::st(pdf + at(slot, t.npad, n), R(v - wgt(j) * kp.rho_s), kp.scale);
  }
}

// Store a canonical FP64 state F[19][N] into a grid of the given layout (the
// general form of k_init_eq: the fluid puller's value is read from F at that
// node).
template <int PREC, bool RIA>
__global__ void __launch_bounds__(kBlock) k_load_canonical(DevTables t, KParams kp, const double* __restrict__ F,
                                                           typename St<PREC>::T* pdf, int layout, int N) {
  using R = typename St<PREC>::R;
  const int n0 = blockIdx.x * kBlock;
  const int n = n0 + threadIdx.x;
  if (layout >= LBM_LAYOUT_ET_EVEN) {
    if (n >= N) return;
    int loc[7];
    et_locations(t, n, loc);
    St<PREC>::st(pdf + n, R(F[n] - wgt(0) * kp.rho_s), kp.scale);
#pragma unroll
    for (int i = 1; i < kQ; ++i)
      St<PREC>::st(pdf + at(layout == LBM_LAYOUT_ET_ODD ? inv(i) : i, t.spad, loc[et_row(inv(i)) + 1]),
                   R(F[size_t(i) * N + n] - wgt(i) * kp.rho_s), kp.scale);
    return;
  }
  int m[18];
  if (layout != LBM_LAYOUT_AA_EVEN) {
    if (RIA) {
      if (n >= N) return;
      nbr_ria(t, ria_locate(t, n), m);
    } else {
      if (n >= N) return;
      nbr_adj(t, n, m);
    }
  } else if (n >= N) {
    return;
  }
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    double v;
    int slot = j;
    if (layout == LBM_LAYOUT_AA_EVEN || j == 0) {
      v = F[size_t(j) * N + n];
    } else {
      const int mp = m[inv(j) - 1];
      if (mp >= 0) {
        v = F[size_t(j) * N + mp];
      } else {
        v = F[size_t(inv(j)) * N + n];
        if (mp < -1) v = wgt(j) * 2.0 * (mp == LBM_MARK_INLET ? kp.rho_in : kp.rho_out) - v;
      }
      if (layout == LBM_LAYOUT_AA_ODD) slot = inv(j);
    }
    St<PREC>::st(pdf + at(slot, t.npad, n), R(v - wgt(j) * kp.rho_s), kp.scale);
  }
}

// Canonical pre-collision state of one node, FP64, unshifted.
// SHIFT: add the storage shift w_i rho_s back (the canonical PDFs); without
// it F holds the stored deviations, for callers that form exact moments.
template <int PREC, bool RIA, bool SHIFT = true>
__device__ __forceinline__ bool node_canonical(const DevTables& t, const KParams& kp,
                                               const CollConst<typename St<PREC>::R>& c,
                                               const typename St<PREC>::T* pdf, int layout, int n, int N,
                                               double (&F)[kQ]) {
  using R = typename St<PREC>::R;
  R d[kQ];
  if (layout >= LBM_LAYOUT_ET_EVEN) {
    if (n >= N) return false;
    int loc[7];
    et_locations(t, n, loc);
    d[0] = St<PREC>::ld(pdf + n, kp.inv_scale);
#pragma unroll
    for (int i = 1; i < kQ; ++i)
      d[i] = St<PREC>::ld(pdf + at(layout == LBM_LAYOUT_ET_ODD ? inv(i) : i, t.spad, loc[et_row(inv(i)) + 1]),
                          kp.inv_scale);
#pragma unroll
    for (int i = 0; i < kQ; ++i) F[i] = SHIFT ? double(d[i]) + wgt(i) * kp.rho_s : double(d[i]);
    return true;
  }
  int m[18];
  if (layout != LBM_LAYOUT_AA_EVEN) {
    if (RIA) {
      if (n >= N) return false;
      nbr_ria(t, ria_locate(t, n), m);
    } else {
      if (n >= N) return false;
      nbr_adj(t, n, m);
    }
  } else if (n >= N) {
    return false;
  }
  if (layout == LBM_LAYOUT_AA_EVEN) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) d[i] = St<PREC>::ld(pdf + at(i, t.npad, n), kp.inv_scale);
  } else if (layout == LBM_LAYOUT_OSNT) {
    gather<PREC, false>(pdf, t.npad, n, m, d, kp.inv_scale, c.abb_in, c.abb_out, t.pressure);
  } else {
    gather<PREC, true>(pdf, t.npad, n, m, d, kp.inv_scale, c.abb_in, c.abb_out, t.pressure);
  }
#pragma unroll
  for (int i = 0; i < kQ; ++i) F[i] = SHIFT ? double(d[i]) + wgt(i) * kp.rho_s : double(d[i]);
  return true;
}

template <int PREC, bool RIA>
__global__ void __launch_bounds__(kBlock) k_canonical(DevTables t, KParams kp, CollConst<typename St<PREC>::R> c,
                                                      const typename St<PREC>::T* pdf, int layout,
                                                      double* __restrict__ F, int N) {
  const int n0 = blockIdx.x * kBlock;
  const int n = n0 + threadIdx.x;
  double f[kQ];
  if (!node_canonical<PREC, RIA>(t, kp, c, pdf, layout, n, N, f)) return;
#pragma unroll
  for (int i = 0; i < kQ; ++i) F[size_t(i) * N + n] = f[i];
}

// Block-wide sum of 4 doubles; result valid in thread 0.  Fixed order.
__device__ __forceinline__ void block_sum4(double (&v)[4], double (*s_red)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) s_red[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double acc = s_red[0][k];
      for (int j = 1; j < int(blockDim.x >> 5); ++j) acc += s_red[j][k];
      v[k] = acc;
    }
  }
}

// rho, u = (j0/rho + g/2)/(1 + s/2) per node and per-CTA partial sums of
// [rho, rho u_x, rho u_y, rho u_z] (FP64).
template <int PREC, bool RIA>
__global__ void __launch_bounds__(kBlock) k_macro(DevTables t, KParams kp, CollConst<typename St<PREC>::R> c,
                                                  const typename St<PREC>::T* pdf, int layout,
                                                  const float* __restrict__ s, double* __restrict__ rho,
                                                  double* __restrict__ u, double* __restrict__ partials, int N) {
  __shared__ double s_red[kBlock / 32][4];
  const int n0 = blockIdx.x * kBlock;
  const int n = n0 + threadIdx.x;
  double f[kQ];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (node_canonical<PREC, RIA>(t, kp, c, pdf, layout, n, N, f)) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      r += f[i];
      if (cx(i)) jx += cx(i) > 0 ? f[i] : -f[i];
      if (cy(i)) jy += cy(i) > 0 ? f[i] : -f[i];
      if (cz(i)) jz += cz(i) > 0 ? f[i] : -f[i];
    }
    const double kd = s ? 1.0 / (1.0 + 0.5 * double(s[n])) : 1.0;
    const double ux = (jx / r + 0.5 * kp.g[0]) * kd;
    const double uy = (jy / r + 0.5 * kp.g[1]) * kd;
    const double uz = (jz / r + 0.5 * kp.g[2]) * kd;
    if (rho) rho[n] = r;
    if (u) {
      u[n] = ux;
      u[size_t(N) + n] = uy;
      u[2 * size_t(N) + n] = uz;
    }
    acc[0] = r;
    acc[1] = r * ux;
    acc[2] = r * uy;
    acc[3] = r * uz;
  }
  if (!partials) return;
  __syncthreads();
  block_sum4(acc, s_red);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) partials[size_t(blockIdx.x) * 4 + k] = acc[k];
}

// Sum nparts x 4 partials into out[4] with one CTA in a fixed order.
template <int PREC>
__global__ void __launch_bounds__(512) k_finish4(const double* __restrict__ partials, int64_t nparts,
                                                 double* __restrict__ out) {
  __shared__ double s_red[16][4];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t p = threadIdx.x; p < nparts; p += blockDim.x)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += partials[p * 4 + k];
  block_sum4(acc, s_red);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = acc[k];
}

}  // namespace dev

// ---- launchers, one set per storage precision ----------------------------------------------

inline int cuda_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return LBM_OK;
}

inline unsigned grid_of(int64_t N) { return unsigned((N + dev::kBlock - 1) / dev::kBlock); }

inline bool has_force(const KParams& kp) { return kp.g[0] != 0.0 || kp.g[1] != 0.0 || kp.g[2] != 0.0; }

// The l+ = 1 collision (see collide) is instantiated for the FP64-storage
// paths only, which are bound by their FP64 arithmetic; the FP32 / FP16 steps
// are bound by memory and take the general form.
template <int PREC> constexpr bool kLp1Path = PREC == LBM_F64 || PREC == LBM_F64_DF;
template <int PREC> inline bool use_lp1(const KParams& kp) { return kLp1Path<PREC> && kp.lp == 1.0; }

// Launch KERNEL<PREC, ARGS..., LP1> with LP1 = lp1 where that instantiation
// exists, on grid g of blk-thread CTAs.
#define LBM_LAUNCH_LP1(KERNEL, TARGS, LAUNCH_ARGS)                             \
  do {                                                                         \
    if constexpr (kLp1Path<PREC>) {                                            \
      if (lp1) {                                                               \
        dev::KERNEL<PREC, TARGS, true><<<g, blk, 0, st>>> LAUNCH_ARGS;         \
        break;                                                                 \
      }                                                                        \
    }                                                                          \
    dev::KERNEL<PREC, TARGS, false><<<g, blk, 0, st>>> LAUNCH_ARGS;            \
  } while (0)
#define LBM_TARGS3(A_, B_, C_) A_, B_, C_
#define LBM_TARGS4(A_, B_, C_, D_) A_, B_, C_, D_
#define LBM_TARGS2(A_, B_) A_, B_

template <int PREC>
int launch_osnt_t(const lbm_lattice* L, const KParams& kp, const void* src, void* dst, const float* s, int ria,
                  void* stream) {
  using T = typename dev::St<PREC>::T;
  auto st = static_cast<cudaStream_t>(stream);
  const unsigned blk = ria ? dev::OsntBlock<PREC, true>::value : dev::OsntBlock<PREC, false>::value;
  const unsigned g = unsigned((L->N + blk - 1) / blk);
  const T* a = static_cast<const T*>(src);
  T* b = static_cast<T*>(dst);
  const int N = int(L->N);
  const bool f = has_force(kp);
  const auto c = dev::make_coll_step<PREC>(kp);
  const bool lp1 = use_lp1<PREC>(kp);
#define LBM_OSNT(R_, F_, D_) LBM_LAUNCH_LP1(k_osnt, LBM_TARGS3(R_, F_, D_), (L->dev, kp, c, a, b, s, N))
  if (s) {
    if (ria) LBM_OSNT(true, true, true); else LBM_OSNT(false, true, true);
  } else if (f) {
    if (ria) LBM_OSNT(true, true, false); else LBM_OSNT(false, true, false);
  } else {
    if (ria) LBM_OSNT(true, false, false); else LBM_OSNT(false, false, false);
  }
#undef LBM_OSNT
  return cuda_check("OS-NT step launch");
}

#ifndef LBM_ODD_X2
#define LBM_ODD_X2 1
#endif
constexpr bool kOddX2 = LBM_ODD_X2 != 0;

template <int PREC>
int launch_aa_t(const lbm_lattice* L, const KParams& kp, void* pdf, int parity, const float* s, int ria,
                void* stream) {
  using T = typename dev::St<PREC>::T;
  auto st = static_cast<cudaStream_t>(stream);
  const unsigned blk = dev::kBlock;
  const unsigned g = grid_of(L->N);
  T* A = static_cast<T*>(pdf);
  const int N = int(L->N);
  const bool f = has_force(kp);
  const bool lp1 = use_lp1<PREC>(kp);
  const auto c = dev::make_coll_step<PREC>(kp);
  if constexpr (PREC == LBM_F16S) {
    if (parity == 0) {
    const unsigned g2 = unsigned((L->N + 2 * dev::kBlock - 1) / (2 * dev::kBlock));
    __half* H = reinterpret_cast<__half*>(pdf);
    const auto cf = dev::make_coll_step<LBM_F16S>(kp);
    if (s) dev::k_aa_even_h2<true, true><<<g2, dev::kBlock, 0, st>>>(L->dev, kp, cf, H, s, N);
    else if (f) dev::k_aa_even_h2<true, false><<<g2, dev::kBlock, 0, st>>>(L->dev, kp, cf, H, s, N);
    else dev::k_aa_even_h2<false, false><<<g2, dev::kBlock, 0, st>>>(L->dev, kp, cf, H, s, N);
    return cuda_check("AA even step launch");
    }
  }
  if (parity == 0) {
    if (s) LBM_LAUNCH_LP1(k_aa_even, LBM_TARGS2(true, true), (L->dev, kp, c, A, s, N));
    else if (f) LBM_LAUNCH_LP1(k_aa_even, LBM_TARGS2(true, false), (L->dev, kp, c, A, s, N));
    else LBM_LAUNCH_LP1(k_aa_even, LBM_TARGS2(false, false), (L->dev, kp, c, A, s, N));
    return cuda_check("AA even step launch");
  }
  if constexpr (PREC == LBM_F32) {
    if (ria && L->dev.run_slot && kOddX2) {
      const unsigned g2 = unsigned((L->N + 2 * dev::kBlock - 1) / (2 * dev::kBlock));
      if (s) dev::k_aa_odd_x2<PREC, true, true><<<g2, dev::kBlock, 0, st>>>(L->dev, kp, c, A, s, N);
      else if (f) dev::k_aa_odd_x2<PREC, true, false><<<g2, dev::kBlock, 0, st>>>(L->dev, kp, c, A, s, N);
      else dev::k_aa_odd_x2<PREC, false, false><<<g2, dev::kBlock, 0, st>>>(L->dev, kp, c, A, s, N);
      return cuda_check("AA odd step launch");
    }
  }
#define LBM_AAODD(R_, F_, D_) LBM_LAUNCH_LP1(k_aa_odd, LBM_TARGS3(R_, F_, D_), (L->dev, kp, c, A, s, N))
  if (s) {
    if (ria) LBM_AAODD(true, true, true); else LBM_AAODD(false, true, true);
  } else if (f) {
    if (ria) LBM_AAODD(true, true, false); else LBM_AAODD(false, true, false);
  } else {
    if (ria) LBM_AAODD(true, false, false); else LBM_AAODD(false, false, false);
  }
#undef LBM_AAODD
  return cuda_check("AA odd step launch");
}

template <int PREC>
int launch_et_t(const lbm_lattice* L, const KParams& kp, void* pdf, int parity, const float* s, int ria,
                void* stream) {
  using T = typename dev::St<PREC>::T;
  auto st = static_cast<cudaStream_t>(stream);
  const unsigned blk = dev::kBlock;
  const unsigned g = grid_of(L->N);
  T* A = static_cast<T*>(pdf);
  const int N = int(L->N);
  const bool f = has_force(kp);
  const auto c = dev::make_coll_step<PREC>(kp);
  const bool lp1 = use_lp1<PREC>(kp);
#define LBM_ET(R_, O_, F_, D_) LBM_LAUNCH_LP1(k_et, LBM_TARGS4(R_, O_, F_, D_), (L->dev, kp, c, A, s, N))
#define LBM_ET_R(O_, F_, D_) \
  do {                       \
    if (ria)                 \
      LBM_ET(true, O_, F_, D_); \
    else                     \
      LBM_ET(false, O_, F_, D_); \
  } while (0)
  if (s) {
    if (parity) LBM_ET_R(true, true, true); else LBM_ET_R(false, true, true);
  } else if (f) {
    if (parity) LBM_ET_R(true, true, false); else LBM_ET_R(false, true, false);
  } else {
    if (parity) LBM_ET_R(true, false, false); else LBM_ET_R(false, false, false);
  }
#undef LBM_ET_R
#undef LBM_ET
  return cuda_check("Esoteric Twist step launch");
}

template <int PREC>
int launch_init_eq_t(const lbm_lattice* L, const KParams& kp, void* pdf, int layout, double rho0, const double u0[3],
                     void* stream) {
  using T = typename dev::St<PREC>::T;
  if (L->N == 0) return LBM_OK;
  dev::Feq19 feq;
  const double uu = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
  for (int i = 0; i < kQ; ++i) {
    const double cu = kCX[i] * u0[0] + kCY[i] * u0[1] + kCZ[i] * u0[2];
    feq.v[i] = dev::wgt(i) * rho0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
  }
  auto st = static_cast<cudaStream_t>(stream);
  const bool ria = !(L->uploaded & LBM_TABLES_ADJ);
  if (ria)
    dev::k_init_eq<PREC, true><<<grid_of(L->N), dev::kBlock, 0, st>>>(L->dev, kp, feq, static_cast<T*>(pdf), layout,
                                                                     int(L->N));
  else
    dev::k_init_eq<PREC, false><<<grid_of(L->N), dev::kBlock, 0, st>>>(L->dev, kp, feq, static_cast<T*>(pdf), layout,
                                                                      int(L->N));
  return cuda_check("init launch");
}

template <int PREC>
int launch_load_canonical_t(const lbm_lattice* L, const KParams& kp, const double* F, void* pdf, int layout,
                            void* stream) {
  using T = typename dev::St<PREC>::T;
  if (L->N == 0) return LBM_OK;
  auto st = static_cast<cudaStream_t>(stream);
  const bool ria = !(L->uploaded & LBM_TABLES_ADJ);
  if (ria)
    dev::k_load_canonical<PREC, true><<<grid_of(L->N), dev::kBlock, 0, st>>>(L->dev, kp, F, static_cast<T*>(pdf),
                                                                            layout, int(L->N));
  else
    dev::k_load_canonical<PREC, false><<<grid_of(L->N), dev::kBlock, 0, st>>>(L->dev, kp, F, static_cast<T*>(pdf),
                                                                             layout, int(L->N));
  return cuda_check("load launch");
}

template <int PREC>
int launch_canonical_t(const lbm_lattice* L, const KParams& kp, const void* pdf, int layout, double* F,
                       void* stream) {
  using T = typename dev::St<PREC>::T;
  if (L->N == 0) return LBM_OK;
  auto st = static_cast<cudaStream_t>(stream);
  const bool ria = !(L->uploaded & LBM_TABLES_ADJ);
  const auto c = dev::make_coll<typename dev::St<PREC>::R>(kp);
  if (ria)
    dev::k_canonical<PREC, true><<<grid_of(L->N), dev::kBlock, 0, st>>>(L->dev, kp, c, static_cast<const T*>(pdf),
                                                                       layout, F, int(L->N));
  else
    dev::k_canonical<PREC, false><<<grid_of(L->N), dev::kBlock, 0, st>>>(L->dev, kp, c, static_cast<const T*>(pdf),
                                                                        layout, F, int(L->N));
  return cuda_check("canonical launch");
}

template <int PREC>
int launch_macroscopic_t(const lbm_lattice* L, const KParams& kp, const void* pdf, int layout, const float* s,
                         double* rho, double* u, double* sums, double* partials, int64_t nparts, void* stream) {
  using T = typename dev::St<PREC>::T;
  auto st = static_cast<cudaStream_t>(stream);
  double* part = sums ? partials : nullptr;
  if (L->N > 0) {
    const bool ria = !(L->uploaded & LBM_TABLES_ADJ);
    const auto c = dev::make_coll<typename dev::St<PREC>::R>(kp);
    if (ria)
      dev::k_macro<PREC, true><<<grid_of(L->N), dev::kBlock, 0, st>>>(L->dev, kp, c, static_cast<const T*>(pdf),
                                                                     layout, s, rho, u, part, int(L->N));
    else
      dev::k_macro<PREC, false><<<grid_of(L->N), dev::kBlock, 0, st>>>(L->dev, kp, c, static_cast<const T*>(pdf),
                                                                      layout, s, rho, u, part, int(L->N));
    if (int rc = cuda_check("macroscopic launch")) return rc;
  }
  if (sums) {
    dev::k_finish4<PREC><<<1, 512, 0, st>>>(partials, L->N > 0 ? nparts : 0, sums);
    return cuda_check("reduction launch");
  }
  return LBM_OK;
}

#define LBM_INSTANTIATE_STEP_LAUNCHERS(P)                                                                          \
  template int launch_osnt_t<P>(const lbm_lattice*, const KParams&, const void*, void*, const float*, int, void*); \
  template int launch_aa_t<P>(const lbm_lattice*, const KParams&, void*, int, const float*, int, void*);           \
  template int launch_et_t<P>(const lbm_lattice*, const KParams&, void*, int, const float*, int, void*);

#define LBM_INSTANTIATE_LAUNCHERS(P)                                                                               \
  template int launch_osnt_t<P>(const lbm_lattice*, const KParams&, const void*, void*, const float*, int, void*); \
  template int launch_aa_t<P>(const lbm_lattice*, const KParams&, void*, int, const float*, int, void*);           \
  template int launch_et_t<P>(const lbm_lattice*, const KParams&, void*, int, const float*, int, void*);                \
  template int launch_init_eq_t<P>(const lbm_lattice*, const KParams&, void*, int, double, const double*, void*);  \
  template int launch_load_canonical_t<P>(const lbm_lattice*, const KParams&, const double*, void*, int, void*);   \
  template int launch_canonical_t<P>(const lbm_lattice*, const KParams&, const void*, int, double*, void*);        \
  template int launch_macroscopic_t<P>(const lbm_lattice*, const KParams&, const void*, int, const float*,          \
                                       double*, double*, double*, double*, int64_t, void*);

}  // namespace lbm
