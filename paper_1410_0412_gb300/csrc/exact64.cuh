// Integer-pipe arithmetic for the FP64 collision.
//
// GB300 executes FP64 arithmetic on two lanes per SM per clock, against 64
// integer and 128 FP32 lanes, so the native FP64 step is bound by its FP64
// instruction count while the other pipes idle.  Two pieces of the collision
// are exact in integer arithmetic and move there:
//
//  * the moments that the TRT collision (Sect. 2) starts from, the density
//    and momentum sums and the pair sums and differences: the 19 PDFs of a
//    node are converted to 64-bit fixed point with a per-node scale (the largest
//    exponent among them, with 5 bits of headroom), summed exactly, and each
//    sum is rounded once to the nearest double.  A PDF at most 5 binades below
//    the node's largest converts exactly; smaller ones lose bits below 2^-57
//    of the largest.  A moment's error is at most 19 * 2^-57 * max|f_i| plus
//    half an ulp of the result, below the error bound (n - 1) * 2^-53 * sum|f_i|
//    of the IEEE double sum of n terms that it replaces;
//  * halving: an exponent decrement, identical to 0.5 * x for every x whose
//    half is a normal number, Inf or NaN.
//
// All functions are __host__ __device__ so that a host test can check the
// moments bit for bit against exact rational arithmetic.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace lbm {
namespace dev {

__host__ __device__ __forceinline__ uint64_t dbits(double x) {
#ifdef __CUDA_ARCH__
  return static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

__host__ __device__ __forceinline__ double dfrom(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(static_cast<long long>(b));
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

__host__ __device__ __forceinline__ int clz64(uint64_t a) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(a));
#else
  return a ? __builtin_clzll(a) : 64;
#endif
}

constexpr uint64_t kSignBit = 0x8000000000000000ull;

// x / 2 without an FP64 instruction.  Exponent fields 2..2046 lose one; Inf and
// NaN pass through; zero, subnormals and the smallest binade shift their
// magnitude right (truncating the last subnormal bit).
__host__ __device__ __forceinline__ double halve_exact(double x) {
  const uint64_t b = dbits(x);
  const unsigned ef = static_cast<unsigned>(b >> 52) & 0x7ffu;
  uint64_t r;
  if (ef - 2u < 2045u)
    r = b - (uint64_t(1) << 52);
  else if (ef == 2047u)
    r = b;
  else
    r = (b & kSignBit) | ((b & ~kSignBit) >> 1);
  return dfrom(r);
}

// Smallest node scale: PDFs below 2^-959 (biased exponent 64) flush to zero.
constexpr int kFxMinExp = 64;
// Node scales at or above this biased exponent (|f| >= 2^1017) mark the node as
// diverged: the moments come out NaN, as an IEEE sum of such PDFs would.
constexpr int kFxMaxExp = 2040;

// Fixed-point image of the double with bits b at the node scale emax (the
// largest biased exponent among the node's PDFs, >= kFxMinExp):
// x * 2^(1080 - emax), truncated toward zero; |result| < 2^58.
__host__ __device__ __forceinline__ int64_t fx_of(uint64_t b, int emax) {
  const int e = static_cast<int>(b >> 52) & 0x7ff;
  const uint64_t m = ((b & 0x000fffffffffffffull) | 0x0010000000000000ull) << 10;  // < 2^63
  int sh = emax - e + 5;  // >= 5; zero and subnormal inputs (e = 0) shift out entirely
  sh = sh < 63 ? sh : 63;
  const uint64_t v = m >> sh;
  return (b & kSignBit) ? -static_cast<int64_t>(v) : static_cast<int64_t>(v);
}

// The double nearest to v * 2^(emax - 1080) (round to nearest, ties to even),
// for |v| < 2^63 and kFxMinExp <= emax < kFxMaxExp.
__host__ __device__ __forceinline__ double fx_to_double(int64_t v, int emax) {
  if (v == 0) return 0.0;
  const uint64_t s = static_cast<uint64_t>(v) & kSignBit;
  uint64_t a = v < 0 ? uint64_t(0) - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
  const int lz = clz64(a);  // >= 1
  a <<= lz;                 // leading one at bit 63
  uint64_t m = a >> 11;     // 53 significant bits
  const unsigned rest = static_cast<unsigned>(a) & 0x7ffu;
  m += (rest > 0x400u || (rest == 0x400u && (m & 1u))) ? 1u : 0u;
  // value = m * 2^(emax - lz - 1069); the biased exponent is emax + 6 - lz, and
  // adding m (hidden bit included, possibly 2^53 after rounding) to
  // (exponent - 1) << 52 assembles the bits with the carry in place.
  return dfrom(((static_cast<uint64_t>(emax + 5 - lz) << 52) + m) | s);
}

// 32-bit funnel shifts (the PTX shf instructions) with a portable host image.
__host__ __device__ __forceinline__ uint32_t shf_l(uint32_t lo, uint32_t hi, unsigned n) {  // n in [0, 31]
#ifdef __CUDA_ARCH__
  return __funnelshift_l(lo, hi, n);
#else
  return n ? (hi << n) | (lo >> (32 - n)) : hi;
#endif
}
__host__ __device__ __forceinline__ uint32_t shf_r(uint32_t lo, uint32_t hi, unsigned n) {  // n in [0, 31]
#ifdef __CUDA_ARCH__
  return __funnelshift_r(lo, hi, n);
#else
  return n ? (lo >> n) | (hi << (32 - n)) : lo;
#endif
}
__host__ __device__ __forceinline__ int clz32(uint32_t a) {
#ifdef __CUDA_ARCH__
  return __clz(static_cast<int>(a));
#else
  return a ? __builtin_clz(a) : 32;
#endif
}

// fx_of for the common case, in 32-bit halves: a positive double (sign bit
// clear) at most 5 binades below the node's largest, so that fx_of's value
// m * 2^(10 - sh) is the significand m shifted left by k = 5 - (emax - e) in
// [0, 5].  Same value as fx_of (exact here).
__host__ __device__ __forceinline__ int64_t fx_of_pos_near(uint64_t b, unsigned k) {
  const uint32_t hi = static_cast<uint32_t>(b >> 32), lo = static_cast<uint32_t>(b);
  const uint32_t mh = (hi & 0x000fffffu) | 0x00100000u;  // significand bits 52..32, hidden bit included
  return static_cast<int64_t>((static_cast<uint64_t>(shf_l(lo, mh, k)) << 32) | (lo << k));
}

// fx_to_double for the common case, in 32-bit halves: 2^32 <= v < 2^63 (the
// high word is a positive int32).  Same bits as fx_to_double.
__host__ __device__ __forceinline__ double fx_to_double_pos(int64_t v, int emax) {
  const uint32_t hi = static_cast<uint32_t>(static_cast<uint64_t>(v) >> 32), lo = static_cast<uint32_t>(v);
  const int lz = clz32(hi);                                // 1..31
  const uint32_t ah = shf_l(lo, hi, lz), al = lo << lz;    // leading one at bit 63
  const uint32_t mh = ah >> 11, ml = shf_r(al, ah, 11);    // 53 significant bits
  // round to nearest, ties to even: the 11 bits below plus 0x3ff plus the
  // last kept bit reach 2^11 exactly when rounding up
  const uint32_t up = ((al & 0x7ffu) + 0x3ffu + (ml & 1u)) >> 11;
  const uint64_t m = ((static_cast<uint64_t>(mh) << 32) | ml) + up;  // may carry to 2^53: exponent + 1
  return dfrom((static_cast<uint64_t>(emax + 5 - lz) << 52) + m);
}

// True when fx_to_double_pos applies to v.
__host__ __device__ __forceinline__ bool fx_pos_wide(int64_t v) { return (v >> 32) >= 1; }

// fx_to_double through the hardware's int64 -> double conversion (round to
// nearest, ties to even: the same rounding, so the same bits), then an exact
// scaling by 2^(emax - 1080) as an exponent-field add.  The conversion runs
// on the FP64 pipe, the rest on the integer pipe; the kernels use it for part
// of the outputs to balance the two.  For kFxMinExp - 4 <= emax < kFxMaxExp
// every non-zero result is a normal number.
__host__ __device__ __forceinline__ double fx_to_double_cvt(int64_t v, int emax) {
#ifdef __CUDA_ARCH__
  const double x = __ll2double_rn(static_cast<long long>(v));
#else
  const double x = static_cast<double>(v);
#endif
  const uint64_t scaled = dbits(x) + (static_cast<uint64_t>(static_cast<int64_t>(emax - 1080)) << 52);
  return v == 0 ? 0.0 : dfrom(scaled);
}

// Node scale of the 19 PDFs: the largest biased exponent, at least kFxMinExp.
template <int Q>
__host__ __device__ __forceinline__ int fx_scale(const uint64_t (&b)[Q]) {
  int emax = kFxMinExp;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int e = static_cast<int>(b[i] >> 52) & 0x7ff;
    emax = e > emax ? e : emax;
  }
  return emax;
}

// The exact fixed-point moments of one D3Q19 node from its 19 PDFs d (pair
// k = 1..9 holds the opposite directions 2k-1 and 2k; the first directions of
// the pairs are (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1) (1,0,-1)
// (0,1,1) (0,1,-1)) at the node scale emax (returned): pair sums Sk[k] (only
// when NEED_SA) and differences D[k], the density deviation S = sum d_i and
// the momentum J = sum c_i d_i, all as integers times 2^(emax - 1080).
// FAST: the caller has checked fx_pos_near (positive PDFs within 5 binades
// of the largest) and passes the node scale it found as emax_fast; the
// conversions take the shorter fx_of_pos_near, and the integers are the same.
template <bool NEED_SA, bool FAST = false>
__host__ __device__ __forceinline__ int fx_moments(const double (&d)[19], int64_t (&Sk)[10], int64_t (&D)[10],
                                                   int64_t& S, int64_t& Jx, int64_t& Jy, int64_t& Jz,
                                                   int emax_fast = 0) {
  uint64_t b[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) b[i] = dbits(d[i]);
  int64_t f[19];
  int emax;
  if (FAST) {
    // positive: the exponent is the high word shifted, no sign to clear
    emax = emax_fast;
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = fx_of_pos_near(b[i], static_cast<unsigned>(static_cast<int>(b[i] >> 52) + 5 - emax));
  } else {
    emax = fx_scale(b);
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = fx_of(b[i], emax);
  }
  S = f[0];
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int64_t s = f[2 * k - 1] + f[2 * k];
    D[k] = f[2 * k - 1] - f[2 * k];
    S += s;
    if (NEED_SA) Sk[k] = s;
  }
  Jx = D[1] + D[4] + D[5] + D[6] + D[7];
  Jy = D[2] + D[4] - D[5] + D[8] + D[9];
  Jz = D[3] + D[6] - D[7] + D[8] - D[9];
  return emax;
}

// True when the fast conversions of fx_moments apply: every PDF positive and
// finite-scaled (node scale below kFxMaxExp) and at most 5 binades below the
// largest (so fx_of_pos_near's shift stays in [0, 5]; PDFs near w_i rho span
// 4).  emax: the node scale (the largest exponent field; meaningful when true).
__host__ __device__ __forceinline__ bool fx_pos_near(const double (&d)[19], int& emax) {
  uint32_t sgn = 0;
  int emin = 2047;
  emax = 0;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const uint32_t hi = static_cast<uint32_t>(dbits(d[i]) >> 32);
    sgn |= hi;
    const int e = static_cast<int>(hi >> 20);
    emax = e > emax ? e : emax;
    emin = e < emin ? e : emin;
  }
  return !(sgn & 0x80000000u) && emin >= kFxMinExp && emax < kFxMaxExp && emax - emin <= 5;
}

// The moments as doubles: pair sums sa_k (only when NEED_SA) and differences
// da_k, the density deviation drho = sum d_i and the momentum j = sum c_i d_i,
// each the double nearest to the exact fixed-point sum.  A node whose scale
// reaches kFxMaxExp (an Inf, a NaN or |d_i| >= 2^1017) gets drho = NaN.
template <bool NEED_SA>
__host__ __device__ __forceinline__ void exact_moments(const double (&d)[19], double (&sa)[10], double (&da)[10],
                                                       double& drho, double& jx, double& jy, double& jz) {
  int64_t Sk[10], D[10], S, Jx, Jy, Jz;
  const int emax = fx_moments<NEED_SA>(d, Sk, D, S, Jx, Jy, Jz);
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    if (NEED_SA) sa[k] = fx_to_double(Sk[k], emax);
    da[k] = fx_to_double(D[k], emax);
  }
  drho = emax < kFxMaxExp ? fx_to_double(S, emax) : dfrom(0x7ff8000000000000ull);
  jx = fx_to_double(Jx, emax);
  jy = fx_to_double(Jy, emax);
  jz = fx_to_double(Jz, emax);
}

// floor(a * b / 2^64) for signed 64-bit a, b: the product of a Q64 fraction
// (|a| < 2^63, the value a / 2^64) with a fixed-point value, at the latter's scale.
__host__ __device__ __forceinline__ int64_t mulhi_q64(int64_t a, int64_t b) {
#ifdef __CUDA_ARCH__
  return __mul64hi(a, b);
#else
  return static_cast<int64_t>((static_cast<__int128>(a) * b) >> 64);
#endif
}

// Biased exponent field of a double.
__host__ __device__ __forceinline__ int dexp(double x) { return static_cast<int>(dbits(x) >> 52) & 0x7ff; }

// The pair update of the FP64 collision in fixed point (scale 2^(emax - 1080),
// the node's moment scale).  Given the class values of the TRT collision with
// Guo forcing -- the velocity u, the even constant K0 and the vectors T and O
// of the axis class (the diagonal class uses them halved) -- and the exact
// pair sums Sk and differences Dk, the post-collision pair is
//   e = K0 + (c.u)(c.T) [+ qp Sk],  o = qm Dk + c.O,  p_a = e + o,  p_b = e - o,
// with qm = (1 - l-)/2 and qp = (1 - l+)/2 as Q64 fractions.  The pair stage
// works at a scale kx bits finer than the moments, 2^(es - 1080) with
// es = emax - kx (kx = 4 when qp = 0, else 2): Dk and Sk enter shifted left by
// kx, exactly.  Every sum is exact; the products (c.u)(c.T), qm Dk and qp Sk
// are truncated to the scale (floor), and so are u, K0, T and O when they
// enter.  The error of p before its one rounding to double is below 8 units
// of 2^(es - 1080), i.e. below 2^-(54 + kx) of B = 2^(emax - 1023), the
// binade of the node's largest PDF (for PDFs near w_i rho, below a quarter of
// an ulp of the smallest, the diagonal ones, when kx = 4).
//
// Valid when |u_a| < 1/4 (biased exponent <= 1020), |K0| < B/2 (exponent
// <= emax - 2) and |T_a|, |O_a| < B/4 (exponent <= emax - 3); with every
// |d_i| < 2B this keeps |c.u| < 1/2 and every intermediate below 2^63 at
// either kx.  fx_class_ok checks it.
struct FxClass {
  int64_t ux, uy, uz;  // Q64
  int64_t K0, Tx, Ty, Tz, Ox, Oy, Oz;
};

__host__ __device__ __forceinline__ bool fx_class_ok(int emax, double ux, double uy, double uz, double K0, double Tx,
                                                     double Ty, double Tz, double Ox, double Oy, double Oz) {
  int eu = dexp(ux);
  eu = dexp(uy) > eu ? dexp(uy) : eu;
  eu = dexp(uz) > eu ? dexp(uz) : eu;
  int eto = dexp(Tx);
  const double v[5] = {Ty, Tz, Ox, Oy, Oz};
#pragma unroll
  for (int i = 0; i < 5; ++i) eto = dexp(v[i]) > eto ? dexp(v[i]) : eto;
  return emax < kFxMaxExp && eu <= 1020 && dexp(K0) <= emax - 2 && eto <= emax - 3;
}

// The class values at the pair scale es (see above).
__host__ __device__ __forceinline__ FxClass fx_class(int es, double ux, double uy, double uz, double K0, double Tx,
                                                     double Ty, double Tz, double Ox, double Oy, double Oz) {
  FxClass q;
  q.ux = fx_of(dbits(ux), 1016);  // u * 2^64
  q.uy = fx_of(dbits(uy), 1016);
  q.uz = fx_of(dbits(uz), 1016);
  q.K0 = fx_of(dbits(K0), es);
  q.Tx = fx_of(dbits(Tx), es);
  q.Ty = fx_of(dbits(Ty), es);
  q.Tz = fx_of(dbits(Tz), es);
  q.Ox = fx_of(dbits(Ox), es);
  q.Oy = fx_of(dbits(Oy), es);
  q.Oz = fx_of(dbits(Oz), es);
  return q;
}

// c . v for a direction with components X, Y, Z in {-1, 0, 1} (exact integer sums).
template <int X, int Y, int Z>
__host__ __device__ __forceinline__ int64_t fx_cdot(int64_t vx, int64_t vy, int64_t vz) {
  int64_t acc = 0;
  if (X) acc = X > 0 ? vx : -vx;
  if (Y) acc = X ? (Y > 0 ? acc + vy : acc - vy) : (Y > 0 ? vy : -vy);
  if (Z) acc = (X || Y) ? (Z > 0 ? acc + vz : acc - vz) : (Z > 0 ? vz : -vz);
  return acc;
}

// Pair with first direction (X, Y, Z): DIAG for the face diagonals (weight
// 1/36: K0, T and O halved), LP1 when qp = 0.  The two values are converted
// with fx_to_double_pos when both qualify in every thread of the warp (on the
// host: in this node), otherwise with fx_to_double; the bits are the same.
// CVT: convert with fx_to_double_cvt (the FP64 pipe's int64 -> double).
template <int X, int Y, int Z, bool DIAG, bool LP1, bool GENERAL = false, bool CVT = false>
__host__ __device__ __forceinline__ void fx_pair(const FxClass& q, int64_t Dk, int64_t Sk, int64_t qm, int64_t qp,
                                                 int es, double& pa, double& pb) {
  const int64_t cu = fx_cdot<X, Y, Z>(q.ux, q.uy, q.uz);
  const int64_t ct = fx_cdot<X, Y, Z>(q.Tx, q.Ty, q.Tz);
  const int64_t co = fx_cdot<X, Y, Z>(q.Ox, q.Oy, q.Oz);
  int64_t e = q.K0 + mulhi_q64(cu, ct);
  int64_t o = mulhi_q64(qm, Dk);
  if (DIAG) {
    e >>= 1;
    o += co >> 1;
  } else {
    o += co;
  }
  if (!LP1) e += mulhi_q64(qp, Sk);
  const int64_t va = e + o, vb = e - o;
  if (CVT && !GENERAL) {
    pa = fx_to_double_cvt(va, es);
    pb = fx_to_double_cvt(vb, es);
    return;
  }
  bool fast = !GENERAL && fx_pos_wide(va) && fx_pos_wide(vb);
#ifdef __CUDA_ARCH__
  fast = __all_sync(__activemask(), fast);
#endif
  if (fast) {
    pa = fx_to_double_pos(va, es);
    pb = fx_to_double_pos(vb, es);
  } else {
    pa = fx_to_double(va, es);
    pb = fx_to_double(vb, es);
  }
}

#ifndef LBM_FX_CVT_PAIRS
#define LBM_FX_CVT_PAIRS 2
#endif
constexpr int kFxCvtPairs = LBM_FX_CVT_PAIRS;

// The nine pairs in the direction order of the lattice (see fx_moments), from
// the moment-scale D and Sk of fx_moments; es = emax - KX.
template <bool LP1, int KX, bool GENERAL = false>
__host__ __device__ __forceinline__ void fx_pairs(const FxClass& q, const int64_t (&D)[10], const int64_t (&Sk)[10],
                                                  int64_t qm, int64_t qp, int es, double (&p)[19]) {
  int64_t Df[10], Sf[10];
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    Df[k] = static_cast<int64_t>(static_cast<uint64_t>(D[k]) << KX);
    Sf[k] = LP1 ? 0 : static_cast<int64_t>(static_cast<uint64_t>(Sk[k]) << KX);
  }
  // the first kFxCvtPairs pairs convert on the FP64 pipe (fx_to_double_cvt)
  fx_pair<1, 0, 0, false, LP1, GENERAL, (kFxCvtPairs > 0)>(q, Df[1], Sf[1], qm, qp, es, p[1], p[2]);
  fx_pair<0, 1, 0, false, LP1, GENERAL, (kFxCvtPairs > 1)>(q, Df[2], Sf[2], qm, qp, es, p[3], p[4]);
  fx_pair<0, 0, 1, false, LP1, GENERAL, (kFxCvtPairs > 2)>(q, Df[3], Sf[3], qm, qp, es, p[5], p[6]);
  fx_pair<1, 1, 0, true, LP1, GENERAL, (kFxCvtPairs > 3)>(q, Df[4], Sf[4], qm, qp, es, p[7], p[8]);
  fx_pair<1, -1, 0, true, LP1, GENERAL, (kFxCvtPairs > 4)>(q, Df[5], Sf[5], qm, qp, es, p[9], p[10]);
  fx_pair<1, 0, 1, true, LP1, GENERAL, (kFxCvtPairs > 5)>(q, Df[6], Sf[6], qm, qp, es, p[11], p[12]);
  fx_pair<1, 0, -1, true, LP1, GENERAL, (kFxCvtPairs > 6)>(q, Df[7], Sf[7], qm, qp, es, p[13], p[14]);
  fx_pair<0, 1, 1, true, LP1, GENERAL, (kFxCvtPairs > 7)>(q, Df[8], Sf[8], qm, qp, es, p[15], p[16]);
  fx_pair<0, 1, -1, true, LP1, GENERAL, (kFxCvtPairs > 8)>(q, Df[9], Sf[9], qm, qp, es, p[17], p[18]);
}

// Q64 image of a rate constant |x| < 1/2: round(x * 2^64).
inline int64_t q64_of(double x) { return static_cast<int64_t>(std::llround(std::ldexp(x, 64))); }

}  // namespace dev
}  // namespace lbm
