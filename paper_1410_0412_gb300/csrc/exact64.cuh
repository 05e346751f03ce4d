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

// The moments of one D3Q19 node from its 19 PDFs d (pair k = 1..9 holds the
// opposite directions 2k-1 and 2k; the first directions of the pairs are
// (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1)):
// pair sums sa_k (only when NEED_SA) and differences da_k, the density
// deviation drho = sum d_i and the momentum j = sum c_i d_i, each the double
// nearest to the exact fixed-point sum.  A node whose scale reaches kFxMaxExp
// (an Inf, a NaN or |d_i| >= 2^1017) gets drho = NaN.
template <bool NEED_SA>
__host__ __device__ __forceinline__ void exact_moments(const double (&d)[19], double (&sa)[10], double (&da)[10],
                                                       double& drho, double& jx, double& jy, double& jz) {
  uint64_t b[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) b[i] = dbits(d[i]);
  const int emax = fx_scale(b);
  int64_t f[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = fx_of(b[i], emax);
  int64_t S = f[0], D[10];
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int64_t Sk = f[2 * k - 1] + f[2 * k];
    D[k] = f[2 * k - 1] - f[2 * k];
    S += Sk;
    if (NEED_SA) sa[k] = fx_to_double(Sk, emax);
    da[k] = fx_to_double(D[k], emax);
  }
  drho = emax < kFxMaxExp ? fx_to_double(S, emax) : dfrom(0x7ff8000000000000ull);
  jx = fx_to_double(D[1] + D[4] + D[5] + D[6] + D[7], emax);
  jy = fx_to_double(D[2] + D[4] - D[5] + D[8] + D[9], emax);
  jz = fx_to_double(D[3] + D[6] - D[7] + D[8] - D[9], emax);
}

}  // namespace dev
}  // namespace lbm
