// Fixed-point conversions of the integer FP64 operator (k_operator_fx.cu),
// host-compilable so that a CPU test can check them bit for bit against exact
// rational rounding.
//
// fx_of:      a double as an integer multiple of a tile's step, |X| < 2^53
// fx_limbs:   an integer (|v| < 2^54) as lo + hi 2^25, lo in [0, 2^25)
// fx_to_f64:  (c0 + c1 2^25 + c2 2^50 + c3 2^75) 2^-K as the nearest double
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define SEM_FX_FN __host__ __device__ __forceinline__
#else
#define SEM_FX_FN inline
#endif

namespace sem {

SEM_FX_FN uint64_t fx_bits(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  std::memcpy(&b, &v, sizeof b);
  return b;
#endif
}

SEM_FX_FN double fx_double(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  std::memcpy(&v, &b, sizeof v);
  return v;
#endif
}

SEM_FX_FN int fx_clz64(uint64_t v) {  // v != 0
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

// x = X 2^(emax - 1075) with emax >= the exponent field of x: X is the
// mantissa (hidden bit included) divided by 2^(emax - exponent), rounded to
// nearest, ties away from zero; 0 for zeros and subnormals.  |X| < 2^53.
SEM_FX_FN int64_t fx_of(double v, int emax) {
  const uint64_t b = fx_bits(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return 0;
  const int64_t m = (int64_t)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  const int sh = emax - ex;  // >= 0
  int64_t X;
  if (sh == 0) X = m;
  else if (sh <= 53) X = (m + ((int64_t)1 << (sh - 1))) >> sh;
  else X = 0;
  return (b >> 63) ? -X : X;
}

SEM_FX_FN void fx_limbs(int64_t v, int& lo, int& hi) {
  const int64_t h = v >> 25;  // floor
  lo = (int)(v - h * ((int64_t)1 << 25));
  hi = (int)h;
}

// top: the 64 bits of a magnitude from its leading one down (bit 63 set);
// sticky: anything nonzero below them; the leading one has weight 2^e.
// Rounded to nearest, ties to even.
SEM_FX_FN double fx_round(uint64_t top, bool sticky, int e, bool neg) {
  uint64_t m = top >> 11;  // 53 bits
  const bool rb = ((top >> 10) & 1ULL) != 0;
  const bool st = sticky || (top & 0x3FFULL) != 0;
  if (rb && (st || (m & 1ULL))) ++m;
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  const int be = e + 1023;
  if (be <= 0 || be >= 2047) {  // outside the normal range: scale in FP64 (subnormals round twice)
    const double d = ldexp((double)m, e - 52);
    return neg ? -d : d;
  }
  return fx_double(((uint64_t)neg << 63) | ((uint64_t)be << 52) | (m & ((1ULL << 52) - 1)));
}

// (c0 + c1 2^25 + c2 2^50 + c3 2^75) 2^-K for |c| < 2^62, rounded to the
// nearest double (ties to even; normal results exactly so)
SEM_FX_FN double fx_to_f64(int64_t c0, int64_t c1, int64_t c2, int64_t c3, int K) {
  const int64_t B = (int64_t)1 << 25;
  int64_t q = c0 >> 25;  // carries: c0, c1, c2 into [0, 2^25)
  c0 -= q * B;
  c1 += q;
  q = c1 >> 25;
  c1 -= q * B;
  c2 += q;
  q = c2 >> 25;
  c2 -= q * B;
  c3 += q;
  // value = c3 2^75 + R, R = rh 2^64 + rl in [0, 2^75)
  uint64_t rl = ((uint64_t)c2 << 50) | ((uint64_t)c1 << 25) | (uint64_t)c0;
  uint64_t rh = (uint64_t)c2 >> 14;
  const bool neg = c3 < 0;
  uint64_t A = (uint64_t)c3;
  if (neg) {  // magnitude (-c3) 2^75 - R = (-c3 - 1) 2^75 + (2^75 - R)
    A = 0ULL - (uint64_t)c3;
    if (rl | rh) {
      A -= 1;
      rh = (1ULL << 11) - rh - (rl != 0 ? 1ULL : 0ULL);
      rl = 0ULL - rl;
    }
  }
  // magnitude = A 2^75 + rh 2^64 + rl, A < 2^63, rh < 2^11
  if (A != 0) {
    const int lz = fx_clz64(A);
    const int s2 = 75 - lz;  // bits of R below the top 64: 12 .. 75
    uint64_t low;            // R >> s2
    bool sticky;
    if (s2 >= 64) {
      low = s2 >= 75 ? 0ULL : (rh >> (s2 - 64));
      sticky = rl != 0 || (s2 >= 75 ? rh != 0 : (rh & ((1ULL << (s2 - 64)) - 1)) != 0);
    } else {
      low = (rh << (64 - s2)) | (rl >> s2);
      sticky = (rl << (64 - s2)) != 0;
    }
    return fx_round((lz == 0 ? A : (A << lz)) | low, sticky, 138 - lz - K, neg);
  }
  if (rh != 0) {
    const int lz = fx_clz64(rh);  // >= 53
    return fx_round((rh << lz) | (rl >> (64 - lz)), (rl << lz) != 0, 127 - lz - K, neg);
  }
  if (rl == 0) return 0.0;
  const int lz = fx_clz64(rl);
  return fx_round(rl << lz, false, 63 - lz - K, neg);
}

}  // namespace sem
