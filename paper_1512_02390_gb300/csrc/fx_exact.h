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
// Without branches: a shift of 54 or more leaves 0 (the mantissa is below
// 2^53, the rounding half below 2^(shift - 1)), so the shift is capped at 63.
SEM_FX_FN int64_t fx_of(double v, int emax) {
  const uint64_t b = fx_bits(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  const uint64_t m = ex != 0 ? ((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52)) : 0ULL;
  const int d = emax - ex;  // >= 0
  const int sh = d < 63 ? d : 63;
  const uint64_t X = (m + ((1ULL << sh) >> 1)) >> sh;
  const int64_t sg = -(int64_t)(b >> 63);  // 0 or -1
  return ((int64_t)X ^ sg) - sg;
}

SEM_FX_FN void fx_limbs(int64_t v, int& lo, int& hi) {
  lo = (int)(v & (((int64_t)1 << 25) - 1));  // v mod 2^25 (two's complement)
  hi = (int)(v >> 25);                        // floor(v / 2^25), |v| < 2^54
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
// nearest double (ties to even; normal results exactly so).  The value V can
// need 138 bits, so it is held as V = W 2^11 + s with W = floor(V / 2^11)
// a 128-bit two's complement (|W| < 2^127) and s in [0, 2^11); the branches
// left are the rare zero and out-of-range results.
SEM_FX_FN double fx_to_f64(int64_t c0, int64_t c1, int64_t c2, int64_t c3, int K) {
  // S = c0 + c1 2^25 + c2 2^50, |S| < 2^113, as the words (sh, sl)
  uint64_t sl = (uint64_t)c0, sh = (uint64_t)(c0 >> 63);
  uint64_t t = (uint64_t)c1 << 25;
  sl += t;
  sh += (uint64_t)(c1 >> 39) + (sl < t ? 1ULL : 0ULL);
  t = (uint64_t)c2 << 50;
  sl += t;
  sh += (uint64_t)(c2 >> 14) + (sl < t ? 1ULL : 0ULL);
  // W = floor(S / 2^11) + c3 2^64 (c3 2^75 is a multiple of 2^11), s = S mod 2^11
  const uint64_t s = sl & 0x7FFULL;
  uint64_t wl = (sl >> 11) | (sh << 53);
  uint64_t wh = (uint64_t)((int64_t)sh >> 11) + (uint64_t)c3;
  // |V| = M 2^11 + z: V >= 0: M = W, z = s; V < 0: M = -W - (s != 0) = ~W + (s == 0),
  // z = (2^11 - s) mod 2^11
  const uint64_t ng = (uint64_t)((int64_t)wh >> 63);  // all ones when V < 0
  const uint64_t inc = ng & (s == 0 ? 1ULL : 0ULL);
  wl ^= ng;
  wh ^= ng;
  wl += inc;
  wh += wl < inc ? 1ULL : 0ULL;
  const uint64_t z = ((ng != 0 ? 0x800ULL - s : s) & 0x7FFULL) << 53;
  // |V| 2^53 = wh 2^128 + wl 2^64 + z: its leading nonzero word a, the next b, the rest c
  const bool h0 = wh == 0, h1 = h0 && wl == 0;
  const uint64_t a = h0 ? (h1 ? z : wl) : wh;
  const uint64_t b = h0 ? (h1 ? 0ULL : z) : wl;
  const uint64_t c = h0 ? 0ULL : z;
  if (a == 0) return 0.0;
  const int l = fx_clz64(a);
  const uint64_t top = (a << l) | ((b >> 1) >> (63 - l));
  const bool sticky = (b << l) != 0 || c != 0;
  const int e = (h0 ? (h1 ? 63 : 127) : 191) - l - 53 - K;  // the leading one has weight 2^e
  uint64_t m = top >> 11;                                     // 53 bits
  const uint64_t rb = (top >> 10) & 1ULL;
  const uint64_t st = ((top & 0x3FFULL) != 0 || sticky) ? 1ULL : 0ULL;
  m += rb & (st | (m & 1ULL));
  const int be = e + 1023;  // biased exponent before a carry out of the rounding
  const int bc = be + (int)(m >> 53);
  if (bc <= 0 || bc >= 2047) return fx_round(top, sticky, e, ng != 0);
  // m in [2^52, 2^53]: a carry to 2^53 moves into the exponent field
  return fx_double((ng & (1ULL << 63)) | (((uint64_t)(be - 1) << 52) + m));
}

}  // namespace sem
