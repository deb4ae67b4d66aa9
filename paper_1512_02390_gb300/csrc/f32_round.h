// Roundings by integer operations on the bit fields.
//
// IEEE 754 binary64 -> binary32 conversion, round to nearest, ties to even.  On this GPU the conversion
// instruction issues on the narrow FP64 pipe; in the FP64-bound MGCG update
// the integer form runs on the idle integer ALU instead.  Results whose
// binary32 form is normal or overflows (|x| >= 2^-126) are formed here; zero
// keeps its sign; the rest (binary32 subnormals, NaN) take the conversion
// instruction.  Host-compilable so that a CPU test can check it bit for bit.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define SEM_F32R_FN __host__ __device__ __forceinline__
#else
#define SEM_F32R_FN inline
#endif

namespace sem {

SEM_F32R_FN float f32_from_f64_rn(double x) {
  uint64_t b;
#ifdef __CUDA_ARCH__
  b = (uint64_t)__double_as_longlong(x);
#else
  std::memcpy(&b, &x, sizeof b);
#endif
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);  // biased binary64 exponent
  uint32_t f;
  if (e >= 897 && e <= 1150) {  // binary32 exponent e - 1023 + 127 in [1, 254]
    const uint64_t m = b & 0x000fffffffffffffull;  // 52 fraction bits
    const uint32_t keep = (uint32_t)(m >> 29);     // the 23 that stay
    const uint32_t rest = (uint32_t)(m & 0x1fffffffu);
    // ties to even; a carry out of the fraction raises the exponent (to
    // infinity from the largest binade), as the format requires
    const uint32_t up = (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) ? 1u : 0u;
    f = sign | ((((uint32_t)(e - 896)) << 23) + keep + up);
  } else if (e > 1150 && e < 0x7ff) {  // finite, beyond the binary32 range
    f = sign | 0x7f800000u;
  } else if ((b << 1) == 0) {  // +-0
    f = sign;
  } else {
    return (float)x;  // binary32 subnormal or zero after rounding, infinity, NaN
  }
  float out;
#ifdef __CUDA_ARCH__
  out = __uint_as_float(f);
#else
  std::memcpy(&out, &f, sizeof out);
#endif
  return out;
}

// binary32 -> TF32 (the sign, the 8 exponent bits and the top 10 of the 23
// fraction bits; the 13 dropped bits are zero in the result), round to
// nearest, ties away from zero, on the bit pattern: add half a unit of the
// last kept bit (bit 12) to the magnitude and clear the dropped bits.  A
// carry out of the fraction moves the value to the next binade, which is the
// correctly rounded result.  For finite values below the largest binade.
SEM_F32R_FN uint32_t tf32_bits_rna(uint32_t f32_bits) { return (f32_bits + 0x1000u) & 0xFFFFE000u; }

}  // namespace sem
