// IEEE-754 binary64 / binary32 bit manipulations for the mixed-precision scale and correction
// kernels: exact power-of-two scaling and round-to-nearest-even narrowing done with integer
// operations only, because on this part the FP64 pipe (2 lanes per clock per SM) is the scarce
// unit and a conversion or multiply there costs as much as an addition of the stencil.
//
// Each fast path states when it applies and returns false otherwise; the kernels then take the
// plain floating-point form, whose result the fast path reproduces bit for bit whenever it
// applies.  The header compiles for the device (nvcc) and for the host (a C++ test checks it
// against the host compiler's own conversions).
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define GB_HD __host__ __device__ __forceinline__
#else
#define GB_HD inline
#endif

namespace gbmg {
namespace bits {

GB_HD uint64_t d2u(double d) {
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
}
GB_HD double u2d(uint64_t u) {
  double d;
  std::memcpy(&d, &u, 8);
  return d;
}
GB_HD uint32_t f2u(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
GB_HD float u2f(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
GB_HD int clz64(uint64_t x) {  // x != 0
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}
GB_HD int clz32(uint32_t x) {  // x != 0
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return __builtin_clz(x);
#endif
}

// e with 2^e <= s < 2^(e+1), for finite s > 0 (normal or subnormal).
GB_HD int floor_log2(double s) {
  const uint64_t b = d2u(s);
  const int E = (int)((b >> 52) & 0x7FF);
  return E ? E - 1023 : 63 - clz64(b) - 1074;
}

// 2^k exactly: 0 below the subnormal range, infinity above the normal range.
GB_HD double pow2(int k) {
  if (k > 1023) return u2d(0x7FF0000000000000ull);
  if (k >= -1022) return u2d((uint64_t)(k + 1023) << 52);
  if (k >= -1074) return u2d(1ull << (k + 1074));
  return 0.0;
}

// *out = r * 2^-e rounded to the nearest binary32 (ties to even), i.e. the value of
// (float)(r * 2^-e) with an exact product.  Applies when r is a normal double and the result is
// a normal float or rounds up to infinity; false otherwise (zero, subnormal, infinite or NaN r,
// or a result in the float subnormal range).
GB_HD bool scale_to_f32(double r, int e, float* out) {
  const uint64_t b = d2u(r);
  const int Er = (int)((b >> 52) & 0x7FF);
  if (Er == 0 || Er == 0x7FF) return false;
  const long long F = (long long)Er - 1023 - e + 127;  // biased binary32 exponent
  if (F < 1 || F > 254) return false;
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;          // 52 fraction bits
  uint32_t base = (uint32_t)(b >> 63) << 31 | (uint32_t)F << 23 | (uint32_t)(m >> 29);
  const uint64_t rem = m & 0x1FFFFFFFull, half = 0x10000000ull;  // the 29 dropped bits
  base += (rem > half || (rem == half && (base & 1u))) ? 1u : 0u;  // a carry bumps the exponent
  *out = u2f(base);
  return true;
}

// *out = 2^k * v exactly, for a finite float v whose scaled value is a normal double (zero
// included); false for infinite or NaN v or a result outside the normal double range.
GB_HD bool scaled_f32_to_f64(float v, int k, double* out) {
  const uint32_t u = f2u(v);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  int E = (int)((u >> 23) & 0xFF);
  uint32_t m = u & 0x7FFFFFu;
  if (E == 0xFF) return false;
  if (E == 0) {
    if (m == 0) {
      *out = u2d(sign);  // signed zero
      return true;
    }
    const int sh = clz32(m) - 8;  // normalise a subnormal float
    m = (m << sh) & 0x7FFFFFu;
    E = 1 - sh;
  }
  const long long D = (long long)E - 127 + 1023 + k;  // biased binary64 exponent
  if (D < 1 || D > 2046) return false;
  *out = u2d(sign | (uint64_t)D << 52 | (uint64_t)m << 29);
  return true;
}

}  // namespace bits
}  // namespace gbmg
