// Exact rounding of an integer quotient to FP32, shared by the segment pass
// (centroids) and the soft-label weight means.
#pragma once

#include <cstdint>

namespace sbki {

// round(T 2^E / n) to FP32, nearest with ties to even, for 0 < T < 2^64 and
// 0 < n < 2^16; false when the result is below the FP32 normal range.  The
// integer quotient is estimated twice with a single-precision reciprocal of n,
// every rounding toward zero so that no estimate exceeds the true quotient,
// and each estimate is corrected with its exact integer remainder.
__device__ __forceinline__ bool round_mean64(unsigned long long T, uint32_t n, int E, float& out) {
  const int bt = 64 - __clzll((long long)T), bn = 32 - __clz((int)n);
  const int k = 26 + bn - bt;  // q = floor(T 2^k / n) lies in [2^25, 2^27)
  unsigned long long num;
  bool sticky;
  if (k >= 0) {
    num = T << k;  // below 2^(26 + bn) <= 2^42
    sticky = false;
  } else {
    num = T >> -k;
    sticky = (T & ((1ull << -k) - 1ull)) != 0ull;
  }
  const float r = __frcp_rz((float)n);
  unsigned long long q = (unsigned long long)__fmul_rz(__ull2float_rz(num), r);  // short by at most 48
  unsigned long long rem = num - q * n;                                           // below 49 n < 2^22
  q += (unsigned long long)__fmul_rz((float)rem, r);                              // short by at most 1
  rem = num - q * n;
  if (rem >= n) {
    ++q;
    rem -= n;
  }
  sticky = sticky || rem != 0ull;
  const int qb = 64 - __clzll((long long)q);  // 26 or 27
  const int lead = qb - 1 - k + E;            // exponent of the leading bit
  if (lead < -126) return false;
  const int sh = qb - 24;
  uint32_t mant = (uint32_t)(q >> sh);
  const uint32_t rb = (uint32_t)q & ((1u << sh) - 1u), half = 1u << (sh - 1);
  if (rb > half || (rb == half && (sticky || (mant & 1u)))) ++mant;
  int ex = lead;
  if (mant == (1u << 24)) {
    mant >>= 1;
    ++ex;
  }
  out = __uint_as_float(((uint32_t)(ex + 127) << 23) | (mant & 0x7fffffu));
  return true;
}

}  // namespace sbki
