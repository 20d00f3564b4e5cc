// Generated by gen_kernel_poly.py - do not edit.
// Sparse kernel f(r) of Eq. (kernel) as f = u^5 Q(u^2), u = 1 - r, with Q a degree-9
// Chebyshev interpolant on w = u^2 in [0, 1], stored as monomials in x = 2w - 1.
#pragma once

namespace sbki {

constexpr int kPolyDegree = 9;
__device__ __forceinline__ float kernel_q(float w) {
  const float x = __fmaf_rn(2.0f, w, -1.0f);
  float acc = -1.271203416e-07f;
  acc = __fmaf_rn(acc, x, 2.851444719e-06f);
  acc = __fmaf_rn(acc, x, -5.188967920e-05f);
  acc = __fmaf_rn(acc, x, 7.551263435e-04f);
  acc = __fmaf_rn(acc, x, -8.489830386e-03f);
  acc = __fmaf_rn(acc, x, 7.085110312e-02f);
  acc = __fmaf_rn(acc, x, -4.154038182e-01f);
  acc = __fmaf_rn(acc, x, 1.578207132e+00f);
  acc = __fmaf_rn(acc, x, -3.405347269e+00f);
  acc = __fmaf_rn(acc, x, 3.179476721e+00f);
  return acc;
}

}  // namespace sbki
