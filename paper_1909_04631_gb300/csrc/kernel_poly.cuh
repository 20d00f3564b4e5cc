// Generated by gen_kernel_poly.py - do not edit.
// Sparse kernel f(r) of Eq. (kernel) as f = u^5 Q(u^2) and its slope as
// df/dr = -u^4 D(u^2), u = 1 - r, with Q and D Chebyshev interpolants on
// w = u^2 in [0, 1], stored as monomials in x = 2w - 1.
#pragma once

namespace sbki {

constexpr int kPolyDegree = 9;
constexpr int kSlopeDegree = 10;
// Q(w), degree 9
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

// D(w), degree 10
__device__ __forceinline__ float kernel_dq(float w) {
  const float x = __fmaf_rn(2.0f, w, -1.0f);
  float acc = 1.146870215e-07f;
  acc = __fmaf_rn(acc, x, -2.831900989e-06f);
  acc = __fmaf_rn(acc, x, 5.735115500e-05f);
  acc = __fmaf_rn(acc, x, -9.404646384e-04f);
  acc = __fmaf_rn(acc, x, 1.211086324e-02f);
  acc = __fmaf_rn(acc, x, -1.182858189e-01f);
  acc = __fmaf_rn(acc, x, 8.361659899e-01f);
  acc = __fmaf_rn(acc, x, -4.002633205e+00f);
  acc = __fmaf_rn(acc, x, 1.171144129e+01f);
  acc = __fmaf_rn(acc, x, -1.752460235e+01f);
  acc = __fmaf_rn(acc, x, 9.086689068e+00f);
  return acc;
}

}  // namespace sbki
