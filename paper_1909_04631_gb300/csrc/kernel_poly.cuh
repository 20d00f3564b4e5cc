// Generated by gen_kernel_poly.py - do not edit.
// Sparse kernel f(r) of Eq. (kernel) as f = u^5 Q(u^2) and its slope as
// df/dr = -u^4 D(u^2), u = 1 - r, with Q and D Chebyshev interpolants on
// w = u^2 in [0, 1], stored as monomials in x = 2w - 1.
#pragma once

namespace sbki {

constexpr int kPolyDegree = 7;
constexpr int kSlopeDegree = 10;
// Q(w), degree 7
__device__ __forceinline__ float kernel_q(float w) {
  const float x = __fmaf_rn(2.0f, w, -1.0f);
  float acc = -5.214391041e-05f;
  acc = __fmaf_rn(acc, x, 7.608289382e-04f);
  acc = __fmaf_rn(acc, x, -8.489671500e-03f);
  acc = __fmaf_rn(acc, x, 7.084753925e-02f);
  acc = __fmaf_rn(acc, x, -4.154038500e-01f);
  acc = __fmaf_rn(acc, x, 1.578207845e+00f);
  acc = __fmaf_rn(acc, x, -3.405347268e+00f);
  acc = __fmaf_rn(acc, x, 3.179476699e+00f);
  return acc;
}

// Q(w), degree 7, two arguments at once (packed FP32)
__device__ __forceinline__ float2 kernel_q2(float2 w) {
  const float2 x = __ffma2_rn(make_float2(2.0f, 2.0f), w, make_float2(-1.0f, -1.0f));
  float2 acc = make_float2(-5.214391041e-05f, -5.214391041e-05f);
  acc = __ffma2_rn(acc, x, make_float2(7.608289382e-04f, 7.608289382e-04f));
  acc = __ffma2_rn(acc, x, make_float2(-8.489671500e-03f, -8.489671500e-03f));
  acc = __ffma2_rn(acc, x, make_float2(7.084753925e-02f, 7.084753925e-02f));
  acc = __ffma2_rn(acc, x, make_float2(-4.154038500e-01f, -4.154038500e-01f));
  acc = __ffma2_rn(acc, x, make_float2(1.578207845e+00f, 1.578207845e+00f));
  acc = __ffma2_rn(acc, x, make_float2(-3.405347268e+00f, -3.405347268e+00f));
  acc = __ffma2_rn(acc, x, make_float2(3.179476699e+00f, 3.179476699e+00f));
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
