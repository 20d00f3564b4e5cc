// The sparse kernel of Eq. (kernel), k(d) = sigma0 f(d/l) for d < l, else 0,
//   f(r) = (2 + cos 2 pi r)(1 - r)/3 + sin(2 pi r)/(2 pi).
// kernel_f_poly: f = u^5 Q(u^2) with u = 1 - r (kernel_poly.cuh), accurate to a
//   few 1e-7 relative over the whole support, no cancellation near r = 1.
// kernel_f_trig: the textbook form with sincospif, kept as the reference the
//   polynomial is tested against (it loses relative accuracy as r -> 1).
#pragma once
#include "kernel_poly.cuh"

namespace sbki {

constexpr float kInvPi = 0.318309886183790671538f;

__device__ __forceinline__ float kernel_f_poly_u(float u) {
  u = fminf(fmaxf(u, 0.0f), 1.0f);
  const float w = u * u;
  return w * w * u * kernel_q(w);
}

__device__ __forceinline__ float kernel_f_poly(float r) { return kernel_f_poly_u(1.0f - r); }

__device__ __forceinline__ float kernel_f_trig(float r) {
  r = fminf(fmaxf(r, 0.0f), 1.0f);
  float s, c;
  sincospif(r, &s, &c);
  return (1.0f - r) * (1.0f - (2.0f / 3.0f) * s * s) + s * c * kInvPi;
}

}  // namespace sbki
