"""Writes kernel_poly.cuh: the sparse kernel of Eq. (kernel) in a form that
FP32 evaluates to a small *relative* error everywhere on [0, l).

f(r) = (2 + cos 2 pi r)(1 - r)/3 + sin(2 pi r)/(2 pi) has a fifth-order zero at
r = 1 (f ~ 4 pi^4 / 45 (1 - r)^5), so the textbook form loses all relative
precision there to cancellation.  With u = 1 - r,
    f = u^5 Q(u^2),   Q(w) = f(1 - sqrt(w)) / w^(5/2),
and Q is analytic and bounded on [0, 1] (Q(0) = 4 pi^4 / 45, Q(1) = 1).
Q is approximated by Chebyshev interpolation of degree N at the N+1
Chebyshev nodes of [0, 1] (values from mpmath at 60 digits), converted to
monomials in x = 2w - 1 for a Horner evaluation.  Degree 7 is enough: FP32
Horner evaluation of degrees 7, 8 and 9 all land at about 3.4e-7 relative
(the rounding floor), degree 6 at about 1e-6.  A second evaluator,
kernel_q2, takes two arguments at once with the packed FP32 instructions of
sm_100 and later (fma.rn.f32x2), with the same operations per lane.

The backward pass needs the slope.  In u, f is odd (f = (2 + cos 2 pi u) u/3
- sin(2 pi u)/(2 pi)), so df/du is even with a fourth-order zero at u = 0:
    df/dr = -df/du = -u^4 D(u^2),   D(w) = (df/du)(sqrt(w)) / w^2,
with D analytic on [0, 1] (D(0) = 4 pi^4 / 9, D(1) = 0), interpolated the same
way (degree ND).

Run:  python gen_kernel_poly.py   (from this directory)
"""
import os

import mpmath as mp
import numpy as np
from numpy.polynomial import chebyshev as Ch

N = 7
ND = 10
mp.mp.dps = 60


def f(r):
    r = mp.mpf(r)
    return (2 + mp.cos(2 * mp.pi * r)) * (1 - r) / 3 + mp.sin(2 * mp.pi * r) / (2 * mp.pi)


def Q(w):
    u = mp.sqrt(mp.mpf(w))
    return f(1 - u) / u ** 5


def dfdu(u):
    u = mp.mpf(u)
    return (2 - 2 * mp.cos(2 * mp.pi * u)) / 3 - 2 * mp.pi * u * mp.sin(2 * mp.pi * u) / 3


def D(w):
    u = mp.sqrt(mp.mpf(w))
    return dfdu(u) / u ** 4


def coefficients(fn=Q, n=N):
    k = np.arange(n + 1)
    x = np.cos(np.pi * (k + 0.5) / (n + 1))
    vals = np.array([float(fn((xi + 1) / 2)) for xi in x])
    return Ch.cheb2poly(Ch.chebfit(x, vals, n))


def horner(name, c, what):
    lines = ["// %s" % what,
             "__device__ __forceinline__ float %s(float w) {" % name,
             "  const float x = __fmaf_rn(2.0f, w, -1.0f);",
             "  float acc = %.9ef;" % c[-1]]
    for a in c[-2::-1]:
        lines.append("  acc = __fmaf_rn(acc, x, %.9ef);" % a)
    lines += ["  return acc;", "}", ""]
    return lines


def horner2(name, c, what):
    lines = ["// %s, two arguments at once (packed FP32)" % what,
             "__device__ __forceinline__ float2 %s(float2 w) {" % name,
             "  const float2 x = __ffma2_rn(make_float2(2.0f, 2.0f), w, make_float2(-1.0f, -1.0f));",
             "  float2 acc = make_float2(%.9ef, %.9ef);" % (c[-1], c[-1])]
    for a in c[-2::-1]:
        lines.append("  acc = __ffma2_rn(acc, x, make_float2(%.9ef, %.9ef));" % (a, a))
    lines += ["  return acc;", "}", ""]
    return lines


def main():
    lines = [
        "// Generated by gen_kernel_poly.py - do not edit.",
        "// Sparse kernel f(r) of Eq. (kernel) as f = u^5 Q(u^2) and its slope as",
        "// df/dr = -u^4 D(u^2), u = 1 - r, with Q and D Chebyshev interpolants on",
        "// w = u^2 in [0, 1], stored as monomials in x = 2w - 1.",
        "#pragma once",
        "",
        "namespace sbki {",
        "",
        "constexpr int kPolyDegree = %d;" % N,
        "constexpr int kSlopeDegree = %d;" % ND,
    ]
    lines += horner("kernel_q", coefficients(Q, N), "Q(w), degree %d" % N)
    lines += horner2("kernel_q2", coefficients(Q, N), "Q(w), degree %d" % N)
    lines += horner("kernel_dq", coefficients(D, ND), "D(w), degree %d" % ND)
    lines += ["}  // namespace sbki", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kernel_poly.cuh")
    with open(out, "w") as fh:
        fh.write("\n".join(lines))
    print("wrote", out)


if __name__ == "__main__":
    main()
