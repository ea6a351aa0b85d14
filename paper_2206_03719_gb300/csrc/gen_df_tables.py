"""Write df_tables.h: the constant tables of the float-pair exp and normal
quantile (dfloat.cuh), computed in 50-digit arithmetic with mpmath.

    python paper_2206_03719_gb300/csrc/gen_df_tables.py

Tables:
* 2^(j/128), j = 0..127, as float pairs, for exp(a) = 2^n 2^(j/128) exp(r);
* ln2 / 128 split into three floats (Cody and Waite's reduction): the first
  with few enough bits that k times it is exact for every |k| < 2^14;
* for the double-precision exp: 2^(j/128) rounded to double and ln2 / 128 in
  two doubles (the reduction runs in fused multiply-adds, so the first part
  needs no trailing zeros);
* G(z) = Phi(z) exp(z^2 / 2) on z <= 0 (Phi the standard normal
  distribution function) as one polynomial in x = z - c per interval,
  fitted by interpolation at Chebyshev nodes.  Intervals: [-0.25, 0]
  (c = 0), [-0.5, -0.25] (c = -0.375), then (-(i/2), -(i-1)/2] for
  i = 2..17 (c the midpoint).  For every |z| >= 0.25 the midpoint and z are
  multiples of ulp(z) less than 2^24 ulps apart, so x = z - c is exact in
  float.  Coefficients up to x^(N_PAIR - 1) are float pairs; the rest, whose
  terms stay below 2^-25 of G on the interval, are floats.
"""
import os

import mpmath as mp

mp.mp.dps = 50

N_EXP = 128
DEGREE = 11
N_PAIR = 9
N_INTERVALS = 18


def f32(x):
    import numpy as np
    return float(np.float32(float(x)))


def split(x):
    """x -> (hi, lo) floats, hi = float(x), lo = float(x - hi)."""
    hi = f32(x)
    lo = f32(mp.mpf(x) - mp.mpf(hi))
    return hi, lo


def short_float(x, bits):
    """x rounded to a float with at most `bits` significant bits."""
    e = mp.floor(mp.log(abs(x), 2))
    q = mp.mpf(2) ** (e - bits + 1)
    return float(mp.nint(x / q) * q)


def G(z):
    return mp.ncdf(z) * mp.exp(z * z / 2)


def interval(i):
    if i == 0:
        return mp.mpf(-0.25), mp.mpf(0), mp.mpf(0)
    if i == 1:
        return mp.mpf(-0.5), mp.mpf(-0.25), mp.mpf(-0.375)
    a, b = -mp.mpf(i) / 2, -mp.mpf(i - 1) / 2
    return a, b, (a + b) / 2


def fit(a, b, c):
    n = DEGREE + 1
    nodes = [(a + b) / 2 + (b - a) / 2 * mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n)
             for k in range(n)]
    A = mp.matrix([[(t - c) ** j for j in range(n)] for t in nodes])
    y = mp.matrix([G(t) for t in nodes])
    coef = mp.lu_solve(A, y)
    worst = 0
    for s in range(401):
        t = a + (b - a) * s / 400
        p = sum(coef[j] * (t - c) ** j for j in range(n))
        worst = max(worst, abs(p / G(t) - 1))
    h = max(abs(a - c), abs(b - c))
    gmin = min(G(a), G(b))
    tail = sum(abs(coef[j]) * h ** j for j in range(N_PAIR, n)) / gmin
    assert worst < 1e-16, (a, b, worst)
    assert tail < 2 ** -25, (a, b, tail)
    return coef, worst, tail


def main():
    out = []
    w = out.append
    w("// df_tables.h -- written by gen_df_tables.py (50-digit mpmath); do not edit.")
    w("#pragma once")
    w("")
    w("#include <cuda_runtime.h>")
    w("")
    w("namespace lsmc {")
    w("")
    L = mp.log(2) / N_EXP
    c1 = short_float(L, 10)
    c2 = f32(L - c1)
    c3 = f32(L - c1 - c2)
    w("constexpr int kExpTab = %d;" % N_EXP)
    w("constexpr float kExpInvL = %.9ef;  // %d / ln 2" % (f32(1 / L), N_EXP))
    w("constexpr float kExpC1 = %.9ef;    // ln 2 / %d in three parts" % (c1, N_EXP))
    w("constexpr float kExpC2 = %.9ef;" % c2)
    w("constexpr float kExpC3 = %.9ef;" % c3)
    w("")
    w("// 2^(j / %d), j = 0..%d: (hi, lo)" % (N_EXP, N_EXP - 1))
    w("static __device__ const float2 kExp2Frac[%d] = {" % N_EXP)
    for j in range(N_EXP):
        hi, lo = split(mp.mpf(2) ** (mp.mpf(j) / N_EXP))
        w("    {%.9ef, %.9ef}," % (hi, lo))
    w("};")
    w("")
    # double-precision exp: 2^(j / 128) rounded to double, ln 2 / 128 in two parts
    w("// double exp: 2^(j / %d), j = 0..%d, rounded to double" % (N_EXP, N_EXP - 1))
    w("static __device__ const double kExp2F64[%d] = {" % N_EXP)
    for j0 in range(0, N_EXP, 4):
        w("    " + ", ".join("%.17e" % float(mp.mpf(2) ** (mp.mpf(j) / N_EXP))
                             for j in range(j0, j0 + 4)) + ",")
    w("};")
    d1 = float(L)
    d2 = float(L - mp.mpf(d1))
    w("constexpr double kExpF64InvL = %.17e;  // %d / ln 2" % (float(1 / L), N_EXP))
    w("constexpr double kExpF64C1 = %.17e;    // ln 2 / %d in two parts" % (d1, N_EXP))
    w("constexpr double kExpF64C2 = %.17e;" % d2)
    w("")
    w("constexpr int kQDegree = %d;       // G polynomials: degree" % DEGREE)
    w("constexpr int kQPair = %d;         // coefficients 0..kQPair-1 are pairs" % N_PAIR)
    w("constexpr int kQIntervals = %d;" % N_INTERVALS)
    centres = []
    coefs = []
    for i in range(N_INTERVALS):
        a, b, c = interval(i)
        coef, worst, tail = fit(a, b, c)
        centres.append(float(c))
        coefs.append(coef)
        w("// interval %2d: [%6.3f, %6.3f] centre %7.4f: max rel. error %.1e, float tail %.1e"
          % (i, float(a), float(b), float(c), float(worst), float(tail)))
    w("static __device__ const float kQCentre[%d] = {%s};" % (
        N_INTERVALS, ", ".join("%.4ff" % c for c in centres)))
    w("// [k][interval]: coefficient of x^k (pairs for k < kQPair)")
    w("static __device__ const float2 kQCoefPair[%d][%d] = {" % (N_PAIR, N_INTERVALS))
    for k in range(N_PAIR):
        w("    {" + ", ".join("{%.9ef, %.9ef}" % split(coefs[i][k]) for i in range(N_INTERVALS)) + "},")
    w("};")
    w("static __device__ const float kQCoefFloat[%d][%d] = {" % (DEGREE + 1 - N_PAIR, N_INTERVALS))
    for k in range(N_PAIR, DEGREE + 1):
        w("    {" + ", ".join("%.9ef" % f32(coefs[i][k]) for i in range(N_INTERVALS)) + "},")
    w("};")
    w("")
    w("}  // namespace lsmc")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "df_tables.h")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
