"""Write quantile_f32.h: the coefficients of the single-precision normal
quantile of the forward pass, fitted in 40-digit arithmetic with mpmath.

    python paper_2206_03719_gb300/csrc/gen_quantile_f32.py

Method (the variable transformation of M. Giles, "Approximating the erfinv
function", GPU Computing Gems Jade Edition, 2011; the coefficients here are
this script's own fit): with x = 2u - 1 and w = -log(1 - x^2) =
-log(4 u (1 - u)), erfinv(x) / x is a smooth function of w, so

    Phi^-1(u) = sqrt(2) erfinv(x) = x P(w - 2.5)         for w < 5,
              = x Q(sqrt(w) - 3)                         for w >= 5,

P and Q polynomials of degree 8 (the factor sqrt(2) folded into their
coefficients), fitted by relative least squares at Chebyshev nodes on
w in [0, 5] and sqrt(w) in [sqrt(5), sqrt(w_max)], w_max the value at the
23-bit uniform grid's end points u = 2^-24, 1 - 2^-24.  Evaluated in float
(u (1 - u) rounded once, the logarithm on the special-function unit, Horner
steps by fused multiply-adds), the result is within 1e-6 of the exact
quantile on every point of the grid, max(1, |z|) relative, under the
worst-case errors of the logarithm and square root (checked by
tests/test_quantile_f32.py, which emulates the float arithmetic).
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
DEGREE = 8
NODES = 400


def f32(x):
    return float(np.float32(float(x)))


def erfinv_over_x(w):
    x = mp.sqrt(-mp.expm1(-w))
    return mp.erfinv(x) / x if x > 0 else mp.sqrt(mp.pi) / 2


def fit(fn, lo, hi):
    """Coefficients c_0..c_DEGREE of sum c_k t^k ~ fn(t) on [lo, hi], least
    squares in the relative error at Chebyshev nodes (40-digit solve)."""
    ts = [(lo + hi) / 2 + (hi - lo) / 2 * mp.cos(mp.pi * (k + mp.mpf(0.5)) / NODES)
          for k in range(NODES)]
    ys = [fn(t) for t in ts]
    A = mp.matrix(NODES, DEGREE + 1)
    b = mp.matrix(NODES, 1)
    for i, (t, y) in enumerate(zip(ts, ys)):
        for k in range(DEGREE + 1):
            A[i, k] = t ** k / y
        b[i] = 1
    c = mp.lu_solve(A.T * A, A.T * b)
    return [c[k] for k in range(DEGREE + 1)]


def main():
    w_max = -mp.log(4 * mp.mpf(2) ** -24 * (1 - mp.mpf(2) ** -24))
    sqrt2 = mp.sqrt(2)
    # central: t = w - 2.5 on [-2.5, 2.5]; tail: s = sqrt(w) - 3
    cen = fit(lambda t: sqrt2 * erfinv_over_x(t + mp.mpf(2.5)), mp.mpf(-2.5), mp.mpf(2.5))
    s_lo, s_hi = mp.sqrt(5) - 3, mp.sqrt(w_max) - 3
    tail = fit(lambda s: sqrt2 * erfinv_over_x((s + 3) ** 2), s_lo, s_hi)
    ln2 = mp.log(2)
    lines = [
        "// quantile_f32.h -- written by gen_quantile_f32.py (40-digit mpmath); do not edit.",
        "#pragma once",
        "",
        "namespace lsmc {",
        "",
        "// Phi^-1(u) = x P(w - 2.5) (w < 5) or x Q(sqrt(w) - 3) (w >= 5), x = 2u - 1,",
        "// w = -log(4 u (1 - u)); P(t) = sum kQfP<k> t^k, Q(s) = sum kQfQ<k> s^k.",
        "constexpr float kQfNegLn2 = %.9ef;  // -ln 2" % f32(-ln2),
        "constexpr float kQfShift = %.9ef;   // -2 ln 2 - 2.5" % f32(-2 * ln2 - mp.mpf(2.5)),
        "constexpr float kQfSplit = 2.5f;             // w = 5",
    ]
    lines += ["constexpr float kQfP%d = %.9ef;" % (k, f32(c)) for k, c in enumerate(cen)]
    lines += ["constexpr float kQfQ%d = %.9ef;" % (k, f32(c)) for k, c in enumerate(tail)]
    lines += ["", "}  // namespace lsmc", ""]
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "quantile_f32.h"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
