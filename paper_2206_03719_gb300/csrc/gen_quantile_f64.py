"""Write quantile_f64.h: the double-precision normal quantile and logarithm
of the forward pass, coefficients and tables computed in 50-digit arithmetic
with mpmath.

    python paper_2206_03719_gb300/csrc/gen_quantile_f64.py

Quantile (the variable transformation of M. Giles, "Approximating the erfinv
function", GPU Computing Gems Jade Edition, 2011; the coefficients here are
this script's own fit): with x = 2u - 1 and w = -log(4 u (1 - u)),

    Phi^-1(u) = x C(w - 3.125)            for w < 6.25,
              = x T1(sqrt(w) - 3.25)      for sqrt(w) in [2.5, 4),
              = x T2(sqrt(w) - 5.0)       for sqrt(w) >= 4,

C, T1, T2 polynomials of degree 23, 18 and 16 (the factor sqrt(2) of
Phi^-1(u) = sqrt(2) erfinv(2u - 1) folded in; evaluated by Horner's rule in
the functions qd_central, qd_tail1, qd_tail2 written here), fitted by
relative least squares at Chebyshev nodes; the last interval reaches the 52-bit uniform
grid's end points u = 2^-53, 1 - 2^-53 (sqrt(w) = 5.946).  With the
coefficients rounded to double, the polynomials are within 2.5e-16 of the
exact quotient on their intervals (checked below and by
tests/test_quantile_f64.py).

Logarithm (the table-driven reduction of P. T. P. Tang, "Table-driven
implementation of the logarithm function in IEEE floating-point arithmetic",
ACM TOMS 16(4), 1990, in the form with tabulated reciprocals): a = 2^e m,
m in [1, 2), j = the nearest integer to 128 (m - 1), c_j = 1 / (1 + j / 128)
rounded to double, t = m c_j - 1 by one fused multiply-add (|t| < 0.0040),
and log a = e ln 2 - log c_j + log1p(t), with -log c_j tabulated as a pair
(hi + lo) and log1p(t) by its Taylor series to t^7 (remainder below
|t|^8 / 8 < 6e-21).
"""
import os

import mpmath as mp

mp.mp.dps = 50
NODES = 300
W_SPLIT = mp.mpf("6.25")
S_SPLIT = mp.mpf(4)
T1_CENTRE = mp.mpf("3.25")
T2_CENTRE = mp.mpf(5)
DEG_C, DEG_T1, DEG_T2 = 23, 18, 16
LOG_TAB = 128


def g_of_w(w):
    """sqrt(2) erfinv(x) / x with w = -log(1 - x^2)."""
    x = mp.sqrt(-mp.expm1(-w))
    return mp.sqrt(2) * mp.erfinv(x) / x if x > 0 else mp.sqrt(mp.pi / 2)


def fit(fn, lo, hi, deg):
    """c_0..c_deg of sum c_k t^k ~ fn(t) on [lo, hi], least squares in the
    relative error at Chebyshev nodes (50-digit solve)."""
    ts = [(lo + hi) / 2 + (hi - lo) / 2 * mp.cos(mp.pi * (k + mp.mpf(0.5)) / NODES)
          for k in range(NODES)]
    A = mp.matrix(NODES, deg + 1)
    b = mp.matrix(NODES, 1)
    for i, t in enumerate(ts):
        y = fn(t)
        for k in range(deg + 1):
            A[i, k] = t ** k / y
        b[i] = 1
    c = mp.lu_solve(A.T * A, A.T * b)
    return [float(c[k]) for k in range(deg + 1)]


def max_rel_err(fn, coef, lo, hi, n=800):
    """Largest |p(t) / fn(t) - 1| of the double-rounded coefficients,
    evaluated exactly, on n + 1 equispaced points."""
    worst = mp.mpf(0)
    for k in range(n + 1):
        t = lo + (hi - lo) * mp.mpf(k) / n
        p = mp.mpf(0)
        for c in reversed(coef):
            p = p * t + mp.mpf(c)
        worst = max(worst, abs(p / fn(t) - 1))
    return float(worst)


def main():
    s_max = mp.sqrt(-mp.log(4 * mp.mpf(2) ** -53 * (1 - mp.mpf(2) ** -53)))
    half = W_SPLIT / 2
    central = fit(lambda t: g_of_w(t + half), -half, half, DEG_C)
    e_c = max_rel_err(lambda t: g_of_w(t + half), central, -half, half)
    lo1, hi1 = mp.sqrt(W_SPLIT) - T1_CENTRE, S_SPLIT - T1_CENTRE
    tail1 = fit(lambda t: g_of_w((t + T1_CENTRE) ** 2), lo1, hi1, DEG_T1)
    e_1 = max_rel_err(lambda t: g_of_w((t + T1_CENTRE) ** 2), tail1, lo1, hi1)
    lo2, hi2 = S_SPLIT - T2_CENTRE, s_max + mp.mpf("0.01") - T2_CENTRE
    tail2 = fit(lambda t: g_of_w((t + T2_CENTRE) ** 2), lo2, hi2, DEG_T2)
    e_2 = max_rel_err(lambda t: g_of_w((t + T2_CENTRE) ** 2), tail2, lo2, hi2)
    print("max relative error of the polynomials: central %.3g, tail 1 %.3g, tail 2 %.3g"
          % (e_c, e_1, e_2))
    assert max(e_c, e_1, e_2) < 2.5e-16

    # logarithm: reciprocals and -log of them (hi + lo); ln 2 in two parts,
    # the first with 42 significant bits so that e ln2_hi is exact for |e| < 2^11
    ln2 = mp.log(2)
    ln2_hi = float(mp.floor(ln2 * 2 ** 42) / 2 ** 42)
    ln2_lo = float(ln2 - mp.mpf(ln2_hi))
    recip, neg_hi, neg_lo = [], [], []
    for j in range(LOG_TAB + 1):
        c = float(1 / (1 + mp.mpf(j) / LOG_TAB))
        L = -mp.log(mp.mpf(c))
        hi = float(L)
        recip.append(c)
        neg_hi.append(hi)
        neg_lo.append(float(L - mp.mpf(hi)))

    def arr(name, vals):
        body = ",\n".join("    %.17e" % v for v in vals)
        return ["static __device__ const double %s[%d] = {" % (name, len(vals)), body, "};"]

    def coefs(prefix, vals):
        return ["constexpr double %s%d = %.17e;" % (prefix, k, v) for k, v in enumerate(vals)]

    lines = [
        "// quantile_f64.h -- written by gen_quantile_f64.py (50-digit mpmath); do not edit.",
        "#pragma once",
        "",
        "namespace lsmc {",
        "",
        "// Phi^-1(u) = x C(w - 3.125) (w < 6.25), x T1(sqrt(w) - 3.25) (sqrt(w) < 4),",
        "// x T2(sqrt(w) - 5) beyond; x = 2u - 1, w = -log(4 u (1 - u)).",
        "constexpr double kQdSplitW = 6.25;",
        "constexpr double kQdCentreW = 3.125;",
        "constexpr double kQdSplitS = 4.0;",
        "constexpr double kQdCentreS1 = 3.25;",
        "constexpr double kQdCentreS2 = 5.0;",
    ]
    lines += coefs("kQdC", central) + coefs("kQdT1_", tail1) + coefs("kQdT2_", tail2)

    def horner(fname, prefix, n):
        out = ["", "__device__ __forceinline__ double %s(double t) {" % fname,
               "  double r = %s%d;" % (prefix, n)]
        out += ["  r = fma(r, t, %s%d);" % (prefix, k) for k in range(n - 1, -1, -1)]
        return out + ["  return r;", "}"]

    lines += horner("qd_central", "kQdC", DEG_C) + horner("qd_tail1", "kQdT1_", DEG_T1)
    lines += horner("qd_tail2", "kQdT2_", DEG_T2)
    lines += [
        "",
        "// log: a = 2^e m, j = round(128 (m - 1)), t = m kLogRecip[j] - 1,",
        "// log a = e ln2 + (kLogNegHi[j] + kLogNegLo[j]) + log1p(t)",
        "constexpr double kLn2Hi = %.17e;  // 42 significant bits" % ln2_hi,
        "constexpr double kLn2Lo = %.17e;" % ln2_lo,
    ]
    lines += arr("kLogRecip", recip) + arr("kLogNegHi", neg_hi) + arr("kLogNegLo", neg_lo)
    lines += ["", "}  // namespace lsmc", ""]
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "quantile_f64.h"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
