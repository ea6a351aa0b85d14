"""The double-precision logarithm and normal quantile of the forward pass
(device_common.cuh log_f64 and norm_quantile_f64, tables and coefficients in
quantile_f64.h) emulated on the CPU operation by operation, every fused
multiply-add rounded once from its exact value (Python fractions), against
the exact functions (mpmath, 40 digits): the logarithm within 1.5 units in
the last place, the quantile within 6e-16 of Phi^-1(u), max(1, |z|)
relative, on the 52-bit uniform grid's end points, around the branch points
and on random grid points.  tests/test_gpu_quantile.py checks that the
device gives these emulated values bit for bit."""
import math
import os
import re
import struct
from fractions import Fraction

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2206_03719_gb300", "csrc", "quantile_f64.h")


def _tables():
    text = open(HEADER).read()
    consts = {k: float(v) for k, v in
              re.findall(r"constexpr double (k\w+) = ([-+0-9.e]+);", text)}
    arrays = {}
    for name in ("kLogRecip", "kLogNegHi", "kLogNegLo"):
        block = text[re.search(name + r"\[\d+\] = \{", text).end():]
        block = block[:block.index("};")]
        arrays[name] = [float(x) for x in block.replace("\n", " ").split(",") if x.strip()]
    return consts, arrays


C, T = _tables()


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _from_bits(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def log_f64(a):
    bits = _bits(a)
    assert 0x0010000000000000 <= bits < 0x7ff0000000000000
    e = float((bits >> 52) - 1023)
    m = _from_bits((bits & 0x000fffffffffffff) | 0x3ff0000000000000)
    j = (((bits >> 44) & 0xff) + 1) >> 1
    t = fma(m, T["kLogRecip"][j], -1.0)
    q = fma(t, 1.0 / 7.0, -1.0 / 6.0)
    q = fma(q, t, 1.0 / 5.0)
    q = fma(q, t, -1.0 / 4.0)
    q = fma(q, t, 1.0 / 3.0)
    q = fma(q, t, -0.5)
    lp = fma(t * t, q, t)
    hi = fma(e, C["kLn2Hi"], T["kLogNegHi"][j])
    return hi + fma(e, C["kLn2Lo"], T["kLogNegLo"][j] + lp)


def _horner(prefix, n, t):
    r = C["%s%d" % (prefix, n)]
    for k in range(n - 1, -1, -1):
        r = fma(r, t, C["%s%d" % (prefix, k)])
    return r


def quantile_f64(u, omu):
    w = -log_f64(4.0 * (u * omu))
    x = u - omu
    if w < C["kQdSplitW"]:
        r = _horner("kQdC", 23, w - C["kQdCentreW"])
    else:
        s = math.sqrt(w)
        r = (_horner("kQdT1_", 18, s - C["kQdCentreS1"]) if s < C["kQdSplitS"]
             else _horner("kQdT2_", 16, s - C["kQdCentreS2"]))
    return x * r


def grid_points():
    """Points (m + 1/2) 2^-52 of the uniform grid: both end points, the
    neighbourhoods of u = 1/2, of w = 6.25 and of sqrt(w) = 4 (both sides),
    and seeded random points spread over log(u)."""
    ms = [0, 1, 2, 3, (1 << 52) - 1, (1 << 52) - 2, (1 << 51) - 1, 1 << 51, (1 << 51) + 1]
    for w_b in (6.25, 16.0):
        # 4 u (1 - u) = exp(-w_b) on the lower side
        u_b = 0.5 * (1.0 - math.sqrt(1.0 - math.exp(-w_b)))
        m0 = int(u_b * 2.0 ** 52)
        ms += [m0 + d for d in range(-3, 4)]
        ms += [(1 << 52) - 1 - (m0 + d) for d in range(-3, 4)]
    rng = np.random.default_rng(64)
    logs = rng.uniform(-52.0 * math.log(2.0), math.log(0.5), 1500)
    for lu in logs:
        m = int(math.exp(lu) * 2.0 ** 52)
        ms += [m, (1 << 52) - 1 - m]
    return sorted({min(max(m, 0), (1 << 52) - 1) for m in ms})


def test_log_f64_within_1_5_ulp():
    mp.mp.dps = 40
    rng = np.random.default_rng(65)
    xs = list(np.exp(rng.uniform(-40.0, 40.0, 3000))) + [1.0, 2.0, 0.5, 1.0 - 2.0 ** -53,
                                                        1.0 + 2.0 ** -52, 2.0 ** -1000, 1e300]
    xs += list(1.0 + rng.uniform(-0.01, 0.01, 500))
    worst = 0.0
    for x in xs:
        x = float(x)
        got = log_f64(x)
        ref = mp.log(mp.mpf(x))
        if ref == 0:
            assert got == 0.0
            continue
        ulp = math.ulp(float(ref))
        worst = max(worst, float(abs(mp.mpf(got) - ref) / ulp))
    print("log_f64: worst %.3f ulp" % worst)
    assert worst <= 1.5


def test_quantile_f64_within_6e_16():
    mp.mp.dps = 40
    worst = 0.0
    for m in grid_points():
        u = (m + 0.5) * 2.0 ** -52
        omu = 1.0 - u
        assert 1.0 - omu == u  # exact on the grid
        z = quantile_f64(u, omu)
        ref = -mp.sqrt(2) * mp.erfinv(1 - 2 * mp.mpf(u))
        err = float(abs(mp.mpf(z) - ref) / max(1, abs(ref)))
        worst = max(worst, err)
    print("quantile_f64: worst %.3g" % worst)
    assert worst <= 6e-16


def test_quantile_f64_symmetric_and_zero_at_half():
    for m in grid_points()[::7]:
        u = (m + 0.5) * 2.0 ** -52
        assert quantile_f64(u, 1.0 - u) == -quantile_f64(1.0 - u, u)
    assert quantile_f64(0.5, 0.5) == 0.0
