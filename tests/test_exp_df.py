"""The float-pair exponential of the forward pass (df_math.cuh exp_df, the
S = S0 exp(x) of Sec. 2.2.1 on float pairs) emulated in float on the CPU,
operation by operation as the device runs it, against exp computed in
extended precision: within 2e-14 relative for |x| <= 70 (beyond, the low
word of the result leaves float's normal range).  The table and the three
parts of ln 2 / 128 are read from df_tables.h.  The device itself is checked
over the same range in tests/test_gpu_exp.py."""
import os
import re

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2206_03719_gb300", "csrc", "df_tables.h")
F32, F64, LD = np.float32, np.float64, np.longdouble


def _tables():
    text = open(HEADER).read()
    consts = {k: F32(float(v)) for k, v in
              re.findall(r"constexpr float (kExp\w+) = ([-+0-9.e]+)f;", text)}
    block = text[text.index("kExp2Frac["):]
    block = block[:block.index("};")]
    tab = np.array(re.findall(r"\{([-+0-9.e]+)f, ([-+0-9.e]+)f\}", block), dtype=F64)
    return consts, tab.astype(F32)


def _r(x):
    return np.asarray(x, dtype=F64).astype(F32)


def _add(a, b):
    return _r(a.astype(F64) + b.astype(F64))


def _sub(a, b):
    return _r(a.astype(F64) - b.astype(F64))


def _mul(a, b):
    return _r(a.astype(F64) * b.astype(F64))


def _fma(a, b, c):
    # the product of two floats is exact in long double; one rounding of the sum
    return (a.astype(LD) * b.astype(LD) + c.astype(LD)).astype(F32)


def _two_sum(a, b):
    s = _add(a, b)
    bb = _sub(s, a)
    return s, _add(_sub(a, _sub(s, bb)), _sub(b, bb))


def _quick_two_sum(a, b):
    s = _add(a, b)
    return s, _sub(b, _sub(s, a))


def _two_prod(a, b):
    p = _mul(a, b)
    return p, _fma(a, b, -p)


def _add_sloppy(ah, al, bh, bl):
    sh, sl = _two_sum(ah, bh)
    return _quick_two_sum(sh, _add(sl, _add(al, bl)))


def _exp_pair(ah, al, C, tab):
    full = lambda v: np.full_like(ah, v)  # noqa: E731
    kf = np.rint(_mul(ah, full(C["kExpInvL"]))).astype(F32)
    k = kf.astype(np.int64)
    t1 = _fma(-kf, full(C["kExpC1"]), ah)
    p2h, p2l = _two_prod(kf, full(C["kExpC2"]))
    dh, dl = _two_sum(t1, -p2h)
    eh, el = _two_sum(dh, al)
    rh, rl = _quick_two_sum(eh, _add(el, _sub(dl, _fma(kf, full(C["kExpC3"]), p2l))))
    r2h, r2l = _two_prod(rh, rh)
    r2l = _fma(_add(rh, rh), rl, r2l)
    tail = _mul(_mul(r2h, rh), _fma(rh, _fma(rh, full(F32(1 / 120)), full(F32(1 / 24))),
                                    full(F32(1 / 6))))
    sh, sl = _add_sloppy(rh, rl, _mul(r2h, full(F32(0.5))), _mul(r2l, full(F32(0.5))))
    sl = _add(sl, tail)
    th, tl = tab[k & 127, 0], tab[k & 127, 1]
    # T (1 + e) - T as an unnormalised product pair, then added to T
    p = _mul(th, sh)
    e = _fma(tl, sh, _fma(th, sl, _fma(th, sh, -p)))
    resh, resl = _add_sloppy(th, tl, p, e)
    scale = np.ldexp(np.ones_like(ah, dtype=F64), k >> 7).astype(F32)
    return _mul(resh, scale), _mul(resl, scale)


def test_float_pair_exponential_emulated():
    if np.finfo(LD).nmant < 60:
        pytest.skip("no extended-precision long double on this host")
    C, tab = _tables()
    assert tab.shape == (128, 2) and len(C) == 4
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-12.0, 12.0, 1 << 18), rng.uniform(-70.0, 70.0, 1 << 18),
                        np.array([0.0, 1e-30, -1e-30, 1.0, -1.0, 70.0, -70.0])])
    hi = x.astype(F32)
    lo = (x - hi.astype(F64)).astype(F32)
    held = hi.astype(LD) + lo.astype(LD)
    yh, yl = _exp_pair(hi, lo, C, tab)
    y = yh.astype(LD) + yl.astype(LD)
    rel = np.abs(y - np.exp(held)) / np.exp(held)
    assert rel.max() <= 2e-14, (float(rel.max()), x[np.argmax(rel)])
    assert yh[x == 0.0][0] == 1.0 and yl[x == 0.0][0] == 0.0
