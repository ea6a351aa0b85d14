"""The single-precision normal quantile of the forward pass (device_common.cuh
norm_quantile_f32, coefficients in quantile_f32.h) emulated in float on the
CPU over every point of the 23-bit uniform grid, against the double-precision
quantile (scipy's ndtri).  The emulation rounds to float after every
operation, as the device does; the device's logarithm and square root
(special-function unit, approximate) are bracketed by perturbing them by
their error bounds both ways.  The device itself is checked against the
oracle's quantile in tests/test_gpu_stages.py."""
import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2206_03719_gb300", "csrc", "quantile_f32.h")


def _consts():
    text = open(HEADER).read()
    return {k: np.float32(float(v)) for k, v in
            re.findall(r"constexpr float (kQf\w+) = ([-+0-9.e]+)f;", text)}


def _r(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def _fma(a, b, c):
    # a * b of two floats is exact in double; one rounding of the sum
    return _r(a.astype(np.float64) * np.float64(b) + np.float64(c)) if np.isscalar(b) else \
        _r(a.astype(np.float64) * b.astype(np.float64) + np.float64(c))


def _quantile(u, omu, C, log_rel=0.0, sqrt_rel=0.0):
    p = _r(u.astype(np.float64) * omu.astype(np.float64))
    lg = _r(np.log2(p.astype(np.float64)) * (1.0 + log_rel))
    t = _fma(lg, C["kQfNegLn2"], C["kQfShift"])
    x = _r(u.astype(np.float64) - omu.astype(np.float64))
    P = np.full_like(t, C["kQfP8"])
    for k in range(7, -1, -1):
        P = _fma(P, t, C["kQfP%d" % k])
    w = _r(t.astype(np.float64) + 2.5)
    s = _r(np.sqrt(w.astype(np.float64)) * (1.0 + sqrt_rel))
    s = _r(s.astype(np.float64) - 3.0)
    Q = np.full_like(s, C["kQfQ8"])
    for k in range(7, -1, -1):
        Q = _fma(Q, s, C["kQfQ%d" % k])
    r = np.where(t < C["kQfSplit"], P, Q)
    return _r(x.astype(np.float64) * r.astype(np.float64)), t < C["kQfSplit"]


@pytest.mark.slow
def test_float_quantile_on_every_grid_point():
    C = _consts()
    assert len(C) == 21
    m = np.arange(0, 1 << 23, dtype=np.float64)
    u = _r((m + 0.5) * 2.0 ** -23)
    omu = _r(1.0 - u.astype(np.float64))
    assert np.array_equal(omu.astype(np.float64), 1.0 - u.astype(np.float64))  # exact
    ref = scipy_special.ndtri(u.astype(np.float64))
    scale = np.maximum(1.0, np.abs(ref))
    for log_rel in (0.0, 2.0 ** -21, -2.0 ** -21):
        for sqrt_rel in (0.0, 2.0 ** -22, -2.0 ** -22):
            z, central = _quantile(u, omu, C, log_rel, sqrt_rel)
            err = np.abs(z.astype(np.float64) - ref) / scale
            assert err.max() < 1e-6, (log_rel, sqrt_rel, err.max(), u[np.argmax(err)])
    # the tail branch serves about 0.34% of the draws
    assert 0.002 < (~central).mean() < 0.005
    # symmetry: quantile(1 - u) = -quantile(u) up to one rounding each
    z, _ = _quantile(u, omu, C)
    zs, _ = _quantile(omu, u, C)
    assert np.array_equal(z, -zs)
