"""Pins of the oracle's dual (Andersen-Broadie primal-dual) upper bound.

* Exact: every pathwise maximum includes n = 0, where the martingale is 0,
  so the bound is never below the payoff of immediate exercise.
* The martingale has mean zero: its value at maturity averages to 0 within
  its standard error (a dropped or shifted increment, or a wrong sign,
  biases it).
* The bound lies above the out-of-sample lower bound, and in the
  Black-Scholes limit the two bracket the binomial Bermudan price.
* More inner paths make the bound tighter (the inner noise biases the
  pathwise maximum upwards).
"""
import numpy as np

import oracle
import refs

H = dict(S0=100.0, r=0.03, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


def test_bound_not_below_immediate_exercise():
    m = oracle.heston(**H)
    # K = 150: exercising at once is optimal (the European put is worth
    # 150 exp(-rT) - 100 < 50); the bound is >= 50 exactly, and above it only
    # by the inner estimates' noise, which the pathwise maximum picks up
    r = oracle.dual_bound(m, [150.0, 100.0], 1.0, 3000, 12, 64, 256, basis=oracle.BASIS_S2,
                          seed=2, stream=5)
    assert r[0]["upper"] >= 50.0 and r[0]["upper"] < 50.0 + 0.5
    assert r[1]["upper"] >= 0.0


def test_martingale_has_mean_zero():
    m = oracle.heston(**H)
    for K, row in zip([90.0, 100.0, 115.0],
                      oracle.dual_bound(m, [90.0, 100.0, 115.0], 1.0, 4000, 16, 256, 32,
                                        basis=oracle.BASIS_SV2, seed=7, stream=1)):
        assert abs(row["pi_N"]) < 4.0 * row["pi_N_se"], (K, row)
        assert row["pi_N_se"] > 0.0


def test_upper_above_lower():
    m = oracle.heston(**H)
    for row in oracle.dual_bound(m, [90.0, 100.0, 110.0], 1.0, 6000, 16, 192, 64,
                                 basis=oracle.BASIS_SV2, seed=3, stream=1):
        se = np.hypot(row["lower_se"], row["upper_se"])
        assert row["upper"] > row["lower"] - 2.0 * se
        assert row["upper"] - row["lower"] < 0.2 * row["lower"]


def test_bounds_bracket_the_binomial_bermudan():
    m = oracle.heston(S0=100.0, r=0.05, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=1e-4, rho=0.0)
    N, T = 12, 1.0
    for K, row in zip([95.0, 105.0], oracle.dual_bound(m, [95.0, 105.0], T, 20000, N, 200, 100,
                                                        basis=oracle.BASIS_S2, seed=5, stream=2)):
        ref = refs.crr_bermudan(100.0, K, T, 0.05, 0.0, 0.2, False, N, 80)
        assert row["lower"] < ref + 3.0 * row["lower_se"], (K, row, ref)
        assert row["upper"] > ref - 3.0 * row["upper_se"], (K, row, ref)
        assert row["upper"] - ref < 0.05 * ref


def test_more_inner_paths_tighten_the_bound():
    m = oracle.heston(**H)
    kw = dict(basis=oracle.BASIS_S2, seed=4, stream=3)
    few = oracle.dual_bound(m, [100.0], 1.0, 4000, 12, 256, 8, **kw)[0]
    many = oracle.dual_bound(m, [100.0], 1.0, 4000, 12, 256, 128, **kw)[0]
    assert many["lower"] == few["lower"]
    assert many["upper"] < few["upper"]
