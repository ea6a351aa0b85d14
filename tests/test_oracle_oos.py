"""Pins of the oracle's out-of-sample Longstaff-Schwartz estimator.

* Applied to the regression paths themselves it is the in-sample
  estimator, exactly (the stopping time of the estimated policy is the first
  date where the rule exercises, the backward recursion's result).
* European contracts: the discounted mean payoff of the pricing paths.
* Low bias: on independent paths its price stays below the binomial
  Bermudan price of the Black-Scholes limit (the policy is suboptimal), and
  within a few standard errors of it.
"""
import numpy as np
import pytest

import oracle
import refs

H = dict(S0=100.0, r=0.03, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


@pytest.mark.parametrize("basis", [oracle.BASIS_S2, oracle.BASIS_SV2])
@pytest.mark.parametrize("type_,K", [(oracle.PUT, 100.0), (oracle.CALL, 95.0)])
def test_out_of_sample_on_the_same_paths_is_in_sample(basis, type_, K):
    m = oracle.heston(**dict(H, q=0.02))
    S, V = oracle.paths(m, 1.0, oracle.QE, 3000, 20, 9, 0)
    ins = oracle.lsmc(S, V, 100.0, K, 1.0, 0.03, 0.04, type_=type_, basis=basis)
    oos = oracle.lsmc_oos(S, V, S, V, 100.0, K, 1.0, 0.03, 0.04, type_=type_, basis=basis)
    assert oos["price"] == ins["price"]
    assert oos["continuation"] == ins["continuation"]
    assert oos["european_price"] == ins["european_price"]


def test_european_is_the_mean_discounted_payoff():
    m = oracle.heston(**H)
    SA, VA = oracle.paths(m, 1.0, oracle.QE, 2000, 12, 3, 0)
    SB, VB = oracle.paths(m, 1.0, oracle.QE, 2000, 12, 3, 7)
    oos = oracle.lsmc_oos(SA, VA, SB, VB, 100.0, 105.0, 1.0, 0.03, 0.04,
                          style=oracle.EUROPEAN)
    ref = np.exp(-0.03) * np.maximum(105.0 - SB[-1], 0.0).mean()
    assert abs(oos["price"] - ref) <= 1e-12 * ref


def test_low_biased_against_the_binomial_bermudan():
    # Black-Scholes limit (xi -> 0, v0 = theta, rho = 0): the American put
    # with 25 exercise dates has a binomial reference price
    m = oracle.heston(S0=100.0, r=0.05, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=1e-4, rho=0.0)
    P, N, K, T = 60000, 25, 105.0, 1.0
    out = oracle.price_greeks(m, [K], T, P, N, basis=oracle.BASIS_S2, seed=5, stream=2,
                              out_of_sample=True, b=oracle.bumps(greek_mask=0))[0]
    ins = oracle.price_greeks(m, [K], T, P, N, basis=oracle.BASIS_S2, seed=5, stream=2,
                              b=oracle.bumps(greek_mask=0))[0]
    ref = refs.crr_bermudan(100.0, K, T, 0.05, 0.0, 0.2, False, N, 80)
    se = out["price_se"]
    assert out["price"] < ref + 2 * se
    assert abs(out["price"] - ref) < 6 * se + 0.01 * ref
    # two different path sets: the estimates differ
    assert out["price"] != ins["price"]
