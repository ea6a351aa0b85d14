"""Pins of the oracle's STAC-A2 multi-asset path reduction (Sec. 2.2.1,
Sec. 4.1): M = the largest asset value per path and date.

* one asset is the single-asset path generator, bit for bit;
* M is the elementwise maximum of the separately generated asset paths;
* in the Black-Scholes limit (xi -> 0, v0 = theta, rho = 0) each asset's
  log return over [0, T] is normal, the assets' returns are independent
  (rho_assets = 0) or equicorrelated (rho_assets > 0), so
  P(M_T <= K) = Phi(d)^A, or the bivariate normal distribution function
  Phi_2(d, d; rho_assets) for two assets, within binomial error.
"""
import math

import numpy as np
import pytest

import oracle

H = dict(S0=100.0, r=0.02, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


def test_one_asset_is_the_single_asset_path():
    m = oracle.heston(**H)
    for scheme in (oracle.QE, oracle.FT_EULER):
        M = oracle.multi_max([m], 0.75, scheme, 300, 12, 5, 2)
        S, _ = oracle.paths(m, 0.75, scheme, 300, 12, 5, 2)
        assert np.array_equal(M, S)


@pytest.mark.parametrize("rho_assets", [0.0, 0.35])
def test_reduction_is_the_max_of_the_asset_paths(rho_assets):
    models = [oracle.heston(**dict(H, S0=s0, v0=v0, xi=xi))
              for s0, v0, xi in ((100.0, 0.04, 0.3), (95.0, 0.09, 0.5), (105.0, 0.02, 0.2),
                                 (100.0, 0.05, 0.8))]
    P, N, T = 40, 9, 1.5
    M = oracle.multi_max(models, T, oracle.QE, P, N, 11, 4, rho_assets=rho_assets)
    for p in range(P):
        paths = np.stack([oracle.asset_path(m, a, T, oracle.QE, p, N, 11, 4, rho_assets)
                          for a, m in enumerate(models)])
        assert np.array_equal(M[:, p], paths.max(axis=0))
    # each asset draws its own stream: two identical models are not the same path
    twin = oracle.multi_max([models[0], models[0]], T, oracle.QE, P, N, 11, 4)
    single = oracle.multi_max([models[0]], T, oracle.QE, P, N, 11, 4)
    assert np.all(twin >= single) and np.any(twin > single)


def _bs_limit(A, rho_assets, K, P=40000, N=4, T=1.0):
    m = oracle.heston(S0=100.0, r=0.02, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=1e-5, rho=0.0)
    M = oracle.multi_max([m] * A, T, oracle.QE, P, N, 2024, 0, rho_assets=rho_assets)
    frac = float(np.mean(M[N] <= K))
    d = (math.log(K / 100.0) - (0.02 - 0.02) * T) / math.sqrt(0.04 * T)
    return frac, d, P


@pytest.mark.parametrize("K", [95.0, 105.0, 115.0])
def test_black_scholes_limit_independent_assets(K):
    frac, d, P = _bs_limit(3, 0.0, K)
    from scipy.stats import norm
    ref = norm.cdf(d) ** 3
    assert abs(frac - ref) < 4.5 * math.sqrt(ref * (1 - ref) / P)


@pytest.mark.parametrize("rho_assets", [0.3, 0.8])
def test_black_scholes_limit_equicorrelated_pair(rho_assets):
    from scipy.stats import multivariate_normal, norm
    for K in (98.0, 110.0):
        frac, d, P = _bs_limit(2, rho_assets, K)
        ref = multivariate_normal(mean=[0, 0], cov=[[1, rho_assets], [rho_assets, 1]]).cdf([d, d])
        assert abs(frac - ref) < 4.5 * math.sqrt(ref * (1 - ref) / P)
        # a sqrt dropped from the factor loading would give correlation
        # rho^2 or sqrt(rho): far outside the bound
        wrong = multivariate_normal(mean=[0, 0], cov=[[1, rho_assets ** 2],
                                                      [rho_assets ** 2, 1]]).cdf([d, d])
        assert abs(wrong - ref) > 10 * math.sqrt(ref * (1 - ref) / P)
    assert norm.cdf(0.0) == 0.5


def test_rejects_bad_arguments():
    m = oracle.heston(**H)
    with pytest.raises(ValueError):
        oracle.multi_max([m], 1.0, oracle.QE, 10, 4, 1, 0, rho_assets=1.5)
    with pytest.raises(ValueError):
        oracle.multi_max([m], 1.0, oracle.QE, 0, 4, 1, 0)
