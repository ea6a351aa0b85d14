"""Pins of the oracle's Longstaff-Schwartz pass, scenario table and Greeks
(CPU only).

* the per-date regression equals a least-squares solve by QR (numpy lstsq)
  on the in-the-money design matrix, with the regression target rebuilt from
  the exercise decisions as a stopping time (not from the oracle's running
  cash-flow vector);
* the price equals the mean discounted payoff at that stopping time;
* with xi = 0 the model is Black-Scholes: the LSMC Bermudan price matches a
  CRR tree exercising on the same dates, and the Greeks of the European
  price match Black-Scholes Greeks within Monte Carlo error;
* American >= European, American call without dividends = European call,
  prices monotone in the strike.
"""
import math

import numpy as np
import pytest

import oracle
import refs

H = dict(S0=100.0, r=0.02, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


def _payoff(S, K, put):
    return np.maximum(K - S, 0.0) if put else np.maximum(S - K, 0.0)


def _basis(S, V, K, theta, basis, centre=1.0):
    x, w = S / K - centre, V / theta - centre
    cols = [np.ones_like(x), x, x * x]
    if basis == oracle.BASIS_SV2:
        cols += [w, x * w, w * w]
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("basis", [oracle.BASIS_S2, oracle.BASIS_SV2])
@pytest.mark.parametrize("put", [True, False])
@pytest.mark.parametrize("scheme", [oracle.QE, oracle.FT_EULER])
def test_backward_induction_is_least_squares_on_stopping_times(basis, put, scheme):
    P, N, T, r, theta = 256, 8, 0.5, 0.05, 0.04
    K = 100.0 if put else 98.0
    model = oracle.heston(**dict(H, r=r, q=0.03 if not put else 0.0))
    S, V = oracle.paths(model, T, scheme, P, N, 123, 2)
    d = oracle.lsmc(S, V, 100.0, K, T, r, theta, type_=oracle.PUT if put else oracle.CALL,
                    basis=basis, want_detail=True)
    beta, ex = d["beta"], d["exercise"]
    dt = T / N
    B = 3 if basis == oracle.BASIS_S2 else 6
    assert not ex[0].any()
    n_reg = 0
    for n in range(N - 1, 0, -1):
        # stopping time after the decisions at dates > n
        tau = np.full(P, N)
        for m in range(N - 1, n, -1):
            tau = np.where(ex[m] == 1, m, tau)
        Y = np.exp(-r * (tau - n) * dt) * _payoff(S[tau, np.arange(P)], K, put)
        itm = _payoff(S[n], K, put) > 0
        assert not ex[n][~itm].any()
        if np.isnan(beta[n, 0]):
            assert itm.sum() < B or np.linalg.matrix_rank(_basis(S[n][itm], V[n][itm], K, theta, basis)) < B
            assert not ex[n].any()
            continue
        X = _basis(S[n][itm], V[n][itm], K, theta, basis)
        b_ls = np.linalg.lstsq(X, Y[itm], rcond=None)[0]
        cond = np.linalg.cond(X)
        # normal equations: coefficient error grows like cond(X)^2 * eps;
        # the fitted values are far better determined
        assert np.allclose(beta[n, :B], b_ls, rtol=0, atol=cond**2 * 1e-14 * np.abs(b_ls).max()), n
        assert np.allclose(X @ beta[n, :B], X @ b_ls, rtol=0, atol=cond * 1e-13 * np.abs(Y).max()), n
        cont = X @ beta[n, :B]
        h = _payoff(S[n][itm], K, put)
        assert np.array_equal(ex[n][itm] == 1, h > cont)
        n_reg += 1
    assert n_reg >= N - 3
    tau = np.full(P, N)
    for m in range(N - 1, 0, -1):
        tau = np.where(ex[m] == 1, m, tau)
    cont = (np.exp(-r * tau * dt) * _payoff(S[tau, np.arange(P)], K, put)).mean()
    assert abs(d["continuation"] - cont) < 1e-12 * abs(cont)
    assert d["price"] == max(_payoff(np.array([100.0]), K, put)[0], d["continuation"])
    eu = math.exp(-r * T) * _payoff(S[N], K, put).mean()
    assert abs(d["european_price"] - eu) < 1e-12 * eu


def test_regression_invariant_under_basis_scaling():
    # the fitted values span the same space whatever the scale of S and v, so
    # the exercise decisions are unchanged when K and theta rescale the basis:
    # compare the oracle's fit against an unscaled least-squares fit
    P, N, T = 512, 6, 1.0
    model = oracle.heston(**H)
    S, V = oracle.paths(model, T, oracle.QE, P, N, 77, 0)
    d = oracle.lsmc(S, V, 100.0, 100.0, T, 0.02, 0.04, basis=oracle.BASIS_SV2, want_detail=True)
    n = 3
    itm = S[n] < 100.0
    X = _basis(S[n][itm], V[n][itm], 100.0, 0.04, oracle.BASIS_SV2)
    Xu = _basis(S[n][itm], V[n][itm], 1.0, 1.0, oracle.BASIS_SV2, centre=0.0)
    fitted = X @ d["beta"][n]
    # regression target at date n rebuilt from the stopping times
    ex = d["exercise"]
    tau = np.full(P, N)
    for m in range(N - 1, n, -1):
        tau = np.where(ex[m] == 1, m, tau)
    Y = np.exp(-0.02 * (tau - n) * T / N) * np.maximum(100.0 - S[tau, np.arange(P)], 0.0)
    fitted_u = Xu @ np.linalg.lstsq(Xu, Y[itm], rcond=None)[0]
    assert np.allclose(fitted, fitted_u, rtol=0, atol=1e-7 * np.abs(fitted).max())


def test_american_at_least_european_and_call_without_dividends():
    model = oracle.heston(**H)
    P, N, T = 1 << 14, 32, 1.0
    S, V = oracle.paths(model, T, oracle.QE, P, N, 42, 0)
    for K in (90.0, 100.0, 110.0):
        am = oracle.lsmc(S, V, 100.0, K, T, 0.02, 0.04)
        assert am["price"] >= am["european_price"] - 3 * am["price_se"]
        c = oracle.lsmc(S, V, 100.0, K, T, 0.02, 0.04, type_=oracle.CALL)
        # no dividends: early exercise of a call is never optimal, so the
        # LSMC value can only lose to regression noise
        assert abs(c["price"] - c["european_price"]) < 3 * c["price_se"]


def test_prices_monotone_in_strike():
    model = oracle.heston(**H)
    res = oracle.price_greeks(model, [80.0, 90.0, 100.0, 110.0, 120.0], 1.0, 4096, 32,
                              basis=oracle.BASIS_SV2,
                              b=oracle.bumps(greek_mask=0))
    prices = [r["price"] for r in res]
    assert all(a < b for a, b in zip(prices, prices[1:]))
    assert all(r["n_revaluations"] == 1 for r in res)


@pytest.mark.parametrize("K", [100.0, 110.0])
def test_bermudan_put_matches_tree_when_variance_is_constant(K):
    r, sigma, T, N = 0.05, 0.2, 1.0, 32
    model = oracle.heston(**dict(H, r=r, xi=0.0, v0=sigma**2, theta=sigma**2))
    P = 1 << 16
    S, V = oracle.paths(model, T, oracle.FT_EULER, P, N, 2024, 0)
    d = oracle.lsmc(S, V, 100.0, K, T, r, sigma**2)
    tree = refs.crr_bermudan(100.0, K, T, r, 0.0, sigma, False, N, 64)
    eu = refs.bs_price(100.0, K, T, r, 0.0, sigma, False)
    assert tree > eu + 0.1  # a real early-exercise premium is being priced
    assert abs(d["price"] - tree) < 3 * d["price_se"] + 0.01 * tree, (d["price"], tree)
    assert abs(d["european_price"] - eu) < 4 * d["price_se"]


def test_european_greeks_match_black_scholes():
    r, T, N, K, kappa = 0.02, 1.0, 32, 100.0, 1.5
    sigma2 = 0.04
    model = oracle.heston(**dict(H, xi=0.0, v0=sigma2, theta=sigma2, kappa=kappa))
    b = oracle.bumps(rel_dS=0.01, rel_dS_gamma=0.02, rel_dv0=0.01, abs_dr=1e-3,
                     abs_dT=1 / 252, greek_mask=31)
    names = ["price", "delta", "gamma", "vega", "rho", "theta"]
    runs = []
    for seed in range(1, 9):
        res = oracle.price_greeks(model, [K], T, 1 << 13, N, style=oracle.EUROPEAN,
                                  scheme=oracle.FT_EULER, basis=oracle.BASIS_S2, b=b,
                                  seed=seed)[0]
        assert res["n_revaluations"] == 11
        runs.append([res[k] for k in names])
    runs = np.array(runs)
    mean, se = runs.mean(0), runs.std(0, ddof=1) / math.sqrt(len(runs))
    g = refs.bs_greeks_fd(100.0, K, T, r, 0.0, math.sqrt(sigma2), False)
    dt = T / N
    dvar_dv0 = dt * sum((1 - kappa * dt) ** k for k in range(N)) / T
    ref = dict(price=refs.bs_price(100.0, K, T, r, 0.0, 0.2, False), delta=g["delta"],
               gamma=g["gamma"], vega=g["var_vega"] * dvar_dv0, rho=g["rho"], theta=g["theta"])
    for i, k in enumerate(names):
        # Monte Carlo error plus the finite-difference truncation of the bump
        assert abs(mean[i] - ref[k]) < 4 * se[i] + 0.01 * abs(ref[k]), (k, mean[i], se[i], ref[k])


def test_american_put_greeks_have_the_right_signs_and_size():
    model = oracle.heston(**H)
    b = oracle.bumps(rel_dS=0.01, rel_dS_gamma=0.02, greek_mask=31)
    res = oracle.price_greeks(model, [90.0, 100.0, 110.0], 1.0, 1 << 13, 32,
                              basis=oracle.BASIS_SV2, b=b)
    for r_ in res:
        assert -1.0 <= r_["delta"] <= 0.0
        assert r_["gamma"] > 0.0
        assert r_["vega"] > 0.0
        assert r_["rho"] < 0.0
        assert r_["n_revaluations"] == 11
    assert res[0]["delta"] > res[1]["delta"] > res[2]["delta"]


def test_scenario_table_layouts():
    m = oracle.heston(**H)
    sc = oracle.scenarios(m, 1.0, oracle.bumps(rel_dS=0.01, rel_dS_gamma=0.01,
                                               greek_mask=oracle.DELTA | oracle.GAMMA | oracle.VEGA))
    assert [k for k, _, _ in sc] == ["base", "S+", "S-", "v0+", "v0-"]
    assert sc[1][1].S0 == 101.0 and sc[2][1].S0 == 99.0
    assert sc[3][1].v0 == 0.04 * 1.01 and sc[4][1].v0 == 0.04 * 0.99
    sc = oracle.scenarios(m, 1.0, oracle.bumps(rel_dS=0.01, rel_dS_gamma=0.02, greek_mask=31))
    assert [k for k, _, _ in sc] == ["base", "S+", "S-", "Sg+", "Sg-", "v0+", "v0-",
                                     "r+", "r-", "T-", "T+"]
    assert sc[3][1].S0 == 102.0 and sc[4][1].S0 == 98.0
    assert sc[7][1].r == 0.021 and sc[8][1].r == 0.019
    assert sc[9][2] == 1.0 - 1 / 252 and sc[10][2] == 1.0 + 1 / 252
    sc = oracle.scenarios(m, 1.0, oracle.bumps(greek_mask=oracle.GAMMA))
    assert [k for k, _, _ in sc] == ["base", "S+", "S-"]
    with pytest.raises(ValueError):
        oracle.scenarios(m, 0.003, oracle.bumps(greek_mask=oracle.THETA))
    with pytest.raises(ValueError):
        oracle.scenarios(oracle.heston(**dict(H, v0=0.0)), 1.0, oracle.bumps(greek_mask=oracle.VEGA))


def test_invalid_arguments_are_rejected():
    m = oracle.heston(**H)
    with pytest.raises(ValueError):
        oracle.paths(oracle.heston(**dict(H, xi=0.0)), 1.0, oracle.QE, 8, 4, 1)
    with pytest.raises(ValueError):
        oracle.paths(oracle.heston(**dict(H, rho=-1.5)), 1.0, oracle.QE, 8, 4, 1)
    with pytest.raises(ValueError):
        oracle.paths(m, -1.0, oracle.QE, 8, 4, 1)
    with pytest.raises(ValueError):
        oracle.price_greeks(m, [0.0], 1.0, 8, 4)
    S, V = oracle.paths(m, 1.0, oracle.QE, 8, 4, 1)
    with pytest.raises(ValueError):
        oracle.lsmc(S, V, 100.0, 100.0, 1.0, 0.02, 0.04, basis=7)


def test_results_do_not_depend_on_thread_count():
    m = oracle.heston(**H)
    kw = dict(basis=oracle.BASIS_SV2, b=oracle.bumps(rel_dS_gamma=0.02, greek_mask=31))
    a = oracle.price_greeks(m, [90.0, 100.0], 1.0, 3000, 16, n_threads=1, **kw)
    b = oracle.price_greeks(m, [90.0, 100.0], 1.0, 3000, 16, n_threads=5, **kw)
    assert a == b


def test_singular_regression_dates_do_not_exercise():
    # fewer in-the-money paths than basis functions on most dates
    m = oracle.heston(**H)
    S, V = oracle.paths(m, 1.0, oracle.QE, 16, 8, 3)
    d = oracle.lsmc(S, V, 100.0, 70.0, 1.0, 0.02, 0.04, basis=oracle.BASIS_SV2, want_detail=True)
    for n in range(1, 8):
        if (S[n] < 70.0).sum() < 6:
            assert np.isnan(d["beta"][n, 0]) and not d["exercise"][n].any()
    assert d["n_singular"] >= 1
