"""Pins of the oracle's near-tie report and decision reversal (CPU only).

The GPU path rounds differently from the oracle, so an exercise decision
whose payoff lies within rounding reach of the fitted continuation value may
go the other way there.  The parity tests then look for the oracle's result
with some of its near-tie decisions reversed.  These tests pin that hook to
the plain method and to a reconstruction from the stopping times:

* with no decision reversed, the hook changes nothing (bit for bit);
* reversing a decision at the first exercise date (after which no regression
  runs) moves the price by exactly that path's change of discounted cash
  flow over P, computed from the plain run's exercise matrix;
* a reported near tie satisfies |h - c| <= tie_rel max(|c|, h);
* one revaluation re-run on its own reproduces price_greeks's scenario price
  (in-sample, out of sample, 16-bit store), and its subsets of reversed
  decisions equal the backward pass run with those reversals.
"""
import itertools

import numpy as np
import pytest

import oracle

H = dict(S0=100.0, r=0.03, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


def _run(S, V, K=100.0, T=1.0, r=0.03, basis=oracle.BASIS_SV2, **kw):
    return oracle.lsmc(S, V, 100.0, K, T, r, 0.04, basis=basis, **kw)


@pytest.fixture(scope="module")
def paths():
    return oracle.paths(oracle.heston(**H), 1.0, oracle.QE, 3000, 12, 77, 3)


def test_tie_control_without_reversals_is_the_plain_method(paths):
    S, V = paths
    plain = _run(S, V)
    hooked = _run(S, V, tie_rel=1e-9)
    for k in ("price", "price_se", "european_price", "continuation", "n_singular"):
        assert hooked[k] == plain[k], k
    assert hooked["n_near_ties"] == len(hooked["near_ties"])


def _stop_value(S, ex, p, n_from, K, D, N):
    """Cash flow of path p at date n_from if it continues there: the payoff
    at its next exercise date of the plain run (else maturity), discounted to
    n_from one step at a time."""
    m = next((m for m in range(n_from + 1, N) if ex[m, p]), N)
    y = max(K - S[m, p], 0.0)
    for _ in range(m - n_from):
        y *= D
    return y


@pytest.mark.parametrize("exercised", [True, False])
def test_reversal_at_the_first_date_moves_the_price_by_one_cash_flow(paths, exercised):
    S, V = paths
    N, P, K, T, r = S.shape[0] - 1, S.shape[1], 100.0, 1.0, 0.03
    D = np.exp(-r * T / N)
    d = _run(S, V, want_detail=True)
    ex = d["exercise"]
    itm1 = S[1] < K
    cand = np.flatnonzero((ex[1] == 1) if exercised else (itm1 & (ex[1] == 0)))
    assert cand.size > 0
    p = int(cand[cand.size // 2])
    flipped = _run(S, V, flips=[1 * P + p])
    h1 = K - S[1, p]
    cont = _stop_value(S, ex, p, 1, K, D, N)
    # the estimator is mean_p D * Y_p at t_1: one path's Y changes from the
    # payoff to the continued cash flow, or the other way
    delta = D * ((cont - h1) if exercised else (h1 - cont)) / P
    assert d["price"] > 0.0 and flipped["price"] != d["price"]
    assert abs((flipped["price"] - d["price"]) - delta) <= 1e-12 * abs(d["price"])


def test_reported_near_ties_are_near_their_threshold():
    # a coarse radius makes near ties common; every reported one must sit
    # within it of the fitted value (checked against the regression rebuilt
    # from the plain run's coefficients)
    model = oracle.heston(**H)
    S, V = oracle.paths(model, 1.0, oracle.QE, 2000, 10, 5, 0)
    P, N, K, theta = S.shape[1], S.shape[0] - 1, 100.0, 0.04
    d = _run(S, V, want_detail=True)
    t = _run(S, V, tie_rel=1e-3)
    assert t["n_near_ties"] > 5
    for key in t["near_ties"]:
        n, p = divmod(int(key), P)
        assert 1 <= n < N
        s, v = S[n, p], V[n, p]
        x, w = s / K - 1.0, v / theta - 1.0
        c = float(np.dot(d["beta"][n], [1.0, x, x * x, w, x * w, w * w]))
        h = K - s
        assert h > 0.0
        # c is recomputed in another order: allow a few ulps of slack
        assert abs(h - c) <= 1e-3 * max(abs(c), h) * (1 + 1e-9) + 1e-12 * abs(c)


def _wl_args(**kw):
    a = dict(type_=oracle.PUT, style=oracle.AMERICAN, scheme=oracle.QE, basis=oracle.BASIS_SV2,
             b=oracle.bumps(rel_dS_gamma=0.02, greek_mask=31), seed=9, stream=4)
    a.update(kw)
    return a


@pytest.mark.parametrize("variant", [dict(), dict(out_of_sample=True),
                                     dict(store=oracle.STORE_F16), dict(scheme=oracle.FT_EULER)])
def test_one_revaluation_reproduces_the_scenario_price(variant):
    model = oracle.heston(**H)
    strikes = [90.0, 105.0]
    P, N, T = 1500, 9, 0.75
    a = _wl_args(**variant)
    res, scen = oracle.price_greeks(model, strikes, T, P, N, want_scenarios=True, **a)
    kinds = [k for k, _, _ in oracle.scenarios(model, T, a["b"])]
    assert len(kinds) == scen.shape[0] == 11
    for s in range(len(kinds)):
        for k, K in enumerate(strikes):
            prices, _ = oracle.scenario_alternatives(model, K, T, P, N, s, **a)
            assert prices == [scen[s, k]], (kinds[s], K)
    # the Greeks follow from the revaluations as price_greeks forms them
    for k in range(len(strikes)):
        g = oracle.greeks_from_values(model, a["b"], kinds, list(scen[:, k]))
        for key in ("price", "delta", "gamma", "vega", "rho", "theta"):
            assert g[key] == res[k][key], key


@pytest.mark.parametrize("out_of_sample", [False, True])
def test_subsets_of_reversed_decisions_equal_the_reversed_runs(out_of_sample):
    model = oracle.heston(**H)
    P, N, T, K = 1200, 8, 1.0, 100.0
    a = _wl_args(out_of_sample=out_of_sample, b=oracle.bumps(greek_mask=0))
    _, ties = oracle.scenario_alternatives(model, K, T, P, N, 0, tie_rel=2e-3, **a)
    assert len(ties) >= 3
    if out_of_sample:
        # keys of both passes occur; take some of each when there are
        pricing = [t for t in ties if t & oracle.KEY_PRICING]
        regress = [t for t in ties if not t & oracle.KEY_PRICING]
        keys = sorted(regress[:2] + pricing[:1]) if pricing and regress else sorted(ties[:3])
    else:
        keys = sorted(ties[:3])
    prices, _ = oracle.scenario_alternatives(model, K, T, P, N, 0, keys=keys, **a)
    assert len(prices) == 8
    if not out_of_sample:
        S, V = oracle.paths(model, T, oracle.QE, P, N, a["seed"], a["stream"])
        for i in range(8):
            sub = [k for j, k in enumerate(keys) if i >> j & 1]
            assert prices[i] == _run(S, V, K=K, T=T, r=H["r"], flips=sub)["price"], i
    # reversing nothing is the plain revaluation; every non-empty subset
    # changes at least one cash flow
    plain, _ = oracle.scenario_alternatives(model, K, T, P, N, 0, **a)
    assert prices[0] == plain[0]
    assert len(set(prices)) > 1
