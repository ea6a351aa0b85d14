"""Pins for the textbook references of tests/refs.py (CPU only)."""
import math

import numpy as np
import pytest

import refs


def test_bs_put_call_parity_and_known_limits():
    S, K, T, r, q, s = 100.0, 95.0, 0.7, 0.03, 0.01, 0.25
    c = refs.bs_price(S, K, T, r, q, s, True)
    p = refs.bs_price(S, K, T, r, q, s, False)
    assert abs(c - p - (S * math.exp(-q * T) - K * math.exp(-r * T))) < 1e-12
    # deep in the money call tends to the discounted forward intrinsic
    assert abs(refs.bs_price(S, 1e-6, T, r, q, s, True) - S * math.exp(-q * T)) < 1e-6


def test_crr_european_converges_to_bs():
    S, K, T, r, q, s = 100.0, 100.0, 1.0, 0.02, 0.0, 0.2
    bs = refs.bs_price(S, K, T, r, q, s, False)
    tree = refs.crr_bermudan(S, K, T, r, q, s, False, 1, 4000, american=False)
    assert abs(tree - bs) < 2e-3


def test_crr_american_put_premium_and_call_no_premium():
    S, K, T, r, q, s = 100.0, 100.0, 1.0, 0.05, 0.0, 0.2
    eu_put = refs.crr_bermudan(S, K, T, r, q, s, False, 1, 2000, american=False)
    am_put = refs.crr_bermudan(S, K, T, r, q, s, False, 50, 40)
    assert am_put > eu_put + 0.1
    eu_call = refs.crr_bermudan(S, K, T, r, q, s, True, 1, 2000, american=False)
    am_call = refs.crr_bermudan(S, K, T, r, q, s, True, 50, 40)
    assert abs(am_call - eu_call) < 1e-9


P = dict(S0=100.0, r=0.02, q=0.0, T=1.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


def test_heston_cf_normalisation_and_martingale():
    a = (P["S0"], P["r"], P["q"], P["T"], P["v0"], P["kappa"], P["theta"], P["xi"], P["rho"])
    assert abs(refs.heston_cf(0.0, *a) - 1.0) < 1e-14
    # E[S_T] = S0 exp((r - q) T)
    assert abs(refs.heston_cf(-1j, *a).real - P["S0"] * math.exp(P["r"] * P["T"])) < 1e-9


def test_heston_cf_first_cumulant():
    a = (P["S0"], P["r"], P["q"], P["T"], P["v0"], P["kappa"], P["theta"], P["xi"], P["rho"])
    h = 1e-5
    dphi = (refs.heston_cf(h, *a) - refs.heston_cf(-h, *a)) / (2 * h)
    mean_log = (dphi / 1j).real
    ref = refs.heston_mean_log(P["S0"], P["r"], P["q"], P["T"], P["v0"], P["kappa"], P["theta"])
    assert abs(mean_log - ref) < 1e-8
    # and with v0 != theta, where the mean depends on kappa
    a2 = (P["S0"], P["r"], P["q"], P["T"], 0.09, 2.0, 0.03, 0.5, -0.4)
    dphi = (refs.heston_cf(h, *a2) - refs.heston_cf(-h, *a2)) / (2 * h)
    assert abs((dphi / 1j).real - refs.heston_mean_log(100.0, 0.02, 0.0, 1.0, 0.09, 2.0, 0.03)) < 1e-8


def test_heston_price_black_scholes_limit():
    # xi -> 0 with v0 = theta and rho = 0: constant variance theta; the
    # Heston correction is second order in xi
    for K in (80.0, 100.0, 120.0):
        h = refs.heston_price(100.0, K, 1.0, 0.02, 0.0, 0.04, 1.5, 0.04, 1e-3, 0.0, call=False)
        b = refs.bs_price(100.0, K, 1.0, 0.02, 0.0, 0.2, False)
        assert abs(h - b) < 2e-5, (K, h, b)
    # with rho != 0 the correction is first order in xi: it shrinks tenfold
    # when xi does
    d = [refs.heston_price(100.0, 120.0, 1.0, 0.02, 0.0, 0.04, 1.5, 0.04, xi, -0.7, call=False)
         - refs.bs_price(100.0, 120.0, 1.0, 0.02, 0.0, 0.2, False) for xi in (1e-2, 1e-3)]
    assert 8.0 < d[0] / d[1] < 12.0
    # v0 != theta: deterministic variance path, BS with its time average
    v0, th, kp, T = 0.09, 0.03, 2.0, 0.8
    iv = th * T + (v0 - th) * (1 - math.exp(-kp * T)) / kp
    h = refs.heston_price(100.0, 100.0, T, 0.01, 0.0, v0, kp, th, 1e-3, 0.0, call=True)
    b = refs.bs_price(100.0, 100.0, T, 0.01, 0.0, math.sqrt(iv / T), True)
    assert abs(h - b) < 2e-5


def test_heston_negative_rho_skew_orders_implied_vols():
    # negative correlation makes low-strike puts dearer than the BS price at
    # the ATM variance, and high-strike calls cheaper
    lo = refs.heston_price(100.0, 80.0, 1.0, 0.0, 0.0, 0.04, 1.5, 0.04, 0.5, -0.7, call=False)
    hi = refs.heston_price(100.0, 120.0, 1.0, 0.0, 0.0, 0.04, 1.5, 0.04, 0.5, -0.7, call=True)
    assert lo > refs.bs_price(100.0, 80.0, 1.0, 0.0, 0.0, 0.2, False)
    assert hi < refs.bs_price(100.0, 120.0, 1.0, 0.0, 0.0, 0.2, True)


def test_cir_moments_match_direct_sampling_limits():
    # small dt: mean ~ v + kappa (theta - v) dt, var ~ xi^2 v dt
    m, v = refs.cir_moments(0.05, 1e-6, 1.5, 0.04, 0.3)
    assert abs(m - (0.05 + 1.5 * (0.04 - 0.05) * 1e-6)) < 1e-12
    assert abs(v / (0.09 * 0.05 * 1e-6) - 1.0) < 1e-4
    # long horizon: stationary Gamma law, mean theta, var theta xi^2 / (2 kappa)
    m, v = refs.cir_moments(0.05, 50.0, 1.5, 0.04, 0.3)
    assert abs(m - 0.04) < 1e-12
    assert abs(v - 0.04 * 0.09 / 3.0) < 1e-12
