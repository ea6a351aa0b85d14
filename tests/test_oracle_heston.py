"""Pins of the oracle's Heston discretisations (CPU only).

QE variance step: Andersen's scheme matches the first two conditional moments
of the CIR variance exactly in both branches; those moments come from scipy's
noncentral chi-square law.  QE log-price step: as xi -> 0 with v0 = theta it
must reduce to a Black-Scholes log increment with correlated normals.
FT-Euler: xi = 0 gives a deterministic Euler variance and GBM increments.
Prices: European prices from oracle paths against the Heston Fourier price.
"""
import math

import numpy as np
import pytest

import oracle
import refs

H = dict(S0=100.0, r=0.02, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


def _qe_psi(v, dt, kappa, theta, xi):
    m, s2 = refs.cir_moments(v, dt, kappa, theta, xi)
    return m, s2, s2 / (m * m)


@pytest.mark.parametrize("v,dt,kappa,theta,xi", [
    (0.04, 1 / 252, 1.5, 0.04, 0.3),
    (0.09, 0.05, 0.5, 0.02, 0.6),
    (0.01, 0.1, 3.0, 0.09, 0.4),
])
def test_qe_quadratic_branch_matches_cir_moments(v, dt, kappa, theta, xi):
    m, s2, psi = _qe_psi(v, dt, kappa, theta, xi)
    assert psi <= 1.5
    model = oracle.heston(**dict(H, kappa=kappa, theta=theta, xi=xi))
    z, w = np.polynomial.hermite_e.hermegauss(30)
    w = w / w.sum()
    v1 = np.array([oracle.qe_step(model, dt, 0.0, v, 0.5, zi, 0.0)[1] for zi in z])
    mean = (w * v1).sum()
    var = (w * v1 * v1).sum() - mean * mean
    assert abs(mean / m - 1) < 1e-12
    assert abs(var / s2 - 1) < 1e-9


@pytest.mark.parametrize("v,dt,kappa,theta,xi", [
    (1e-4, 0.25, 1.5, 0.04, 0.6),
    (0.0, 0.02, 0.5, 0.02, 0.6),
    (0.002, 0.5, 1.0, 0.03, 0.5),
])
def test_qe_exponential_branch_matches_cir_moments(v, dt, kappa, theta, xi):
    m, s2, psi = _qe_psi(v, dt, kappa, theta, xi)
    assert psi > 1.5
    p = (psi - 1) / (psi + 1)
    model = oracle.heston(**dict(H, kappa=kappa, theta=theta, xi=xi))
    # below the atom's probability the draw is exactly zero
    for u in np.linspace(1e-9, p * (1 - 1e-9), 50):
        assert oracle.qe_step(model, dt, 0.0, v, u, 0.0, 0.0)[1] == 0.0
    # above it: u = 1 - (1 - p) e^{-y}, y ~ Exp(1); Gauss-Laguerre in y
    # v1 is linear in y, so three nodes integrate v1 and v1^2 exactly
    y, w = np.polynomial.laguerre.laggauss(3)
    u = 1.0 - (1.0 - p) * np.exp(-y)
    v1 = np.array([oracle.qe_step(model, dt, 0.0, v, ui, 0.0, 0.0)[1] for ui in u])
    e1 = (1 - p) * (w * v1).sum()
    e2 = (1 - p) * (w * v1 * v1).sum()
    assert abs(e1 / m - 1) < 1e-9
    assert abs((e2 - e1 * e1) / s2 - 1) < 1e-8


@pytest.mark.parametrize("rho", [-0.7, 0.0, 0.5])
def test_qe_log_step_reduces_to_bs_increment_as_xi_vanishes(rho):
    dt, theta = 1 / 252, 0.04
    z = np.random.default_rng(5).standard_normal((64, 2))
    errs = []
    for xi in (1e-4, 1e-5):
        model = oracle.heston(**dict(H, xi=xi, rho=rho, v0=theta, theta=theta, q=0.01))
        e = 0.0
        for zv, zx in z:
            x1, v1 = oracle.qe_step(model, dt, 0.3, theta, 0.5, zv, zx)
            ref = 0.3 + (0.02 - 0.01 - 0.5 * theta) * dt + math.sqrt(theta * dt) * (
                rho * zv + math.sqrt(1 - rho * rho) * zx)
            e = max(e, abs(x1 - ref))
        errs.append(e)
    assert errs[1] < 1e-6
    # the remainder is O(xi): ten times smaller xi, about ten times smaller error
    assert errs[1] < errs[0] / 5 or errs[0] < 1e-9


def test_ft_euler_xi_zero_is_euler_variance_and_gbm():
    model = oracle.heston(**dict(H, xi=0.0, v0=0.06, theta=0.04, kappa=2.0, q=0.01))
    P, N, T, seed, stream = 64, 40, 0.75, 11, 3
    S, V = oracle.paths(model, T, oracle.FT_EULER, P, N, seed, stream)
    dt = T / N
    vn = 0.04 + (0.06 - 0.04) * (1 - 2.0 * dt) ** np.arange(N + 1)
    assert np.allclose(V, vn[:, None], rtol=1e-13, atol=0)
    pp, nn = np.meshgrid(np.arange(P), np.arange(N))
    d = oracle.draws(seed, stream, pp.ravel(), nn.ravel()).reshape(N, P, 3)
    rho = H["rho"]
    inc = (0.02 - 0.01 - 0.5 * vn[:N, None]) * dt + np.sqrt(vn[:N, None] * dt) * (
        rho * d[:, :, 1] + math.sqrt(1 - rho * rho) * d[:, :, 2])
    x = np.vstack([np.zeros((1, P)), np.cumsum(inc, axis=0)])
    assert np.allclose(S, 100.0 * np.exp(x), rtol=1e-12, atol=0)


def test_ft_euler_truncates_negative_variance():
    model = oracle.heston(**H)
    dt = 0.01
    x1, v1, v1p = oracle.ft_step(model, dt, 0.1, -0.02, 1.3, -0.4)
    assert v1 == -0.02 + 1.5 * 0.04 * dt      # no diffusion, drift on v+ = 0
    assert x1 == 0.1 + 0.02 * dt
    assert v1p == max(v1, 0.0)
    x1, v1, v1p = oracle.ft_step(model, dt, 0.0, 0.001, -3.0, 0.0)
    assert v1 < 0 and v1p == 0.0


def test_qe_martingale_within_error():
    model = oracle.heston(**H)
    P, N, T = 1 << 15, 50, 1.0
    S, _ = oracle.paths(model, T, oracle.QE, P, N, 99, 0)
    ST = S[-1]
    se = ST.std(ddof=1) / math.sqrt(P)
    assert abs(ST.mean() - 100.0 * math.exp(0.02 * T)) < 4 * se


@pytest.mark.parametrize("scheme,N", [(oracle.QE, 64), (oracle.FT_EULER, 252)])
def test_european_put_matches_heston_fourier_price(scheme, N):
    model = oracle.heston(**H)
    P, T = 1 << 16, 1.0
    S, V = oracle.paths(model, T, scheme, P, N, 42, 1)
    for K in (90.0, 100.0, 110.0):
        ref = refs.heston_price(100.0, K, T, 0.02, 0.0, 0.04, 1.5, 0.04, 0.3, -0.7, call=False)
        r = oracle.lsmc(S, V, 100.0, K, T, 0.02, 0.04, style=oracle.EUROPEAN)
        # discretisation bias allowance: 0.5% (QE, 64 steps) / 1% (Euler)
        bias = (0.005 if scheme == oracle.QE else 0.01) * ref
        assert abs(r["price"] - ref) < 4 * r["price_se"] + bias, (K, r["price"], ref, r["price_se"])


def test_heston_mean_log_price_within_error():
    model = oracle.heston(**dict(H, v0=0.09, theta=0.03, kappa=2.0, xi=0.5, rho=-0.4))
    P, N, T = 1 << 15, 100, 1.0
    S, _ = oracle.paths(model, T, oracle.QE, P, N, 5, 0)
    lx = np.log(S[-1])
    se = lx.std(ddof=1) / math.sqrt(P)
    ref = refs.heston_mean_log(100.0, 0.02, 0.0, T, 0.09, 2.0, 0.03)
    assert abs(lx.mean() - ref) < 4 * se + 2e-3


@pytest.mark.parametrize("scheme", [oracle.QE, oracle.FT_EULER])
def test_spot_and_rate_move_paths_by_known_factors(scheme):
    # In the Heston model the variance does not depend on S0, r or q, and the
    # log price relative to its start moves by (r - q) t: on common random
    # numbers a spot bump scales every path value by (1 + h) and a rate bump
    # by exp(dr t_n), with the variance paths unchanged.  (These are the facts
    # that let the spot and rate revaluations share the base simulation.)
    T, P, N, h, dr = 1.0, 64, 24, 0.01, 1e-3
    base = oracle.heston(**H)
    S, V = oracle.paths(base, T, scheme, P, N, 42, n_threads=1)
    Ss, Vs = oracle.paths(oracle.heston(**dict(H, S0=H["S0"] * (1 + h))), T, scheme, P, N, 42,
                          n_threads=1)
    Sr, Vr = oracle.paths(oracle.heston(**dict(H, r=H["r"] + dr)), T, scheme, P, N, 42,
                          n_threads=1)
    assert np.array_equal(V, Vs) and np.array_equal(V, Vr)
    np.testing.assert_allclose(Ss / S, 1 + h, rtol=1e-14, atol=0)
    t = (np.arange(N + 1) * (T / N))[:, None]
    np.testing.assert_allclose(np.log(Sr / S), dr * t * np.ones_like(S), rtol=0, atol=1e-13)


@pytest.mark.parametrize("grid", [oracle.GRID_F64, oracle.GRID_F32])
@pytest.mark.parametrize("scheme", [oracle.QE, oracle.FT_EULER])
def test_path_one_is_the_column_of_the_path_matrix(scheme, grid):
    # orc_path_one (the reference of the sampled full-size path checks) must
    # give column p of orc_paths bit for bit: same draws, same steps, the
    # stored variance truncated the same way
    model = oracle.heston(**dict(H, xi=0.6, kappa=0.8, v0=0.02, theta=0.05))
    P, N, T, seed, stream = 2051, 40, 1.5, 2**40 + 9, 7
    S, V = oracle.paths(model, T, scheme, P, N, seed, stream, grid=grid)
    rng = np.random.default_rng(5)
    for p in [0, 1, 1023, 1024, P - 1] + list(rng.integers(0, P, 6)):
        s1, v1 = oracle.path_one(model, T, scheme, int(p), N, seed, stream, grid=grid)
        assert np.array_equal(s1, S[:, p]), p
        assert np.array_equal(v1, V[:, p]), p
    if scheme == oracle.FT_EULER:
        assert (V >= 0).all()
