"""Independent textbook references used to pin the oracle.

None of these shares code with the oracle or the CUDA path:
  * Black-Scholes-Merton prices (closed form, scipy's normal CDF);
  * a Cox-Ross-Rubinstein binomial tree whose early exercise is restricted to
    a given set of dates (Bermudan), and may also exercise at t = 0;
  * the Heston (1993) European price by Fourier inversion of the
    characteristic function of ln S_T, in the rotation-free form of
    Albrecher, Mayer, Schoutens and Tistaert (2007), integrated by
    scipy.integrate.quad;
  * conditional moments of the CIR variance process through scipy's
    noncentral chi-square distribution.
Each is itself pinned in tests/test_refs.py.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, stats


def bs_price(S, K, T, r, q, sigma, call):
    if sigma <= 0.0 or T <= 0.0:
        fwd = S * math.exp(-q * T) - K * math.exp(-r * T)
        return max(fwd, 0.0) if call else max(-fwd, 0.0)
    sd = sigma * math.sqrt(T)
    d1 = (math.log(S / K) + (r - q + 0.5 * sigma * sigma) * T) / sd
    d2 = d1 - sd
    if call:
        return S * math.exp(-q * T) * stats.norm.cdf(d1) - K * math.exp(-r * T) * stats.norm.cdf(d2)
    return K * math.exp(-r * T) * stats.norm.cdf(-d2) - S * math.exp(-q * T) * stats.norm.cdf(-d1)


def bs_greeks_fd(S, K, T, r, q, sigma, call, h=1e-4):
    """Delta, gamma, d/d(sigma^2) (variance vega), rho and -dV/dT of the
    closed form, by central differences of the closed form itself."""
    f = lambda **kw: bs_price(**{**dict(S=S, K=K, T=T, r=r, q=q, sigma=sigma, call=call), **kw})
    dS = S * h
    delta = (f(S=S + dS) - f(S=S - dS)) / (2 * dS)
    gamma = (f(S=S + dS) - 2 * f() + f(S=S - dS)) / (dS * dS)
    v = sigma * sigma
    dv = v * h
    vvega = (f(sigma=math.sqrt(v + dv)) - f(sigma=math.sqrt(v - dv))) / (2 * dv)
    rho = (f(r=r + h) - f(r=r - h)) / (2 * h)
    theta = (f(T=T - h) - f(T=T + h)) / (2 * h)
    return dict(delta=delta, gamma=gamma, var_vega=vvega, rho=rho, theta=theta)


def crr_bermudan(S, K, T, r, q, sigma, call, n_dates, steps_per_date,
                 exercise_at_zero=True, american=True):
    """CRR tree with exercise allowed only at t_n = n T / n_dates,
    n = 1..n_dates (and at t = 0 if exercise_at_zero).  With american=False
    no early exercise at all (European)."""
    M = n_dates * steps_per_date
    dt = T / M
    u = math.exp(sigma * math.sqrt(dt))
    d = 1.0 / u
    p = (math.exp((r - q) * dt) - d) / (u - d)
    disc = math.exp(-r * dt)
    j = np.arange(M + 1)
    ST = S * u ** (M - 2 * j)
    V = np.maximum(ST - K, 0.0) if call else np.maximum(K - ST, 0.0)
    for i in range(M - 1, -1, -1):
        V = disc * (p * V[:-1] + (1 - p) * V[1:])
        if american and (i % steps_per_date == 0) and (i > 0 or exercise_at_zero):
            Si = S * u ** (i - 2 * np.arange(i + 1))
            h = np.maximum(Si - K, 0.0) if call else np.maximum(K - Si, 0.0)
            V = np.maximum(V, h)
    return float(V[0])


def heston_cf(u, S0, r, q, T, v0, kappa, theta, xi, rho):
    """E[exp(i u ln S_T)] for complex u."""
    u = np.asarray(u, dtype=complex)
    iu = 1j * u
    beta = kappa - rho * xi * iu
    d = np.sqrt(beta * beta + xi * xi * (iu + u * u))
    g = (beta - d) / (beta + d)
    e = np.exp(-d * T)
    C = (r - q) * iu * T + (kappa * theta / (xi * xi)) * (
        (beta - d) * T - 2.0 * np.log((1.0 - g * e) / (1.0 - g)))
    D = ((beta - d) / (xi * xi)) * (1.0 - e) / (1.0 - g * e)
    return np.exp(C + D * v0 + iu * math.log(S0))


def heston_price(S0, K, T, r, q, v0, kappa, theta, xi, rho, call=True):
    args = (S0, r, q, T, v0, kappa, theta, xi, rho)
    lnK = math.log(K)
    phi_mi = heston_cf(-1j, *args)

    def f1(u):
        return (np.exp(-1j * u * lnK) * heston_cf(u - 1j, *args) / (1j * u * phi_mi)).real

    def f2(u):
        return (np.exp(-1j * u * lnK) * heston_cf(u, *args) / (1j * u)).real

    I1 = integrate.quad(f1, 0.0, np.inf, limit=2000, epsabs=1e-12, epsrel=1e-11)[0]
    I2 = integrate.quad(f2, 0.0, np.inf, limit=2000, epsabs=1e-12, epsrel=1e-11)[0]
    P1 = 0.5 + I1 / math.pi
    P2 = 0.5 + I2 / math.pi
    c = S0 * math.exp(-q * T) * P1 - K * math.exp(-r * T) * P2
    if call:
        return c
    return c - S0 * math.exp(-q * T) + K * math.exp(-r * T)


def heston_mean_log(S0, r, q, T, v0, kappa, theta):
    """E[ln S_T] = ln S0 + (r - q) T - (1/2) int_0^T E[v_t] dt."""
    iv = theta * T + (v0 - theta) * (1.0 - math.exp(-kappa * T)) / kappa
    return math.log(S0) + (r - q) * T - 0.5 * iv


def cir_moments(v, dt, kappa, theta, xi):
    """Mean and variance of v(t+dt) given v(t) = v for the CIR process
    dv = kappa (theta - v) dt + xi sqrt(v) dW: a scaled noncentral
    chi-square with 4 kappa theta / xi^2 degrees of freedom."""
    c = xi * xi * (1.0 - math.exp(-kappa * dt)) / (4.0 * kappa)
    df = 4.0 * kappa * theta / (xi * xi)
    nc = v * math.exp(-kappa * dt) / c
    mean, var = stats.ncx2.stats(df, nc, moments="mv")
    return float(c * mean), float(c * c * var)
