"""Pins of the oracle's 16-bit path store (the paper's study of reduced
data types, Sec. 4.2 and Table 4, applied to the stored paths only).

* Rounding to binary16 agrees with numpy's float16 conversion on random
  doubles, on every midpoint between adjacent binary16 values (ties to even)
  and one unit in the last place either side of it, and across the
  subnormal and overflow ranges.
* Rounding to bfloat16: on float inputs it agrees with torch's bfloat16
  conversion (round to nearest even); on arbitrary doubles the result is a
  bfloat16 value no farther from the input than either neighbour, with ties
  going to the even neighbour.
* A European payoff is 1-Lipschitz in S, so rounding every stored exp(x) to
  a format with unit roundoff u moves the European price by at most
  exp(-rT) S0 u mean(exp(x_N)), a bound that holds on every path set.
* The American price moves by a fraction of its standard error (the
  rounding flips exercise decisions next to the boundary, noise of the
  in-sample policy, not a bias).
* The rate scenarios read the base simulation's stored values times
  exp(+-dr t_n) (the reading of a rate bump for a 16-bit store).
"""
import numpy as np
import pytest

import oracle

H = dict(S0=100.0, r=0.03, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)
U = {oracle.STORE_F16: 2.0 ** -11, oracle.STORE_BF16: 2.0 ** -8}


def test_binary16_rounding_matches_numpy():
    h = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float64)
    mid = (h[:-1] + h[1:]) / 2  # exact in double
    rng = np.random.default_rng(1)
    rnd = rng.choice([-1.0, 1.0], 100000) * np.exp(rng.uniform(np.log(1e-9), np.log(1e6), 100000))
    xs = np.concatenate([h, mid, -mid, np.nextafter(mid, 0.0), np.nextafter(mid, np.inf), rnd,
                         [65504.0, 65519.99, 65520.0, 1e6, 2.9e-8, 3e-8, 6e-8, 0.0, -0.0]])
    got = oracle.round_store(xs, oracle.STORE_F16)
    with np.errstate(over="ignore"):
        want = xs.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, want)
    # ties go to the even neighbour
    assert oracle.round_store(np.array([1.0 + 2.0 ** -11]), oracle.STORE_F16)[0] == 1.0
    assert oracle.round_store(np.array([1.0 + 3 * 2.0 ** -11]), oracle.STORE_F16)[0] == 1.0 + 2.0 ** -9


def test_bfloat16_rounding_matches_torch_on_floats():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x32 = (rng.choice([-1.0, 1.0], 100000) *
           np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 100000))).astype(np.float32)
    mids = ((rng.integers(0x0080, 0x7F7F, 20000).astype(np.uint32) << 16) | 0x8000).view(np.float32)
    xs = np.concatenate([x32, mids, -mids]).astype(np.float64)
    got = oracle.round_store(xs, oracle.STORE_BF16)
    want = torch.tensor(xs.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, want)


def test_bfloat16_rounding_is_nearest_with_ties_to_even():
    rng = np.random.default_rng(3)
    xs = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 50000))  # doubles, not floats
    r = oracle.round_store(xs, oracle.STORE_BF16)
    bits = r.astype(np.float32).view(np.uint32)
    assert np.array_equal(r.astype(np.float32).astype(np.float64), r)  # a float ...
    assert np.all(bits & 0xFFFF == 0)                                   # ... with 8 bits
    up = (bits + 0x10000).view(np.float32).astype(np.float64)
    dn = (bits - 0x10000).view(np.float32).astype(np.float64)
    d = np.abs(xs - r)
    assert np.all(d <= np.abs(xs - up)) and np.all(d <= np.abs(xs - dn))
    ties = (d == np.abs(xs - up)) | (d == np.abs(xs - dn))
    assert np.all((bits[ties] >> 16) & 1 == 0)


@pytest.mark.parametrize("store", [oracle.STORE_F16, oracle.STORE_BF16])
def test_european_price_within_the_rounding_bound(store):
    m = oracle.heston(**H)
    P, N, T, K = 4000, 16, 1.0, 100.0
    kw = dict(style=oracle.EUROPEAN, basis=oracle.BASIS_S2, seed=11, stream=3,
              b=oracle.bumps(greek_mask=0))
    native = oracle.price_greeks(m, [K], T, P, N, **kw)[0]["price"]
    rounded = oracle.price_greeks(m, [K], T, P, N, store=store, **kw)[0]["price"]
    unit = oracle.heston(**dict(H, S0=1.0))
    E, _ = oracle.paths(unit, T, oracle.QE, P, N, 11, 3)  # rows of exp(x)
    bound = np.exp(-H["r"] * T) * H["S0"] * U[store] * E[-1].mean()
    assert rounded != native
    assert abs(rounded - native) <= bound


@pytest.mark.parametrize("store", [oracle.STORE_F16, oracle.STORE_BF16])
def test_american_price_moves_by_a_fraction_of_its_error(store):
    m = oracle.heston(**H)
    kw = dict(basis=oracle.BASIS_SV2, seed=4, stream=1, b=oracle.bumps(greek_mask=0))
    native = oracle.price_greeks(m, [100.0], 1.0, 6000, 24, **kw)[0]
    rounded = oracle.price_greeks(m, [100.0], 1.0, 6000, 24, store=store, **kw)[0]
    # the rounding flips exercise decisions next to the boundary, each
    # flip moving its path's value by O(price): about 0.1 standard errors
    assert abs(rounded["price"] - native["price"]) < 0.5 * native["price_se"]


def test_rate_scenarios_read_the_base_rows():
    m = oracle.heston(**H)
    P, N, T, K, dr = 3000, 12, 1.0, 100.0, 1e-3
    b = oracle.bumps(abs_dr=dr, greek_mask=8)
    out, scen = oracle.price_greeks(m, [K], T, P, N, basis=oracle.BASIS_SV2, seed=6, stream=2,
                                    store=oracle.STORE_F16, b=b, want_scenarios=True)
    kinds = [k for k, _, _ in oracle.scenarios(m, T, b)]
    unit = oracle.heston(**dict(H, S0=1.0))
    E, V = oracle.paths(unit, T, oracle.QE, P, N, 6, 2)
    E16 = oracle.round_store(E, oracle.STORE_F16)
    V16 = oracle.round_store(V, oracle.STORE_F16)
    t = np.arange(N + 1)[:, None] * (T / N)
    for sign, kind in ((1.0, "r+"), (-1.0, "r-")):
        S = H["S0"] * np.exp(sign * dr * t) * E16
        ref = oracle.lsmc(S, V16, H["S0"], K, T, H["r"] + sign * dr, H["theta"],
                          basis=oracle.BASIS_SV2)
        assert scen[kinds.index(kind), 0] == ref["price"]
