"""Helpers shared by the GPU parity tests."""
import math

import numpy as np
import pytest

import oracle
from paper_2206_03719_gb300 import workloads

_GREEK = {"delta": oracle.DELTA, "gamma": oracle.GAMMA, "vega": oracle.VEGA,
          "rho": oracle.RHO, "theta": oracle.THETA}
KEYS = ("price", "delta", "gamma", "vega", "rho", "theta", "european_price")


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def oracle_args(wl, grid=oracle.GRID_F64):
    """(model, bumps, keyword arguments) of the oracle's pricing of wl."""
    mask = 0
    for g in wl.greeks:
        mask |= _GREEK[g]
    b = oracle.bumps(rel_dS=wl.rel_dS, rel_dS_gamma=wl.rel_dS_gamma, rel_dv0=wl.rel_dv0,
                     abs_dr=wl.abs_dr, abs_dT=wl.abs_dT, greek_mask=mask)
    kw = dict(type_=oracle.PUT if wl.option == "put" else oracle.CALL,
              style=oracle.AMERICAN if wl.style == "american" else oracle.EUROPEAN,
              scheme=oracle.QE if wl.scheme == "qe" else oracle.FT_EULER, grid=grid,
              basis=oracle.BASIS_S2 if wl.basis == "s2" else oracle.BASIS_SV2, b=b,
              seed=wl.seed, stream=wl.stream, out_of_sample=wl.out_of_sample,
              store={"native": oracle.STORE_NATIVE, "fp16": oracle.STORE_F16,
                     "bf16": oracle.STORE_BF16}[wl.store])
    return oracle.heston(**wl.model), b, kw


def oracle_for(wl, grid=oracle.GRID_F64, n_threads=None, want_scenarios=False):
    m, _, kw = oracle_args(wl, grid)
    return oracle.price_greeks(m, wl.strikes, wl.T, wl.n_paths, wl.n_steps,
                               n_threads=n_threads, want_scenarios=want_scenarios, **kw)


FP64_TOL = 1e-10     # FP64 GPU vs FP64 oracle on identical streams
# The oracle's near-tie radius.  The GPU counts a decision as a near tie
# when |hd - c| < 2^-32 max(|c|, hd) (at most 2.3e-10 relative); a decision
# farther from its threshold than this radius is taken the same way by any
# correct rounding of the arithmetic, whose results agree to ~1e-13.
TIE_REL = 1e-9


def _close(a, b, tol):
    if math.isnan(a) and math.isnan(b):
        return True
    return abs(a - b) <= tol * max(abs(b), 1e-12)


def scenario_parity(wl, got, scen, ref=None, ref_scen=None, tol=FP64_TOL, keys=None, what=""):
    """GPU results of workload wl against the FP64 oracle on identical
    random streams, revaluation by revaluation.

    got: the GPU's results per strike; scen: its revaluations per strike
    ({scenario kind: (price, near ties)}, Plan.fetch_scenarios).  Each
    revaluation's price must equal the oracle's within tol; where it does not,
    the GPU took a decision that lay within rounding reach of its threshold
    the other way, and its price must then equal the oracle's with some of the
    oracle's near-tie decisions (|h - c| <= TIE_REL max(|c|, h)) of that
    revaluation reversed (all subsets are tried; the oracle re-simulates that
    revaluation alone).  The price and Greeks must equal the oracle's Greeks
    of the revaluations so matched, within tol.  ref / ref_scen: the oracle's
    results and scenario prices (ref_scen[s][k]: scenario s, strike k) when
    already at hand.  Returns the reversals used, as (strike, kind, keys)."""
    model, b, kw = oracle_args(wl)
    if ref is None:
        ref, ref_scen = oracle_for(wl, want_scenarios=True)
    kinds = [k for k, _, _ in oracle.scenarios(model, wl.T, b)]
    keys = keys or (["price", "european_price"] + list(wl.greeks))
    used = []
    for k, K in enumerate(wl.strikes):
        assert set(scen[k]) == set(kinds), (what, sorted(scen[k]), kinds)
        vals = []
        for s, kind in enumerate(kinds):
            g, r = scen[k][kind][0], float(ref_scen[s][k])
            if _close(g, r, tol):
                vals.append(r)
                continue
            _, ties = oracle.scenario_alternatives(model, K, wl.T, wl.n_paths, wl.n_steps, s,
                                                   tie_rel=TIE_REL, **kw)
            assert 0 < len(ties) <= oracle.MAX_ALT_KEYS, (
                "%s K=%g %s: gpu %.15g oracle %.15g (rel %.3g) with %d oracle near ties" % (
                    what, K, kind, g, r, abs(g - r) / abs(r), len(ties)))
            alts, _ = oracle.scenario_alternatives(model, K, wl.T, wl.n_paths, wl.n_steps, s,
                                                   keys=ties, **kw)
            hit = [i for i, v in enumerate(alts) if _close(g, v, tol)]
            assert hit, ("%s K=%g %s: gpu %.15g matches none of the %d oracle results with "
                         "near ties reversed" % (what, K, kind, g, len(alts)))
            sub = [t for j, t in enumerate(sorted(ties)) if hit[0] >> j & 1]
            used.append((K, kind, sub))
            vals.append(alts[hit[0]])
        exp = dict(ref[k])
        if any(u[0] == K for u in used):
            g = oracle.greeks_from_values(model, b, kinds, vals)
            exp.update({x: g[x] for x in ("price", "delta", "gamma", "vega", "rho", "theta")})
        assert_close(got[k], exp, tol, keys=keys, what="%s K=%g" % (what, K))
        if "n_singular" in exp:
            assert got[k]["n_singular_solves"] == exp["n_singular"], (what, K)
        assert got[k]["n_revaluations"] == len(kinds)
    if used:
        print("%s: revaluations matched with reversed near ties: %s" % (what, used))
    return used


def backward_parity(got, S, V, S0, K, T, r, theta, type_=oracle.PUT, style=oracle.AMERICAN,
                    basis=oracle.BASIS_S2, tol=FP64_TOL, what=""):
    """lsmc_backward's outputs (price, price_se, european price, continuation)
    against oracle.lsmc on the same paths, or, where near-tie decisions went
    the other way, against the oracle's run with a subset of its near-tie
    decisions reversed.  Returns the oracle result matched."""
    names = ("price", "price_se", "european_price", "continuation")
    ref = oracle.lsmc(S, V, S0, K, T, r, theta, type_=type_, style=style, basis=basis,
                      tie_rel=TIE_REL)

    def ok(x):
        return all(_close(float(got[i]), x[n], tol) for i, n in enumerate(names))

    if ok(ref):
        return ref
    ties = sorted(ref["near_ties"])
    assert 0 < len(ties) <= oracle.MAX_ALT_KEYS, (
        "%s K=%g: gpu %s oracle %s with %d oracle near ties" % (
            what, K, list(got[:4]), [ref[n] for n in names], len(ties)))
    for i in range(1, 1 << len(ties)):
        sub = [t for j, t in enumerate(ties) if i >> j & 1]
        alt = oracle.lsmc(S, V, S0, K, T, r, theta, type_=type_, style=style, basis=basis,
                          flips=sub)
        if ok(alt):
            print("%s K=%g: matched with reversed near ties %s" % (what, K, sub))
            return alt
    raise AssertionError("%s K=%g: gpu %s matches no oracle result with near ties reversed"
                         % (what, K, list(got[:4])))


def same_results(a, b):
    """Result dicts (or lists of them) equal bit for bit, NaN (a Greek not
    asked for) equal to NaN."""
    if isinstance(a, list):
        return len(a) == len(b) and all(same_results(x, y) for x, y in zip(a, b))
    return a.keys() == b.keys() and all(
        a[k] == b[k] or (isinstance(a[k], float) and a[k] != a[k] and b[k] != b[k]) for k in a)


def rel_err(a, b):
    """|a - b| / max(|b|, 1e-12); NaN on both sides counts as equal."""
    if math.isnan(b) and math.isnan(a):
        return 0.0
    return abs(a - b) / max(abs(b), 1e-12)


# central-difference denominators of the Greeks for 1% / 2% S bumps, 1% v0,
# 1e-3 r and 1/252 T bumps with S0 = 100, v0 = 0.04: rounding noise of the
# scenario prices, divided by these, is the floor below which a Greek
# difference carries no information
_DENOM = {"delta": 2.0, "gamma": 1.0, "vega": 8e-4, "rho": 2e-3, "theta": 2.0 / 252}


def floored_rel_err(got, ref, k):
    """Relative error of result key k; a Greek relative to itself or, when it
    is much smaller than the price differences it is made of, to price /
    its bump denominator.  NaN on both sides counts as equal."""
    if math.isnan(got[k]) and math.isnan(ref[k]):
        return 0.0
    floor = max(abs(ref.get("price", 1.0)), 1e-2) / _DENOM.get(k, 1.0)
    return abs(got[k] - ref[k]) / max(abs(ref[k]), floor)


def assert_close(got, ref, tol, keys=KEYS, what=""):
    errs = {}
    for k in keys:
        e = floored_rel_err(got, ref, k)
        errs[k] = e
        assert e <= tol, "%s %s: got %.15g ref %.15g rel %.3g" % (what, k, got[k], ref[k], e)
    return errs
