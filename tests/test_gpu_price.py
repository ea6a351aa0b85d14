"""End-to-end GPU parity through the C ABI: prices and Greeks of whole
requests against the FP64 oracle on identical random streams."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from gpu_common import (KEYS, assert_close, floored_rel_err, oracle_args, oracle_for, rel_err,
                        same_results, scenario_parity, torch_cuda)
from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FP64_TOL = 1e-10      # relative, FP64 GPU path vs FP64 oracle on identical streams


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    c = api.Context(workspace_bytes=8 << 30)
    yield c
    c.close()


def test_small_american_put_matches_oracle(ctx):
    wl = workloads.SMALL_FP64
    got, scen = ctx.price_with_scenarios(wl)
    assert same_results(got, ctx.price(wl))  # the plan and the one-call path agree bit for bit
    assert got[0]["n_revaluations"] == 5
    scenario_parity(wl, got, scen, keys=("price", "delta", "gamma", "vega", "european_price"),
                    what="small")
    assert math.isnan(got[0]["rho"]) and math.isnan(got[0]["theta"])
    ref = oracle_for(wl)
    assert abs(got[0]["price_se"] - ref[0]["price_se"]) <= 1e-9 * ref[0]["price_se"]


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_price_greeks_single_contract_call_matches_oracle(ctx, prec):
    # lsmc_price_greeks: one contract, the call of the method's purpose
    # (Sec. 2.2: the Greeks); the small workload's American put with delta,
    # gamma and vega, through the context's default precision
    wl = workloads.SMALL_FP64
    with api.Context(workspace_bytes=256 << 20, precision=prec) as c2:
        m = L.lsmc_heston(**wl.model)
        con = L.lsmc_contract(L.LSMC_PUT, L.LSMC_AMERICAN, wl.strikes[0], wl.T)
        bumps = L.lsmc_bumps(wl.rel_dS, wl.rel_dS_gamma, wl.rel_dv0, wl.abs_dr, wl.abs_dT,
                             L.LSMC_GREEK_DELTA | L.LSMC_GREEK_GAMMA | L.LSMC_GREEK_VEGA, 0)
        got = L.lsmc_price_greeks(c2.ctx, m, con, wl.n_paths, wl.n_steps, L.LSMC_BASIS_S2,
                                  bumps, wl.seed).as_dict()
        # the same request through a plan gives its revaluations
        got_p, scen = c2.price_with_scenarios(wl.replace(precision=prec))
    assert same_results(got, got_p[0])
    assert got["n_revaluations"] == 5
    scenario_parity(wl, [got], scen, keys=("price", "delta", "gamma", "vega", "european_price"),
                    what="lsmc_price_greeks " + prec)


VARIANTS = [
    dict(),
    dict(scheme="ft_euler"),
    dict(option="call", model=dict(workloads.HESTON_BASE, q=0.03), strikes=[95.0, 105.0]),
    dict(style="european"),
    dict(basis="sv2", greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02),
    dict(n_paths=1000, n_steps=7, strikes=[90.0, 100.0, 111.0]),       # ragged tiles
    dict(n_paths=3001, n_steps=1),                                      # one date
    dict(n_paths=5000, n_steps=2, basis="sv2"),
    dict(n_paths=64, n_steps=12, strikes=[60.0]),                       # singular dates
    dict(scheme="ft_euler", model=dict(workloads.HESTON_BASE, xi=0.0), basis="s2"),
    dict(model=dict(workloads.HESTON_BASE, kappa=0.5, theta=0.09, xi=0.6, rho=-0.3, v0=0.01),
         greeks=workloads.ALL_GREEKS, stream=17, seed=2**63 + 5),
    # deep in the money: most paths exercise at every date, so the exercise
    # items collected over a job fill several warps (ragged, several sub-tiles)
    dict(strikes=[112.0, 116.0], n_paths=9000, n_steps=10, basis="sv2"),
]


@pytest.mark.parametrize("prec", ["fp64", "df"])
@pytest.mark.parametrize("kw", VARIANTS, ids=[str(i) for i in range(len(VARIANTS))])
def test_variants_match_oracle(ctx, kw, prec):
    wl = workloads.SMALL_FP64.replace(n_paths=4096, n_steps=24, **kw) if "n_paths" not in kw \
        else workloads.SMALL_FP64.replace(**kw)
    got, scen = ctx.price_with_scenarios(wl.replace(precision=prec))
    scenario_parity(wl, got, scen, what="%s %s" % (prec, kw))


@pytest.mark.parametrize("prec", ["fp64", "df"])
@pytest.mark.parametrize("name", ["paper_fp64", "paper_fp64_ft"])
def test_paper_size_matches_stored_oracle_values(ctx, name, prec):
    path = os.path.join(GOLDEN, name + ".json")
    gold = json.load(open(path))
    wl = workloads.PAPER_FP64.replace(scheme=gold["scheme"], precision=prec)
    assert gold["n_paths"] == wl.n_paths and gold["n_steps"] == wl.n_steps
    got, scen = ctx.price_with_scenarios(wl)
    for k, (g, r) in enumerate(zip(got, gold["results"])):
        assert g["n_revaluations"] == 11
        print("%s %s K=%g near ties %d price rel err %.3g" % (
            name, prec, wl.strikes[k], g["n_near_ties"], rel_err(g["price"], r["price"])))
    # every price and Greek at 1e-10; a revaluation with a decision taken the
    # other way at a near tie is matched by the oracle re-run with it reversed
    model, b, _ = oracle_args(wl)
    kinds = [k for k, _, _ in oracle.scenarios(model, wl.T, b)]
    ref_scen = [[r["scenarios"][kind] for r in gold["results"]] for kind in kinds]
    scenario_parity(wl, got, scen, ref=gold["results"], ref_scen=ref_scen,
                    what="%s %s" % (name, prec))


def test_graph_replay_is_bit_identical(ctx):
    wl = workloads.SMALL_FP64.replace(basis="sv2", greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02,
                                      strikes=[90.0, 100.0])
    plan = ctx.plan([wl])
    plan.launch(use_graph=False)
    a = plan.fetch()
    plan.launch(use_graph=True)
    b = plan.fetch()
    plan.launch(use_graph=True)
    c = plan.fetch()
    plan.close()
    assert a == b == c
    assert a == ctx.price(wl)


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_book_equals_requests_priced_one_by_one(ctx, prec):
    # an uneven book (puts and calls, drawn models, maturities, path and step
    # counts) in one graph-replayed launch: each result equals the request
    # priced alone, and every contract matches the oracle
    book = workloads.book(n_contracts=6, paths_hi=20000, steps=(8, 16, 33), precision=prec)
    together, scen = ctx.price_book_with_scenarios(book, use_graph=True)
    assert same_results(together, ctx.price_book(book))
    alone = [ctx.price(w)[0] for w in book]
    assert same_results(together, alone)
    for i, w in enumerate(book):
        scenario_parity(w.replace(precision="fp64"), [together[i]], [scen[i]],
                        what="book %s contract %d" % (prec, i))


# MIXED (single-precision paths on the 23-bit uniform grid) is not a 1e-4
# form: its paths differ from the FP64 ones by ~1e-6 relative, which moves
# exercise decisions near the boundary, and each moved decision changes a
# price at first order; central differences divide those moves by the bumps.
# The bounds below are the errors this form is reported with at this size
# (32,768 paths x 64 dates), with margin: the price moves by less than half
# its Monte Carlo standard error, and the European price, which has no
# decisions, stays at the single-precision path error.  A Greek's error is
# relative to itself or, where it is much smaller than the price differences
# it is made of, to price / bump denominator (as in assert_close; measured:
# at most 2e-2).
MIXED_BOUNDS = {"price": 3e-3, "european_price": 1e-5, "delta": 0.05, "gamma": 0.05,
                "vega": 0.05, "rho": 0.05, "theta": 0.05}


def test_mixed_precision_errors_against_fp64_oracle_are_within_stated_bounds(ctx):
    wl = workloads.PAPER_FP64.replace(n_paths=32768, n_steps=64, precision="mixed")
    got = ctx.price(wl)
    ref = oracle_for(wl.replace(precision="fp64"))
    worst = {}
    for g, r in zip(got, ref):
        for k in MIXED_BOUNDS:
            worst[k] = max(worst.get(k, 0.0), floored_rel_err(g, r, k))
    print("mixed vs FP64 oracle, worst relative errors:", worst)
    for k, bound in MIXED_BOUNDS.items():
        assert worst[k] <= bound, (k, worst[k], bound)
    for g, r in zip(got, ref):
        assert abs(g["price"] - r["price"]) <= 0.5 * r["price_se"]


def test_invalid_requests_are_rejected_before_launch(ctx):
    for kw in (dict(n_paths=0), dict(strikes=[float("inf")]),
               dict(model=dict(workloads.HESTON_BASE, kappa=-1.0))):
        with pytest.raises(L.LsmcError) as e:
            ctx.price(workloads.SMALL_FP64.replace(**kw))
        assert e.value.status == L.LSMC_EINVAL


def test_autotuned_plans_still_match_oracle(ctx):
    wl = workloads.SMALL_FP64.replace(n_paths=20000, n_steps=20, basis="sv2",
                                      greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02)
    sub, ppt, ms = ctx.autotune([wl])
    assert sub >= 1 and ppt in (2, 4) and ms > 0
    got, scen = ctx.price_with_scenarios(wl)
    scenario_parity(wl, got, scen, what="autotuned")
    # a fixed shape through the context option (other sums' order) matches too
    with api.Context(workspace_bytes=1 << 30) as c2:
        c2.set_backward_shape(3, 2)
        got2, scen2 = c2.price_with_scenarios(wl)
    scenario_parity(wl, got2, scen2, what="fixed shape 3 x 2")


def test_in_the_money_strikes_in_half_size_jobs_match_oracle(ctx):
    # LSMC_SUB_ITM_HALF: the strike in the money at S0 (the 110 put) runs its
    # regressions in jobs of half the sub-tiles; more jobs, the same results
    wl = workloads.SMALL_FP64.replace(n_paths=20000, n_steps=20, basis="sv2",
                                      strikes=[90.0, 100.0, 110.0],
                                      greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02)
    jobs = {}
    for name, sub in (("uniform", 4), ("itm half", 4 | L.LSMC_SUB_ITM_HALF)):
        with api.Context(workspace_bytes=1 << 30) as c:
            c.set_backward_shape(sub, 2)
            p = c.plan([wl])
            jobs[name] = p.info().backward_jobs
            p.close()
            got, scen = c.price_with_scenarios(wl)
        scenario_parity(wl, got, scen, what=name)
    assert jobs["itm half"] > jobs["uniform"]
    for bad in (L.LSMC_SUB_ITM_HALF, 65 | L.LSMC_SUB_ITM_HALF):
        with pytest.raises(L.LsmcError) as e:
            ctx.set_backward_shape(bad, 2)
        assert e.value.status == L.LSMC_EINVAL


def test_external_allocator():
    # every plan allocation through callbacks (here PyTorch's caching
    # allocator, counted): the same results as cudaMalloc, every block
    # handed back once the context is gone
    import torch
    from paper_2206_03719_gb300 import lsmc as L
    torch_cuda()
    wl = workloads.SMALL_FP64.replace(n_paths=3000, n_steps=12)
    calls = {"alloc": 0, "free": 0}

    def alloc(n):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(n)

    def release(ptr):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    with api.Context() as ref_ctx:
        ref = ref_ctx.price(wl)
    ctx = api.Context()
    keep = L.lsmc_set_allocator(ctx.ctx, alloc, release)
    got = ctx.price(wl)
    got_b = ctx.price_bounds(wl.replace(greeks=()), 32, 8)
    ctx.close()
    del keep
    def same(a, b):  # Greeks not asked for are NaN on both sides
        return all(x.keys() == y.keys() and all(
            x[k] == y[k] or (x[k] != x[k] and y[k] != y[k]) for k in x) for x, y in zip(a, b))

    assert len(got) == len(ref) and same(got, ref)
    assert got_b[0]["upper"] > 0.0
    assert calls["alloc"] >= 3 and calls["alloc"] == calls["free"]
    with api.Context(torch_allocator=True) as c2:
        assert same(c2.price(wl), ref)
