"""The stored expected values of tests/golden/ are what the oracle computes
now: the cheapest contracts of the book and serving subsets are priced
again by the script's own oracle call and must give the stored prices and
Greeks, and one revaluation of each paper-size file its stored price.  A change of the oracle's arithmetic, or of the seeded workload
generator, that leaves the stored files behind fails here on the CPU
instead of as a GPU parity failure."""
import importlib.util
import json
import math
import os

import pytest

from paper_2206_03719_gb300 import workloads

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
KEYS = ("price", "price_se", "european_price", "delta", "gamma", "vega", "rho", "theta")


@pytest.fixture(scope="module")
def make_golden():
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(HERE, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _same(a, b):
    if a is None or b is None:
        return a is None and b is None
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    # the same code on the same inputs; the libm of another machine may
    # round an elementary function differently in the last place
    return abs(a - b) <= 1e-12 * max(abs(b), 1e-300)


@pytest.mark.parametrize("subset", ["book_subset", "serving_subset"])
def test_cheapest_stored_contracts_reproduce(make_golden, subset):
    stored = json.load(open(os.path.join(HERE, subset + ".json")))
    wls = make_golden.SUBSETS[subset]()
    assert [w.name for w in wls] == [c["name"] for c in stored["contracts"]]
    order = sorted(range(len(wls)), key=lambda i: wls[i].n_paths * wls[i].n_steps)
    for i in order[:2]:
        got = make_golden.run_oracle(wls[i])[0][0]
        want = stored["contracts"][i]["results"]
        for k in KEYS:
            if k in want:
                assert _same(got[k], want[k]), (wls[i].name, k, got[k], want[k])


@pytest.mark.parametrize("name, wl, k, kind", [
    ("paper_fp64", workloads.PAPER_FP64, 2, "base"),
    ("paper_fp64_ft", workloads.PAPER_FP64.replace(scheme="ft_euler"), 4, "v0+"),
])
def test_one_paper_size_revaluation_reproduces(name, wl, k, kind):
    # one revaluation of one strike of the 131,072 x 252 book, as the
    # oracle's Greeks use it, against the stored scenario price
    import oracle
    from gpu_common import oracle_args
    stored = json.load(open(os.path.join(HERE, name + ".json")))
    assert stored["strikes"] == wl.strikes and stored["scheme"] == wl.scheme
    m, b, kw = oracle_args(wl)
    kinds = [kd for kd, _, _ in oracle.scenarios(m, wl.T, b)]
    prices, _ = oracle.scenario_alternatives(
        m, wl.strikes[k], wl.T, wl.n_paths, wl.n_steps, kinds.index(kind), type_=kw["type_"],
        style=kw["style"], scheme=kw["scheme"], basis=kw["basis"], b=b, seed=kw["seed"],
        stream=kw["stream"])
    assert _same(prices[0], stored["results"][k]["scenarios"][kind])


def test_stored_subsets_name_the_generator_contracts(make_golden):
    book = workloads.book(n_contracts=512)
    stored = json.load(open(os.path.join(HERE, "book_subset.json")))
    assert stored["indices"] == make_golden.BOOK_SUBSET
    assert [c["name"] for c in stored["contracts"]] == [book[i].name for i in stored["indices"]]
