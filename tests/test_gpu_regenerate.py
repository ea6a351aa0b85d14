"""Regenerate mode (LSMC_FLAG_REGENERATE): no path store, states saved every
ceil(sqrt(N)) dates and each segment simulated again before its backward
rounds.  The random inputs are counter-based, so every result must be the
stored-path result bit for bit, with a fraction of the device memory."""
import json
import math
import os

import pytest

import oracle
from gpu_common import oracle_args, scenario_parity, torch_cuda
from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu


def _same(a, b):
    """Equal results, bit for bit (NaN, the Greeks not asked for, equals NaN)."""
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.keys() == y.keys()
        for k in x:
            same_nan = isinstance(x[k], float) and math.isnan(x[k]) and math.isnan(y[k])
            assert same_nan or x[k] == y[k], (k, x[k], y[k])


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    with api.Context(workspace_bytes=6 << 30) as c:
        yield c


@pytest.mark.parametrize("precision", ["fp64", "df", "mixed"])
@pytest.mark.parametrize("scheme,basis", [("qe", "sv2"), ("ft_euler", "s2")])
def test_regenerate_equals_store(ctx, precision, scheme, basis):
    wl = workloads.SMALL_FP64.replace(n_paths=5000, n_steps=50, basis=basis, scheme=scheme,
                                      greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02,
                                      strikes=[90.0, 100.0, 110.0])
    got = ctx.price(wl.replace(regenerate=True), precision=precision)
    ref = ctx.price(wl, precision=precision)
    _same(got, ref)


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("scheme,basis", [("qe", "sv2"), ("ft_euler", "s2")])
def test_regenerate_matches_oracle(ctx, precision, scheme, basis):
    # the segments simulated again from the saved states are the paths of
    # Sec. 2.2.1 (variance, log price, exponential): priced against the
    # oracle, which simulates every path once from its start
    wl = workloads.SMALL_FP64.replace(n_paths=5000, n_steps=50, basis=basis, scheme=scheme,
                                      greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02,
                                      strikes=[90.0, 100.0, 110.0], regenerate=True)
    got, scen = ctx.price_with_scenarios(wl, precision=precision)
    scenario_parity(wl, got, scen, what="regenerate %s %s" % (precision, scheme))


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("name", ["paper_fp64", "paper_fp64_ft"])
def test_regenerate_paper_size_matches_stored_oracle_values(ctx, name, precision):
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       name + ".json")))
    wl = workloads.PAPER_FP64.replace(scheme=gold["scheme"], precision=precision,
                                      regenerate=True)
    got, scen = ctx.price_with_scenarios(wl)
    model, b, _ = oracle_args(wl)
    kinds = [k for k, _, _ in oracle.scenarios(model, wl.T, b)]
    ref_scen = [[r["scenarios"][kind] for r in gold["results"]] for kind in kinds]
    scenario_parity(wl, got, scen, ref=gold["results"], ref_scen=ref_scen,
                    what="regenerate %s %s" % (name, precision))


def test_regenerate_european_and_one_segment(ctx):
    for wl in (workloads.SMALL_FP64.replace(style="european", n_steps=37),
               workloads.SMALL_FP64.replace(n_steps=1),
               workloads.SMALL_FP64.replace(n_steps=4, n_paths=333)):
        _same(ctx.price(wl.replace(regenerate=True)), ctx.price(wl))


def test_regenerate_paper_size_and_footprint(ctx):
    wl = workloads.PAPER_FP64
    need = L.lsmc_request_footprint(None, api.Request(wl).c)
    need_r = L.lsmc_request_footprint(None, api.Request(wl.replace(regenerate=True)).c)
    assert need_r < need / 4
    _same(ctx.price(wl.replace(regenerate=True)), ctx.price(wl))


def test_regenerate_rejections(ctx):
    a = workloads.SMALL_FP64.replace(regenerate=True)
    b = workloads.SMALL_FP64.replace(regenerate=True, n_steps=20)
    with pytest.raises(L.LsmcError) as e:
        ctx.price_book([a, b])
    assert e.value.status == L.LSMC_ENOTIMPL
    with pytest.raises(L.LsmcError) as e:
        ctx.price_book([a, workloads.SMALL_FP64])
    assert e.value.status == L.LSMC_ENOTIMPL
    r = api.Request(workloads.SMALL_FP64)
    r.c.flags = 16  # no such flag
    with pytest.raises(L.LsmcError) as e:
        L.lsmc_price_request(ctx.ctx, r.c)
    assert e.value.status == L.LSMC_EINVAL
