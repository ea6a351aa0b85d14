"""16-bit path store (LSMC_FLAG_STORE_FP16 / LSMC_FLAG_STORE_BF16) on the GPU
against the oracle's 16-bit store: exp(x) and v rounded to nearest even when
written, widened exactly when read, every step computed in the request's
precision.  Identical rounded inputs on both sides, so the parity bound is
the one of the full-precision store."""
import math

import pytest

from gpu_common import oracle_for, scenario_parity, torch_cuda
from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu


def _same(a, b):
    """Equal results, bit for bit (NaN, the Greeks not asked for, equals NaN)."""
    assert len(a) == len(b)
    for x, y in zip(a, b):
        for k in x:
            same_nan = isinstance(x[k], float) and math.isnan(x[k]) and math.isnan(y[k])
            assert same_nan or x[k] == y[k], (k, x[k], y[k])


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    with api.Context(workspace_bytes=4 << 30) as c:
        yield c


def _wl(**kw):
    return workloads.SMALL_FP64.replace(n_paths=6000, n_steps=24, basis="sv2",
                                        greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02,
                                        strikes=[90.0, 100.0, 112.0]).replace(**kw)


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("store", ["fp16", "bf16"])
def test_store16_matches_oracle(ctx, precision, store):
    wl = _wl(store=store)
    got, scen = ctx.price_with_scenarios(wl, precision=precision)
    scenario_parity(wl, got, scen, what="%s/%s" % (precision, store))


@pytest.mark.parametrize("store", ["fp16", "bf16"])
def test_store16_call_s2_ft_euler(ctx, store):
    wl = _wl(store=store, option="call", basis="s2", scheme="ft_euler", n_paths=4500,
             model=dict(workloads.SMALL_FP64.model, q=0.03))
    got, scen = ctx.price_with_scenarios(wl)
    scenario_parity(wl, got, scen, what='test_gpu_store16.py')


def test_store16_out_of_sample_matches_oracle(ctx):
    wl = _wl(store="fp16", out_of_sample=True)
    got, scen = ctx.price_with_scenarios(wl)
    scenario_parity(wl, got, scen, what='test_gpu_store16.py')


@pytest.mark.parametrize("precision", ["fp64", "df", "mixed"])
def test_store16_regenerate_equals_store16(ctx, precision):
    wl = _wl(store="fp16", n_steps=40, n_paths=3000)
    _same(ctx.price(wl.replace(regenerate=True), precision=precision),
          ctx.price(wl, precision=precision))


def test_store16_mixed_close_to_fp64(ctx):
    wl = _wl(store="fp16", n_paths=20000, greeks=())
    a = ctx.price(wl, precision="mixed")
    b = ctx.price(wl, precision="fp64")
    for x, y in zip(a, b):
        assert abs(x["price"] - y["price"]) < 0.3 * y["price_se"]


def test_store16_footprint(ctx):
    wl = workloads.PAPER_FP64
    need = L.lsmc_request_footprint(None, api.Request(wl).c)
    need16 = L.lsmc_request_footprint(None, api.Request(wl.replace(store="fp16")).c)
    rows = wl.n_paths * wl.n_steps * 5 * 2  # E and V rows of the 5 path groups
    assert need - need16 >= 0.99 * rows * (8 - 2)


def test_store16_flag_rules(ctx):
    r = api.Request(workloads.SMALL_FP64)
    r.c.flags = L.LSMC_FLAG_STORE_FP16 | L.LSMC_FLAG_STORE_BF16
    with pytest.raises(L.LsmcError) as e:
        L.lsmc_price_request(ctx.ctx, r.c)
    assert e.value.status == L.LSMC_EINVAL
    with pytest.raises(L.LsmcError) as e:
        ctx.price_book([workloads.SMALL_FP64.replace(store="fp16"), workloads.SMALL_FP64])
    assert e.value.status == L.LSMC_ENOTIMPL


@pytest.mark.parametrize("store", ["fp16", "bf16"])
@pytest.mark.parametrize("n_paths,n_steps,style", [(33, 5, "american"), (1000, 1, "american"),
                                                   (4097, 9, "european")])
def test_store16_edge_sizes(ctx, store, n_paths, n_steps, style):
    wl = _wl(store=store, n_paths=n_paths, n_steps=n_steps, style=style, strikes=[97.0])
    got, scen = ctx.price_with_scenarios(wl)
    scenario_parity(wl, got, scen, what='test_gpu_store16.py')
