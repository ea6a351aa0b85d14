"""Dual (Andersen-Broadie) upper bound, lsmc_price_bounds, on the GPU against
the oracle's orc_dual_bound on identical streams: the same outer paths
(pricing stream), the same inner paths (counter (j, m, stream ^ 0x40000000,
1 + p N + n)) and the same policy, so lower bound, upper bound and the
martingale's mean at maturity agree to rounding unless an exercise decision
fell within rounding reach of its threshold."""
import pytest

from gpu_common import torch_cuda
from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import lsmc as L
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    with api.Context(workspace_bytes=2 << 30) as c:
        yield c


def _oracle(wl, n_outer, n_inner):
    return oracle.dual_bound(
        oracle.heston(**wl.model), wl.strikes, wl.T, wl.n_paths, wl.n_steps, n_outer, n_inner,
        type_=oracle.PUT if wl.option == "put" else oracle.CALL,
        scheme=oracle.QE if wl.scheme == "qe" else oracle.FT_EULER,
        basis=oracle.BASIS_S2 if wl.basis == "s2" else oracle.BASIS_SV2, seed=wl.seed,
        stream=wl.stream)


def _check(got, ref):
    for g, r in zip(got, ref):
        tol = 1e-10 if g["n_near_ties"] == 0 else 1e-4
        scale = max(abs(r["lower"]), 1e-2)
        for gk, rk in (("lower", "lower"), ("upper", "upper"), ("upper_se", "upper_se"),
                       ("martingale_end", "pi_N")):
            assert abs(g[gk] - r[rk]) <= tol * max(abs(r[rk]), scale), (gk, g[gk], r[rk])
        assert g["upper"] >= g["lower"] - 3.0 * (g["upper_se"] + g["lower_se"])


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("basis", ["s2", "sv2"])
def test_dual_bound_matches_oracle(ctx, precision, basis):
    wl = workloads.SMALL_FP64.replace(n_paths=4000, n_steps=16, basis=basis, greeks=(),
                                      strikes=[90.0, 100.0, 112.0], stream=3)
    got = ctx.price_bounds(wl, 64, 96, precision=precision)
    _check(got, _oracle(wl, 64, 96))


def test_dual_bound_call_full_truncation(ctx):
    wl = workloads.SMALL_FP64.replace(n_paths=3000, n_steps=12, basis="sv2", greeks=(),
                                      option="call", scheme="ft_euler", strikes=[95.0, 105.0],
                                      model=dict(workloads.SMALL_FP64.model, q=0.04), seed=9)
    got = ctx.price_bounds(wl, 50, 130)  # inner paths over two CTA passes
    _check(got, _oracle(wl, 50, 130))


def test_dual_bound_mixed_runs_and_brackets(ctx):
    wl = workloads.SMALL_FP64.replace(n_paths=20000, n_steps=16, basis="sv2", greeks=(),
                                      strikes=[100.0])
    b = ctx.price_bounds(wl, 256, 64, precision="mixed")[0]
    ref = ctx.price_bounds(wl, 256, 64, precision="fp64")[0]
    assert abs(b["upper"] - ref["upper"]) < 0.05 * ref["upper"]
    assert b["upper"] > b["lower"] - 3.0 * (b["upper_se"] + b["lower_se"])


def test_dual_bound_rejections(ctx):
    wl = workloads.SMALL_FP64
    for bad in (dict(wl=wl.replace(style="european"), n_outer=16),
                dict(wl=wl, n_outer=wl.n_paths + 1),
                dict(wl=wl, n_outer=0),
                dict(wl=wl.replace(strikes=[100.0 + i for i in range(17)]), n_outer=16)):
        with pytest.raises(L.LsmcError) as e:
            ctx.price_bounds(bad["wl"], bad["n_outer"], 8)
        assert e.value.status == L.LSMC_EINVAL
    with pytest.raises(L.LsmcError) as e:
        ctx.price_bounds(wl.replace(regenerate=True), 16, 8)
    assert e.value.status == L.LSMC_ENOTIMPL


@pytest.mark.parametrize("n_steps,n_outer,n_inner", [(1, 5, 3), (2, 1, 1), (7, 33, 129)])
def test_dual_bound_edge_sizes(ctx, n_steps, n_outer, n_inner):
    # one date (no regression: the policy never exercises early), one outer or
    # inner path, ragged outer and inner counts
    wl = workloads.SMALL_FP64.replace(n_paths=777, n_steps=n_steps, basis="sv2", greeks=(),
                                      strikes=[95.0, 104.0])
    got = ctx.price_bounds(wl, n_outer, n_inner)
    ref = _oracle(wl, n_outer, n_inner)
    for g, r in zip(got, ref):
        tol = 1e-10 if g["n_near_ties"] == 0 else 1e-4
        scale = max(abs(r["lower"]), 1e-2)
        for gk, rk in (("lower", "lower"), ("upper", "upper"), ("martingale_end", "pi_N")):
            assert abs(g[gk] - r[rk]) <= tol * max(abs(r[rk]), scale), (gk, g[gk], r[rk])


def test_dual_bound_with_a_16_bit_store(ctx):
    # the lower bound prices on the 16-bit rows (the out-of-sample price of
    # the same request), the dual pass re-simulates its outer paths in full
    wl = workloads.SMALL_FP64.replace(n_paths=3000, n_steps=12, basis="sv2", greeks=(),
                                      strikes=[100.0], store="fp16")
    b = ctx.price_bounds(wl, 64, 32)[0]
    oos = ctx.price(wl.replace(out_of_sample=True))[0]
    assert b["lower"] == oos["price"]
    ref = _oracle(wl.replace(store="native"), 64, 32)[0]
    assert abs(b["upper"] - ref["upper"]) < 0.05 * ref["upper"]


def test_dual_bound_sixteen_strikes(ctx):
    # the largest strike count of one call: every strike's rule on the same
    # inner paths, shared-memory sums of 16 strikes per thread
    wl = workloads.SMALL_FP64.replace(n_paths=2000, n_steps=6, basis="s2", greeks=(),
                                      strikes=[84.0 + 2.0 * i for i in range(16)])
    got = ctx.price_bounds(wl, 40, 20)
    _check(got, _oracle(wl, 40, 20))
