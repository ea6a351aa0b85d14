"""Out-of-sample Longstaff-Schwartz (LSMC_FLAG_OUT_OF_SAMPLE) on the GPU
against the oracle's out-of-sample estimator: regressions on the request's
stream, the policy priced on stream ^ 0x80000000."""
import pytest

from gpu_common import oracle_for, scenario_parity, torch_cuda
from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import lsmc as L
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    with api.Context(workspace_bytes=4 << 30) as c:
        yield c


def _oracle_oos(wl):
    mask = 0
    for g in wl.greeks:
        mask |= {"delta": oracle.DELTA, "gamma": oracle.GAMMA, "vega": oracle.VEGA,
                 "rho": oracle.RHO, "theta": oracle.THETA}[g]
    b = oracle.bumps(rel_dS=wl.rel_dS, rel_dS_gamma=wl.rel_dS_gamma, rel_dv0=wl.rel_dv0,
                     abs_dr=wl.abs_dr, abs_dT=wl.abs_dT, greek_mask=mask)
    return oracle.price_greeks(
        oracle.heston(**wl.model), wl.strikes, wl.T, wl.n_paths, wl.n_steps,
        type_=oracle.PUT if wl.option == "put" else oracle.CALL,
        style=oracle.AMERICAN if wl.style == "american" else oracle.EUROPEAN,
        scheme=oracle.QE if wl.scheme == "qe" else oracle.FT_EULER,
        basis=oracle.BASIS_S2 if wl.basis == "s2" else oracle.BASIS_SV2, b=b, seed=wl.seed,
        stream=wl.stream, out_of_sample=True)


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("basis", ["s2", "sv2"])
def test_out_of_sample_matches_oracle(ctx, precision, basis):
    wl = workloads.SMALL_FP64.replace(n_paths=6000, n_steps=24, basis=basis,
                                      greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02,
                                      strikes=[90.0, 100.0, 112.0], out_of_sample=True)
    got, scen = ctx.price_with_scenarios(wl, precision=precision)
    scenario_parity(wl, got, scen, what=precision)


def test_out_of_sample_european_and_against_in_sample(ctx):
    wl = workloads.SMALL_FP64.replace(n_paths=20000, n_steps=16, out_of_sample=True)
    eu = wl.replace(style="european")
    got_eu = ctx.price(eu)[0]
    ref_eu = _oracle_oos(eu)[0]
    assert abs(got_eu["price"] - ref_eu["price"]) <= 1e-10 * ref_eu["price"]
    oos = ctx.price(wl)[0]
    ins = ctx.price(wl.replace(out_of_sample=False))[0]
    assert oos["price"] != ins["price"]
    assert abs(oos["price"] - ins["price"]) < 5 * (oos["price_se"] + ins["price_se"])


def test_out_of_sample_flag_rules(ctx):
    with pytest.raises(L.LsmcError) as e:
        ctx.price(workloads.SMALL_FP64.replace(out_of_sample=True, regenerate=True))
    assert e.value.status == L.LSMC_ENOTIMPL
    with pytest.raises(L.LsmcError) as e:
        ctx.price_book([workloads.SMALL_FP64.replace(out_of_sample=True), workloads.SMALL_FP64])
    assert e.value.status == L.LSMC_ENOTIMPL


@pytest.mark.parametrize("n_paths,n_steps", [(31, 6), (1025, 1), (2049, 3)])
def test_out_of_sample_edge_sizes(ctx, n_paths, n_steps):
    # fewer paths than a warp, a single date (no exercise before maturity),
    # a pricing tile of one path
    wl = workloads.SMALL_FP64.replace(n_paths=n_paths, n_steps=n_steps, basis="sv2",
                                      greeks=("delta",), strikes=[96.0, 103.0],
                                      out_of_sample=True)
    got, scen = ctx.price_with_scenarios(wl)
    scenario_parity(wl, got, scen, what='test_gpu_oos.py')
