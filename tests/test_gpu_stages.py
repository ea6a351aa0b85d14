"""GPU parity of each stage, through the C ABI, against the FP64 oracle:
Philox integers (bit-exact), uniform grids (bit-exact), normal quantiles,
Heston paths, and the Longstaff-Schwartz backward pass on oracle paths."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from gpu_common import backward_parity, torch_cuda
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu

H = dict(S0=100.0, r=0.02, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


@pytest.fixture(scope="module")
def torch():
    t = torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    L.load()
    return t


@pytest.mark.parametrize("n", [1, 255, 100003])
def test_philox_bit_exact(torch, n):
    rng = np.random.default_rng(n)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = [0, 0, 0, 0]
    if n > 1:
        ctr[-1] = [0xFFFFFFFF] * 4
    key = (0x9E3779B9, 0x01234567)
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    d_out = torch.empty_like(d_ctr)
    L.lsmc_philox(d_ctr.data_ptr(), key[0], key[1], d_out.data_ptr(), n)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().view(np.uint32)
    ref = oracle.philox(ctr, np.array(key, dtype=np.uint32))
    assert np.array_equal(got, ref)


def test_philox_empty_launch_is_a_no_op(torch):
    L.lsmc_philox(None, 1, 2, None, 0)


def _pairs(n, seed=0):
    rng = np.random.default_rng(seed)
    path = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    step = rng.integers(0, 600, size=n).astype(np.uint32)
    path[:4] = [0, 1, 131071, 0xFFFFFFFF]
    return path, step


def test_draws_fp64_grid_exact_quantiles_close(torch):
    n = 50001
    path, step = _pairs(n)
    d_path = torch.from_numpy(path.view(np.int32)).cuda()
    d_step = torch.from_numpy(step.view(np.int32)).cuda()
    out = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    L.lsmc_draws(0xABCDEF0123456789, 5, d_path.data_ptr(), d_step.data_ptr(), n, L.LSMC_FP64,
                 out.data_ptr())
    got = out.cpu().numpy()
    ref = oracle.draws(0xABCDEF0123456789, 5, path, step, oracle.GRID_F64)
    assert np.array_equal(got[:, 0], ref[:, 0])
    err = np.abs(got[:, 1:] - ref[:, 1:])
    # quantile: the table-driven logarithm and polynomial quantile
    # (norm_quantile_f64) against the oracle's Newton root of erfc
    assert np.all(err <= 4e-15 * np.maximum(1.0, np.abs(ref[:, 1:])))


def test_draws_pairs_are_the_fp64_draws(torch):
    n = 20001
    path, step = _pairs(n, 2)
    d_path = torch.from_numpy(path.view(np.int32)).cuda()
    d_step = torch.from_numpy(step.view(np.int32)).cuda()
    out = torch.empty((n, 3, 2), dtype=torch.float32, device="cuda")
    L.lsmc_draws(77, 4, d_path.data_ptr(), d_step.data_ptr(), n, L.LSMC_DF, out.data_ptr())
    got = _pairs_to_f64(out.cpu().numpy())
    ref = oracle.draws(77, 4, path, step, oracle.GRID_F64)
    err = np.abs(got - ref)
    assert np.all(err <= 2e-14 * np.maximum(1.0, np.abs(ref)))


def test_draws_fp32_grid_exact_quantiles_close(torch):
    n = 50001
    path, step = _pairs(n, 1)
    d_path = torch.from_numpy(path.view(np.int32)).cuda()
    d_step = torch.from_numpy(step.view(np.int32)).cuda()
    out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    L.lsmc_draws(42, 0, d_path.data_ptr(), d_step.data_ptr(), n, L.LSMC_MIXED, out.data_ptr())
    got = out.cpu().numpy().astype(np.float64)
    ref = oracle.draws(42, 0, path, step, oracle.GRID_F32)
    assert np.array_equal(got[:, 0], ref[:, 0])
    err = np.abs(got[:, 1:] - ref[:, 1:])
    assert np.all(err <= 2e-6 * np.maximum(1.0, np.abs(ref[:, 1:])))


def _pairs_to_f64(a):
    """(..., 2) float32 pairs (hi, lo) -> float64 hi + lo."""
    return a[..., 0].astype(np.float64) + a[..., 1].astype(np.float64)


def _f64_to_pairs(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return np.stack([hi, lo], axis=-1)


def _gpu_paths(torch, model, T, scheme, precision, P, N, seed, stream_id):
    shape = (N + 1, P, 2) if precision == L.LSMC_DF else (N + 1, P)
    dt = torch.float64 if precision == L.LSMC_FP64 else torch.float32
    S = torch.full(shape, float("nan"), dtype=dt, device="cuda")
    V = torch.full(shape, float("nan"), dtype=dt, device="cuda")
    L.lsmc_paths(L.lsmc_heston(**model), T, scheme, precision, P, N, seed, stream_id,
                 S.data_ptr(), V.data_ptr())
    torch.cuda.synchronize()
    if precision == L.LSMC_DF:
        return _pairs_to_f64(S.cpu().numpy()), _pairs_to_f64(V.cpu().numpy())
    return S.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", [L.LSMC_FP64, L.LSMC_DF])
@pytest.mark.parametrize("scheme", [L.LSMC_SCHEME_QE, L.LSMC_SCHEME_FT_EULER])
@pytest.mark.parametrize("P,N", [(1000, 40), (257, 3), (1, 1)])
def test_paths_fp64_and_pairs_match_oracle(torch, prec, scheme, P, N):
    model = dict(H, xi=0.5, v0=0.02)  # both QE branches are visited
    S, V = _gpu_paths(torch, model, 0.75, scheme, prec, P, N, 7, 3)
    So, Vo = oracle.paths(oracle.heston(**model), 0.75, scheme, P, N, 7, 3)
    # float pairs carry about 48 bits
    rtol_s, rtol_v = (1e-12, 1e-11) if prec == L.LSMC_FP64 else (1e-11, 1e-10)
    assert np.allclose(S, So, rtol=rtol_s, atol=0)
    assert np.allclose(V, Vo, rtol=rtol_v, atol=1e-14)


@pytest.mark.parametrize("scheme", [L.LSMC_SCHEME_QE, L.LSMC_SCHEME_FT_EULER])
def test_paths_fp32_match_oracle_on_the_same_stream(torch, scheme):
    P, N = 2048, 64
    model = dict(H, xi=0.5, v0=0.02)
    S, V = _gpu_paths(torch, model, 1.0, scheme, L.LSMC_MIXED, P, N, 11, 0)
    So, Vo = oracle.paths(oracle.heston(**model), 1.0, scheme, P, N, 11, 0, grid=oracle.GRID_F32)
    rel = np.abs(S - So) / So
    assert np.quantile(rel, 0.999) < 2e-5 and rel.max() < 1e-3
    assert np.quantile(np.abs(V - Vo), 0.999) < 2e-6


def _backward(torch, S, V, precision, model, K, T, type_, style, basis):
    N, P = S.shape[0] - 1, S.shape[1]
    if precision == L.LSMC_DF:
        dS = torch.from_numpy(_f64_to_pairs(S)).cuda()
        dV = torch.from_numpy(_f64_to_pairs(V)).cuda()
    else:
        dt = torch.float64 if precision == L.LSMC_FP64 else torch.float32
        dS = torch.from_numpy(S).to(dt).cuda()
        dV = torch.from_numpy(V).to(dt).cuda()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    beta = torch.zeros((N, 6), dtype=torch.float64, device="cuda")
    ns = torch.zeros(1, dtype=torch.int32, device="cuda")
    c = L.lsmc_contract(type_, style, K, T)
    L.lsmc_backward(dS.data_ptr(), dV.data_ptr(), P, N, precision, L.lsmc_heston(**model), c,
                    basis, out.data_ptr(), beta.data_ptr(), ns.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy(), beta.cpu().numpy(), int(ns.cpu().numpy()[0])


@pytest.mark.parametrize("prec", [L.LSMC_FP64, L.LSMC_DF])
@pytest.mark.parametrize("basis", [L.LSMC_BASIS_S2, L.LSMC_BASIS_SV2])
@pytest.mark.parametrize("type_,K", [(L.LSMC_PUT, 100.0), (L.LSMC_CALL, 95.0), (L.LSMC_PUT, 70.0)])
@pytest.mark.parametrize("style", [L.LSMC_AMERICAN, L.LSMC_EUROPEAN])
def test_backward_fp64_and_pairs_match_oracle_on_oracle_paths(torch, prec, basis, type_, K, style):
    model = dict(H, q=0.01)
    P, N, T = 3000, 20, 1.0
    S, V = oracle.paths(oracle.heston(**model), T, oracle.QE, P, N, 99, 0)
    if prec == L.LSMC_DF:  # the oracle sees the paths the pairs hold
        S = _pairs_to_f64(_f64_to_pairs(S))
        V = _pairs_to_f64(_f64_to_pairs(V))
    got, beta, ns = _backward(torch, S, V, prec, model, K, T, type_, style, basis)
    ref = oracle.lsmc(S, V, 100.0, K, T, model["r"], model["theta"], type_=type_, style=style,
                      basis=basis, want_detail=True)
    # price, its standard error, European price and continuation value at
    # 1e-10 (against the oracle with near-tie decisions reversed where the
    # GPU took them the other way)
    backward_parity(got, S, V, 100.0, K, T, model["r"], model["theta"], type_=type_,
                    style=style, basis=basis, what="backward %d" % prec)
    if style == L.LSMC_AMERICAN:
        assert ns == ref["n_singular"]
        rb = ref["beta"]
        assert np.array_equal(np.isnan(beta[1:, 0]), np.isnan(rb[1:, 0]))
        ok = ~np.isnan(rb[1:, 0])
        scale = np.abs(rb[1:][ok]).max() if ok.any() else 1.0
        assert np.allclose(beta[1:][ok], rb[1:][ok], rtol=0, atol=(1e-6 if prec == L.LSMC_FP64 else 1e-4) * scale)


@pytest.mark.parametrize("basis", [L.LSMC_BASIS_S2, L.LSMC_BASIS_SV2])
def test_backward_mixed_matches_oracle_on_fp32_paths(torch, basis):
    model = dict(H)
    P, N, T = 8192, 32, 1.0
    S, V = oracle.paths(oracle.heston(**model), T, oracle.QE, P, N, 5, 0)
    S32 = S.astype(np.float32).astype(np.float64)
    V32 = V.astype(np.float32).astype(np.float64)
    got, _, _ = _backward(torch, S32, V32, L.LSMC_MIXED, model, 100.0, T, L.LSMC_PUT,
                          L.LSMC_AMERICAN, basis)
    ref = oracle.lsmc(S32, V32, 100.0, 100.0, T, model["r"], model["theta"], basis=basis)
    err = abs(got[0] - ref["price"]) / ref["price"]
    print("mixed backward on identical FP32 paths: price rel err %.3g" % err)
    assert err <= 1e-5
    assert abs(got[2] - ref["european_price"]) <= 1e-6 * ref["european_price"]
