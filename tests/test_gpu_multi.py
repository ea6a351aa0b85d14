"""GPU parity of the STAC-A2 multi-asset path reduction (lsmc_multi_asset_max)
against the oracle: elementwise at sizes that span several CTAs and a ragged
tail, and on sampled paths at the paper's Huge shape (50 assets x 1260 dates
x 25,000 paths)."""
import numpy as np
import pytest

import oracle
from gpu_common import torch_cuda
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu

BASE = dict(S0=100.0, r=0.02, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)


@pytest.fixture(scope="module")
def torch():
    t = torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    L.load()
    return t


def _models(A, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for a in range(A):
        out.append(dict(S0=float(rng.uniform(80, 120)), r=0.02, q=float(rng.uniform(0, 0.03)),
                        v0=float(rng.uniform(0.01, 0.09)), kappa=float(rng.uniform(0.5, 3.0)),
                        theta=float(rng.uniform(0.02, 0.09)), xi=float(rng.uniform(0.1, 0.8)),
                        rho=float(rng.uniform(-0.9, -0.3))))
    return out


def _gpu(torch, models, T, scheme, precision, rho_assets, P, N, seed, stream):
    shape = (N + 1, P, 2) if precision == L.LSMC_DF else (N + 1, P)
    dt = torch.float64 if precision == L.LSMC_FP64 else torch.float32
    M = torch.full(shape, float("nan"), dtype=dt, device="cuda")
    L.lsmc_multi_asset_max([L.lsmc_heston(**m) for m in models], T, scheme, precision, rho_assets,
                           P, N, seed, stream, M.data_ptr())
    torch.cuda.synchronize()
    a = M.cpu().numpy()
    if precision == L.LSMC_DF:
        return a[..., 0].astype(np.float64) + a[..., 1].astype(np.float64)
    return a.astype(np.float64)


@pytest.mark.parametrize("prec", [L.LSMC_FP64, L.LSMC_DF])
@pytest.mark.parametrize("scheme", [L.LSMC_SCHEME_QE, L.LSMC_SCHEME_FT_EULER])
@pytest.mark.parametrize("rho_assets", [0.0, 0.4])
@pytest.mark.parametrize("A,P,N", [(5, 1000, 30), (1, 257, 3), (9, 129, 12)])
def test_multi_max_matches_oracle(torch, prec, scheme, rho_assets, A, P, N):
    models = _models(A, A)
    got = _gpu(torch, models, 0.75, scheme, prec, rho_assets, P, N, 77, 5)
    ref = oracle.multi_max([oracle.heston(**m) for m in models], 0.75, scheme, P, N, 77, 5,
                           rho_assets=rho_assets)
    rtol = 1e-12 if prec == L.LSMC_FP64 else 1e-11
    assert np.allclose(got, ref, rtol=rtol, atol=0)


def test_multi_max_single_precision_on_the_same_stream(torch):
    models = _models(6, 3)
    P, N = 2048, 50
    got = _gpu(torch, models, 1.0, L.LSMC_SCHEME_QE, L.LSMC_MIXED, 0.3, P, N, 9, 0)
    ref = oracle.multi_max([oracle.heston(**m) for m in models], 1.0, oracle.QE, P, N, 9, 0,
                           rho_assets=0.3, grid=oracle.GRID_F32)
    rel = np.abs(got - ref) / ref
    assert np.quantile(rel, 0.999) < 2e-5 and rel.max() < 1e-3


def test_one_asset_is_the_path_generator(torch):
    P, N = 300, 20
    got = _gpu(torch, [BASE], 1.0, L.LSMC_SCHEME_QE, L.LSMC_FP64, 0.0, P, N, 3, 1)
    S = torch.empty((N + 1, P), dtype=torch.float64, device="cuda")
    V = torch.empty_like(S)
    L.lsmc_paths(L.lsmc_heston(**BASE), 1.0, L.LSMC_SCHEME_QE, L.LSMC_FP64, P, N, 3, 1,
                 S.data_ptr(), V.data_ptr())
    torch.cuda.synchronize()
    assert np.allclose(got, S.cpu().numpy(), rtol=1e-14, atol=0)


def test_huge_shape_sampled_paths(torch):
    # the paper's Huge problem: 50 assets, 1260 dates, 25,000 paths; the
    # oracle recomputes the sampled paths asset by asset
    A, N, P = 50, 1260, 25000
    models = _models(A, 50)
    got = _gpu(torch, models, 5.0, L.LSMC_SCHEME_QE, L.LSMC_FP64, 0.0, P, N, 2022, 0)
    assert np.all(np.isfinite(got))
    for p in (0, 1, 127, 128, 12345, P - 1):
        paths = np.stack([oracle.asset_path(oracle.heston(**m), a, 5.0, oracle.QE, p, N, 2022, 0)
                          for a, m in enumerate(models)])
        assert np.allclose(got[:, p], paths.max(axis=0), rtol=1e-11, atol=0)


def test_invalid_arguments(torch):
    M = torch.empty((2, 8), dtype=torch.float64, device="cuda")
    bad = [dict(models=[BASE] * 65), dict(rho_assets=1.5), dict(rho_assets=-0.1),
           dict(models=[dict(BASE, kappa=0.0)]), dict(P=0), dict(N=0)]
    for b in bad:
        kw = dict(models=[BASE], rho_assets=0.0, P=8, N=1)
        kw.update(b)
        with pytest.raises(L.LsmcError) as e:
            L.lsmc_multi_asset_max([L.lsmc_heston(**m) for m in kw["models"]], 1.0,
                                   L.LSMC_SCHEME_QE, L.LSMC_FP64, kw["rho_assets"], kw["P"],
                                   kw["N"], 1, 0, M.data_ptr())
        assert e.value.status == L.LSMC_EINVAL


def test_longstaff_schwartz_on_the_reduced_path(torch):
    # the curve fit of the reduced path (a best-of call) is the single-asset
    # backward pass run on M, checked against the oracle's on the oracle's M
    from gpu_common import backward_parity
    models = _models(4, 11)
    P, N, T, K = 4000, 24, 1.0, 105.0
    Mo = oracle.multi_max([oracle.heston(**m) for m in models], T, oracle.QE, P, N, 5, 0)
    S0 = float(Mo[0, 0])
    model = dict(models[0], S0=S0, r=0.02)
    dS = torch.from_numpy(Mo).cuda()
    dV = torch.zeros_like(dS)
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    c = L.lsmc_contract(L.LSMC_CALL, L.LSMC_AMERICAN, K, T)
    L.lsmc_backward(dS.data_ptr(), dV.data_ptr(), P, N, L.LSMC_FP64, L.lsmc_heston(**model), c,
                    L.LSMC_BASIS_S2, out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    backward_parity(got, Mo, np.zeros_like(Mo), S0, K, T, 0.02, model["theta"],
                    type_=oracle.CALL, style=oracle.AMERICAN, basis=oracle.BASIS_S2,
                    what="best-of call")
    assert got[0] >= got[2] - 1e-12  # American >= European
