"""Parity at the full 131,072 x 252 size of the FP64 paper workload, on
outputs the oracle computes one by one (sampled paths) and on the backward
pass run over the oracle's own paths (one scenario, all five strikes)."""
import numpy as np
import pytest

import oracle
from gpu_common import backward_parity, torch_cuda
from paper_2206_03719_gb300 import lsmc as L
from paper_2206_03719_gb300 import workloads

pytestmark = pytest.mark.gpu
WL = workloads.PAPER_FP64


@pytest.fixture(scope="module")
def torch():
    t = torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    return t


@pytest.mark.parametrize("scheme", [L.LSMC_SCHEME_QE, L.LSMC_SCHEME_FT_EULER])
def test_sampled_full_size_paths_match_oracle(torch, scheme):
    P, N = WL.n_paths, WL.n_steps
    S = torch.empty((N + 1, P), dtype=torch.float64, device="cuda")
    V = torch.empty((N + 1, P), dtype=torch.float64, device="cuda")
    L.lsmc_paths(L.lsmc_heston(**WL.model), WL.T, scheme, L.LSMC_FP64, P, N, WL.seed, WL.stream,
                 S.data_ptr(), V.data_ptr())
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = np.concatenate([[0, 1, P - 1], rng.integers(0, P, 300)])
    cols = torch.from_numpy(idx).cuda()
    Sg = S[:, cols].cpu().numpy()
    Vg = V[:, cols].cpu().numpy()
    m = oracle.heston(**WL.model)
    worst_s = worst_v = 0.0
    for j, p in enumerate(idx):
        So, Vo = oracle.path_one(m, WL.T, scheme, int(p), N, WL.seed, WL.stream)
        worst_s = max(worst_s, float(np.max(np.abs(Sg[:, j] - So) / So)))
        worst_v = max(worst_v, float(np.max(np.abs(Vg[:, j] - Vo) / np.maximum(Vo, 1e-3))))
    print("full-size paths: worst rel S %.3g, worst V %.3g" % (worst_s, worst_v))
    assert worst_s < 1e-11 and worst_v < 1e-10


@pytest.mark.parametrize("scheme", [oracle.QE, oracle.FT_EULER])
def test_full_size_backward_on_oracle_paths(torch, scheme):
    P, N = WL.n_paths, WL.n_steps
    m = oracle.heston(**WL.model)
    So, Vo = oracle.paths(m, WL.T, scheme, P, N, WL.seed, WL.stream)
    dS = torch.from_numpy(So).cuda()
    dV = torch.from_numpy(Vo).cuda()
    for K in WL.strikes:
        out = torch.zeros(5, dtype=torch.float64, device="cuda")
        c = L.lsmc_contract(L.LSMC_PUT, L.LSMC_AMERICAN, K, WL.T)
        L.lsmc_backward(dS.data_ptr(), dV.data_ptr(), P, N, L.LSMC_FP64, L.lsmc_heston(**WL.model),
                        c, L.LSMC_BASIS_SV2, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = backward_parity(got, So, Vo, WL.model["S0"], K, WL.T, WL.model["r"],
                              WL.model["theta"], basis=oracle.BASIS_SV2, what="full size")
        e = abs(got[0] - ref["price"]) / ref["price"]
        print("K=%g price gpu %.15g oracle %.15g rel %.3g near ties %d" % (
            K, got[0], ref["price"], e, int(got[4])))
        assert abs(got[2] - ref["european_price"]) <= 1e-12 * ref["european_price"]
