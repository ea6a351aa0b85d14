"""lsmc_backward_noalloc: the backward pass for callers that cannot allocate
device memory (its scratch lives in a fixed array inside the library).  It
must give the results of lsmc_backward on the same paths, call after call.

Named to be collected last, so a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

from gpu_common import torch_cuda
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu

H = dict(S0=100.0, r=0.02, q=0.0, v0=0.04, kappa=1.5, theta=0.04, xi=0.3, rho=-0.7)
TOL = 1e-10  # relative, as for every FP64 parity check of these tests


@pytest.fixture(scope="module")
def torch():
    t = torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    L.load()
    return t


def _paths(torch, model, P, N, precision, seed):
    dt = torch.float64 if precision == L.LSMC_FP64 else torch.float32
    S = torch.empty((N + 1, P), dtype=dt, device="cuda")
    V = torch.empty((N + 1, P), dtype=dt, device="cuda")
    L.lsmc_paths(L.lsmc_heston(**model), 1.0, L.LSMC_SCHEME_QE, precision, P, N, seed, 0,
                 S.data_ptr(), V.data_ptr())
    return S, V


def _run(torch, fn, S, V, P, N, precision, model, K, basis):
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    beta = torch.zeros((N, 6), dtype=torch.float64, device="cuda")
    ns = torch.zeros(1, dtype=torch.int32, device="cuda")
    c = L.lsmc_contract(L.LSMC_PUT, L.LSMC_AMERICAN, K, 1.0)
    fn(S.data_ptr(), V.data_ptr(), P, N, precision, L.lsmc_heston(**model), c, basis,
       out.data_ptr(), beta.data_ptr(), ns.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy(), beta.cpu().numpy(), int(ns.cpu().numpy()[0])


def _same(a, b):
    (oa, ba, na), (ob, bb, nb) = a, b
    assert na == nb
    assert np.all(np.abs(oa - ob) <= TOL * np.abs(ob))
    assert np.array_equal(np.isnan(ba), np.isnan(bb))
    ok = ~np.isnan(bb)
    assert np.all(np.abs(ba[ok] - bb[ok]) <= TOL * np.abs(bb[ok]).max())


def test_noalloc_matches_allocating_backward_on_two_calls_in_a_row(torch):
    cases = [
        (dict(H), 30000, 40, L.LSMC_FP64, 100.0, L.LSMC_BASIS_SV2, 11),
        (dict(H, xi=0.5, v0=0.09), 5000, 17, L.LSMC_FP64, 110.0, L.LSMC_BASIS_S2, 12),
        (dict(H), 20000, 24, L.LSMC_MIXED, 95.0, L.LSMC_BASIS_SV2, 13),
    ]
    for model, P, N, prec, K, basis, seed in cases:
        S, V = _paths(torch, model, P, N, prec, seed)
        n0 = L.lsmc_device_allocations()
        ref = _run(torch, L.lsmc_backward, S, V, P, N, prec, model, K, basis)
        n1 = L.lsmc_device_allocations()
        first = _run(torch, L.lsmc_backward_noalloc, S, V, P, N, prec, model, K, basis)
        second = _run(torch, L.lsmc_backward_noalloc, S, V, P, N, prec, model, K, basis)
        n2 = L.lsmc_device_allocations()
        _same(first, ref)
        _same(second, ref)
        assert ref[0][0] > 0
        # the allocating pass is seen by the library's allocation count; the
        # two calls without allocation leave it where it was
        assert n1 > n0
        assert n2 == n1


def test_noalloc_rejects_requests_beyond_its_scratch(torch):
    # 4M paths need 32 MiB of cash flows, more than the 16 MiB scratch: the
    # call must refuse before launching anything (real buffers are passed so
    # that nothing could read out of bounds even if it did launch)
    P, N = 1 << 22, 1
    S = torch.full((N + 1, P), 100.0, dtype=torch.float64, device="cuda")
    V = torch.full((N + 1, P), 0.04, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    c = L.lsmc_contract(L.LSMC_PUT, L.LSMC_AMERICAN, 100.0, 1.0)
    n0 = L.lsmc_device_allocations()
    with pytest.raises(L.LsmcError) as e:
        L.lsmc_backward_noalloc(S.data_ptr(), V.data_ptr(), P, N, L.LSMC_FP64,
                                L.lsmc_heston(**H), c, L.LSMC_BASIS_SV2, out.data_ptr())
    assert e.value.status == L.LSMC_ENOMEM
    assert L.lsmc_device_allocations() == n0
    assert torch.count_nonzero(out).item() == 0
