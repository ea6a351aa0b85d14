"""Continuous batching: requests of different sizes submitted together are
admitted in batches as slots and memory free up, run concurrently, and each
result is bit-identical to the same request served alone."""
import time

import pytest

from gpu_common import torch_cuda
from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()


def _mix():
    return workloads.book(n_contracts=10, paths_hi=40000, steps=(16, 32, 50), precision="mixed")


def _serve(ctx, ws):
    tickets = [ctx.submit(w) for w in ws]
    out = []
    for t, w in zip(tickets, ws):
        st, res = ctx.wait(t, len(w.strikes), 60.0)
        assert st == L.LSMC_OK
        out.append([r.as_dict() for r in res])
    return out


def test_results_same_alone_and_in_the_mix(setup):
    # alone: each request submitted and finished before the next; in the mix:
    # all submitted at once, so they are batched and overlap on the device
    mix = _mix()
    with api.Context(workspace_bytes=4 << 30, max_inflight=4) as solo:
        alone = [_serve(solo, [w])[0] for w in mix]
    with api.Context(workspace_bytes=4 << 30, max_inflight=2) as srv:
        got = _serve(srv, mix)
    assert got == alone
    # and they agree with the synchronous call within the parity bound
    with api.Context(workspace_bytes=4 << 30) as sync:
        for w, g in zip(mix[:3], got):
            ref = sync.price(w)
            for a, b in zip(g, ref):
                assert abs(a["price"] - b["price"]) <= 1e-4 * abs(b["price"])


def test_admission_by_memory_budget(setup):
    mix = _mix()[:6]
    need = max(L.lsmc_request_footprint(None, api.Request(w).c) for w in mix)
    # room for about two requests at a time
    with api.Context(workspace_bytes=int(2.2 * need) // 256 * 256 + 4096, max_inflight=8) as srv:
        tickets = [srv.submit(w) for w in mix]
        done = [srv.wait(t, len(w.strikes), 120.0) for t, w in zip(tickets, mix)]
        assert all(st == L.LSMC_OK for st, _ in done)
    with api.Context(workspace_bytes=1 << 20) as tiny:
        with pytest.raises(L.LsmcError) as e:
            tiny.submit(mix[0])
        assert e.value.status == L.LSMC_ENOMEM


def test_poll_pending_then_done_and_unknown_ticket(setup):
    w = workloads.SMALL_FP64.replace(n_paths=65536, n_steps=100)
    with api.Context(workspace_bytes=2 << 30) as srv:
        t = srv.submit(w)
        st, _ = srv.poll(t, 1)
        assert st in (L.LSMC_PENDING, L.LSMC_OK)
        t0 = time.time()
        while st == L.LSMC_PENDING and time.time() - t0 < 60:
            time.sleep(0.001)
            st, res = srv.poll(t, 1)
        assert st == L.LSMC_OK and res[0].price > 0
        with pytest.raises(L.LsmcError) as e:
            srv.poll(t, 1)
        assert e.value.status == L.LSMC_ENOTFOUND
