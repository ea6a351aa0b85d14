"""Continuous batching: requests of different sizes submitted together are
admitted in batches as slots and memory free up, run concurrently, and each
result is bit-identical to the same request served alone."""
import time

import pytest

from gpu_common import same_results, torch_cuda
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


def test_results_same_with_a_share_of_the_device(setup):
    # four slots, each batch's persistent backward grid a quarter of the
    # device: batches run side by side and the results do not change
    mix = _mix()
    with api.Context(workspace_bytes=4 << 30, max_inflight=4) as solo:
        alone = [_serve(solo, [w])[0] for w in mix]
    with api.Context(workspace_bytes=4 << 30, max_inflight=4) as srv:
        srv.set_serving_share(0.25)
        got = _serve(srv, mix)
    assert got == alone
    with api.Context(workspace_bytes=1 << 30) as ctx:
        ctx.set_serving_share(0.0)  # the default: a share of 1 / slots
        for bad in (-0.5, 1.5):
            with pytest.raises(L.LsmcError) as e:
                ctx.set_serving_share(bad)
            assert e.value.status == L.LSMC_EINVAL


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


def test_request_finishes_ahead_of_its_batch(setup):
    # one slot: while a blocker runs, a short request (8 dates) and a long one
    # (400 dates) queue and are then admitted together; the backward pass
    # hands the short one over when its own regressions are done, well before
    # the batch ends.  Under one fixed backward shape its results equal, bit
    # for bit, those of the synchronous call (the Greeks kernel's path).
    base = workloads.SMALL_FP64.replace(precision="df", greeks=workloads.ALL_GREEKS,
                                        basis="sv2", rel_dS_gamma=0.02)
    blocker = base.replace(n_paths=65536, n_steps=200)
    short = base.replace(n_paths=8192, n_steps=8, strikes=[95.0, 105.0])
    long_ = base.replace(n_paths=65536, n_steps=400)
    with api.Context(workspace_bytes=4 << 30, max_inflight=1) as srv:
        srv.set_backward_shape(2, 4)
        ts = [srv.submit(w) for w in (blocker, short, long_)]
        got = []
        for t, w in zip(ts, (blocker, short, long_)):
            st, res = srv.wait(t, len(w.strikes), 120.0)
            assert st == L.LSMC_OK
            got.append([r.as_dict() for r in res])
        times = [L.lsmc_ticket_times(srv.ctx, t) for t in ts]
    (_, a_b, d_b), (_, a_s, d_s), (_, a_l, d_l) = times
    assert a_s == a_l > a_b          # admitted together, after the blocker
    assert d_s < d_l                 # the short request left its batch early
    print("short done %.1f ms before the long one" % (1e3 * (d_l - d_s)))
    with api.Context(workspace_bytes=4 << 30) as sync:
        sync.set_backward_shape(2, 4)
        for w, g in zip((short, long_), got[1:]):
            assert same_results(g, sync.price(w)), w.name
