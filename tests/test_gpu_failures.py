"""Failure paths on the GPU, made on the host or by a short wait limit; no
test faults, traps or hangs the device.

* A device-side wait that runs out: the exercise dates of one regression form
  a chain (a job of date n waits for the coefficients of date n + 1, which
  the last job of that date publishes), so with one path tile per date and
  500 dates the later dates' jobs wait for hundreds of microseconds.  A wait
  limit of 20 microseconds must make them give up: the kernels record the
  error and return, the call reports LSMC_ETIMEOUT, and the same context then
  prices the request correctly under the default limit.
* The same expiry in a serving batch: the ticket reports it and the slots
  serve the next requests.
* Device memory refused by the caller's allocator (lsmc_set_allocator): the
  call reports LSMC_ENOMEM, every block handed out is handed back, and the
  context works again once the allocator gives memory.
"""
import pytest

from gpu_common import assert_close, scenario_parity, torch_cuda
from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    return t


def test_device_wait_limit_expires_and_the_context_stays_usable(torch):
    wl = workloads.SMALL_FP64.replace(n_paths=1000, n_steps=500, greeks=(), strikes=[100.0])
    with api.Context(workspace_bytes=256 << 20) as c:
        c.set_wait_limit(20e-6)
        for _ in range(2):
            with pytest.raises(L.LsmcError) as e:
                c.price(wl)
            assert e.value.status == L.LSMC_ETIMEOUT
        c.set_wait_limit(20.0)
        got, scen = c.price_with_scenarios(wl)
        scenario_parity(wl, got, scen, what="after a timeout")
    with pytest.raises(L.LsmcError) as e:
        with api.Context() as c:
            c.set_wait_limit(-1.0)
    assert e.value.status == L.LSMC_EINVAL


def test_served_request_reports_the_expired_wait_and_the_slot_serves_on(torch):
    # the same chain of dates through the serving loop: the batch's kernels
    # give up, the ticket reports LSMC_ETIMEOUT (a request that finished its
    # own regressions before the expiry keeps its results), and the slots
    # serve the next requests under the default limit
    long_ = workloads.SMALL_FP64.replace(n_paths=1000, n_steps=500, greeks=(), strikes=[100.0])
    with api.Context(workspace_bytes=1 << 30, max_inflight=2) as srv:
        srv.set_backward_shape(2, 4)
        srv.set_wait_limit(20e-6)
        t = srv.submit(long_)
        with pytest.raises(L.LsmcError) as e:
            srv.wait(t, 1, 60.0)
        assert e.value.status == L.LSMC_ETIMEOUT
        srv.set_wait_limit(20.0)
        ts = [srv.submit(long_) for _ in range(3)]
        outs = [srv.wait(t, 1, 120.0) for t in ts]
        assert all(st == L.LSMC_OK for st, _ in outs)
        with api.Context(workspace_bytes=256 << 20) as sync:
            sync.set_backward_shape(2, 4)
            ref = sync.price(long_)
        for _, res in outs:  # one backward shape: the same bits
            assert res[0].as_dict()["price"] == ref[0]["price"]


def test_allocator_refusals_report_enomem_and_hand_every_block_back(torch):
    wl = workloads.SMALL_FP64.replace(n_paths=3000, n_steps=12)
    state = {"limit": 0, "alloc": 0, "free": 0, "refused": 0, "live": set()}

    def alloc(n):
        if state["alloc"] >= state["limit"]:
            state["refused"] += 1
            return 0
        state["alloc"] += 1
        p = torch.cuda.caching_allocator_alloc(n)
        state["live"].add(p)
        return p

    def release(p):
        state["free"] += 1
        state["live"].remove(p)
        torch.cuda.caching_allocator_delete(p)

    with api.Context() as ref_ctx:
        ref = ref_ctx.price(wl)
    ctx = api.Context(hbm_budget=256 << 20)  # the serving arena: 256 MiB
    keep = L.lsmc_set_allocator(ctx.ctx, alloc, release)
    try:
        # the plan's memory refused
        with pytest.raises(L.LsmcError) as e:
            ctx.price(wl)
        assert e.value.status == L.LSMC_ENOMEM and state["refused"] == 1
        assert not state["live"]
        # the dual bound: the plan gets its block, the dual pass's scratch is
        # refused; the plan's block comes back
        state["limit"] = state["alloc"] + 1
        with pytest.raises(L.LsmcError) as e:
            ctx.price_bounds(wl.replace(greeks=()), 32, 8)
        assert e.value.status == L.LSMC_ENOMEM and state["refused"] == 2
        assert not state["live"]
        # the serving arena refused: submit fails, nothing is held
        with pytest.raises(L.LsmcError) as e:
            ctx.submit(wl)
        assert e.value.status == L.LSMC_ENOMEM and state["refused"] == 3
        assert not state["live"]
        # memory again: the same context prices, serves and bounds as before
        state["limit"] = 10**9
        again = ctx.price(wl)
        assert len(again) == len(ref) and all(
            x[k] == y[k] or (x[k] != x[k] and y[k] != y[k]) for x, y in zip(again, ref) for k in x)
        t = ctx.submit(wl)
        st, out = ctx.wait(t, len(wl.strikes), 60.0)
        assert st == L.LSMC_OK
        # serving picks its own tile shape: the same results up to the order
        # of the moment sums
        assert_close(out[0].as_dict(), ref[0], 1e-10, what="served after a refusal")
        assert ctx.price_bounds(wl.replace(greeks=()), 32, 8)[0]["upper"] > 0.0
    finally:
        ctx.close()
        del keep
        torch.cuda.empty_cache()
    assert not state["live"]
    assert state["alloc"] == state["free"] and state["alloc"] >= 3
