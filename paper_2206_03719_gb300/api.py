"""Convenience layer over the C ABI for Python callers (tests, benchmark).

Maps the string-valued Workload descriptions to lsmc_request structs and wraps
a context whose device memory is a PyTorch tensor and whose stream is a
PyTorch stream.  No arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes
import weakref
from typing import List, Optional, Sequence

from . import lsmc as L
from .workloads import Workload

_OPTION = {"put": L.LSMC_PUT, "call": L.LSMC_CALL}
_STYLE = {"american": L.LSMC_AMERICAN, "european": L.LSMC_EUROPEAN}
_BASIS = {"s2": L.LSMC_BASIS_S2, "sv2": L.LSMC_BASIS_SV2}
_SCHEME = {"qe": L.LSMC_SCHEME_QE, "ft_euler": L.LSMC_SCHEME_FT_EULER}
_PREC = {"fp64": L.LSMC_FP64, "mixed": L.LSMC_MIXED, "df": L.LSMC_DF}
_GREEK = {"delta": L.LSMC_GREEK_DELTA, "gamma": L.LSMC_GREEK_GAMMA,
          "vega": L.LSMC_GREEK_VEGA, "rho": L.LSMC_GREEK_RHO, "theta": L.LSMC_GREEK_THETA}


class Request:
    """An lsmc_request plus the strike array it points to."""

    def __init__(self, wl: Workload, precision: Optional[str] = None,
                 scheme: Optional[str] = None):
        self.workload = wl
        self.strikes = (ctypes.c_double * len(wl.strikes))(*wl.strikes)
        r = L.lsmc_request()
        r.model = L.lsmc_heston(**wl.model)
        r.type = _OPTION[wl.option]
        r.style = _STYLE[wl.style]
        r.T = wl.T
        r.strikes = ctypes.cast(self.strikes, ctypes.POINTER(ctypes.c_double))
        r.n_strikes = len(wl.strikes)
        r.n_paths = wl.n_paths
        r.n_steps = wl.n_steps
        r.basis = _BASIS[wl.basis]
        r.precision = _PREC[precision or wl.precision]
        r.scheme = _SCHEME[scheme or wl.scheme]
        mask = 0
        for g in wl.greeks:
            mask |= _GREEK[g]
        r.bumps = L.lsmc_bumps(wl.rel_dS, wl.rel_dS_gamma, wl.rel_dv0, wl.abs_dr, wl.abs_dT,
                               mask, 0)
        r.seed = wl.seed
        r.stream_id = wl.stream
        r.flags = (L.LSMC_FLAG_REGENERATE if wl.regenerate else 0) | \
            (L.LSMC_FLAG_OUT_OF_SAMPLE if wl.out_of_sample else 0) | \
            {"native": 0, "fp16": L.LSMC_FLAG_STORE_FP16, "bf16": L.LSMC_FLAG_STORE_BF16}[wl.store]
        self.c = r


class Context:
    """An lsmc context on the current CUDA device, fed PyTorch memory/streams."""

    def __init__(self, workspace_bytes: int = 0, precision: str = "fp64",
                 scheme: str = "qe", hbm_budget: int = 0, max_inflight: int = 8,
                 use_torch_stream: bool = True, device: Optional[int] = None,
                 torch_allocator: bool = False, max_batch: int = 0):
        import torch
        self.torch = torch
        dev = torch.cuda.current_device() if device is None else device
        cfg = L.lsmc_config(dev, _PREC[precision], _SCHEME[scheme], max_batch, hbm_budget,
                            max_inflight, 0)
        self.ctx = L.lsmc_create(cfg)
        self._plans = weakref.WeakSet()
        self._alloc_cbs = None
        if torch_allocator:
            # every allocation outside a workspace from PyTorch's caching allocator
            def alloc(nbytes):
                return torch.cuda.caching_allocator_alloc(nbytes, device=dev)

            self._alloc_cbs = L.lsmc_set_allocator(self.ctx, alloc,
                                                   torch.cuda.caching_allocator_delete)
        self.workspace = None
        if workspace_bytes:
            self.workspace = torch.empty(workspace_bytes, dtype=torch.uint8, device="cuda:%d" % dev)
            L.lsmc_set_workspace(self.ctx, self.workspace.data_ptr(), workspace_bytes)
        self.stream = None
        if use_torch_stream:
            # a stream of its own (the legacy default stream has handle 0,
            # which the library would read as "use your own stream")
            self.stream = torch.cuda.Stream(device=dev)
            L.lsmc_set_stream(self.ctx, self.stream.cuda_stream)
            if self.workspace is not None:
                self.workspace.record_stream(self.stream)

    def close(self):
        for p in list(self._plans):
            p.close()
        if self.ctx:
            L.lsmc_destroy(self.ctx)
            self.ctx = None
        self.workspace = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_wait_limit(self, seconds: float):
        L.lsmc_set_wait_limit(self.ctx, seconds)

    def set_backward_shape(self, sub: int = 0, ppt: int = 0):
        L.lsmc_set_backward_shape(self.ctx, sub, ppt)

    def set_serving_share(self, share: float = 0.0):
        L.lsmc_set_serving_share(self.ctx, share)

    # ---- synchronous ------------------------------------------------------
    def price(self, wl: Workload, **kw) -> List[dict]:
        req = Request(wl, **kw)
        return [r.as_dict() for r in L.lsmc_price_request(self.ctx, req.c)]

    def price_with_scenarios(self, wl: Workload, **kw):
        """(results, revaluations) of one request through a plan: the results
        of price() and, per strike, {scenario kind: (price, near ties)}."""
        return self.price_book_with_scenarios([wl], **kw)

    def price_book_with_scenarios(self, wls: Sequence[Workload], use_graph: bool = False, **kw):
        """price_book() through a plan, with the revaluations of every result."""
        plan = Plan(self, wls, **kw)
        try:
            plan.launch(use_graph)
            return plan.fetch(), plan.fetch_scenarios()
        finally:
            plan.close()

    def price_bounds(self, wl: Workload, n_outer: int, n_inner: int, **kw) -> List[dict]:
        """Lower (out-of-sample) and dual upper bounds of each strike's
        American price (base scenario)."""
        req = Request(wl, **kw)
        return [b.as_dict() for b in L.lsmc_price_bounds(self.ctx, req.c, n_outer, n_inner)]

    def price_book(self, wls: Sequence[Workload], **kw) -> List[dict]:
        reqs = [Request(w, **kw) for w in wls]
        return [r.as_dict() for r in L.lsmc_price_book(self.ctx, [q.c for q in reqs])]

    def layout(self, wls: Sequence[Workload], sub: int, ppt: int = 0, **kw):
        """Counters (lsmc_plan_info) of the plan these workloads would get
        with backward shape (sub | LSMC_SUB_ITM_HALF, ppt), computed on the
        host without allocating."""
        return plan_layout(wls, sub, ppt, ctx=self, **kw)

    def autotune(self, wls: Sequence[Workload], **kw):
        """(sub-tiles per backward job, paths per lane, backward ms) chosen
        for these requests."""
        reqs = [Request(w, **kw) for w in wls]
        return L.lsmc_autotune(self.ctx, [q.c for q in reqs])

    def plan(self, wls: Sequence[Workload], **kw) -> "Plan":
        return Plan(self, wls, **kw)

    # ---- serving ------------------------------------------------------------
    def submit(self, wl: Workload, **kw) -> int:
        req = Request(wl, **kw)
        return L.lsmc_submit(self.ctx, req.c)

    def wait(self, ticket: int, n_strikes: int, timeout_s: float = -1.0):
        return L.lsmc_wait(self.ctx, ticket, n_strikes, timeout_s)

    def poll(self, ticket: int, n_strikes: int):
        return L.lsmc_poll(self.ctx, ticket, n_strikes)


def plan_layout(wls: Sequence[Workload], sub: int, ppt: int = 0, ctx: "Context" = None, **kw):
    """Counters (lsmc_plan_info) of the plan these workloads would get with
    backward shape (sub | LSMC_SUB_ITM_HALF, ppt); host only, no device
    needed."""
    reqs = [Request(w, **kw) for w in wls]
    return L.lsmc_plan_layout_info(ctx.ctx if ctx is not None else None, [q.c for q in reqs],
                                   sub, ppt)


class Plan:
    """A built launch: tables uploaded, device memory reserved."""

    def __init__(self, ctx: Context, wls: Sequence[Workload], **kw):
        self.ctx = ctx
        self.reqs = [Request(w, **kw) for w in wls]
        self.n_results = sum(len(w.strikes) for w in wls)
        self.handle = L.lsmc_plan_create(ctx.ctx, [q.c for q in self.reqs])
        ctx._plans.add(self)

    def launch(self, use_graph: bool = False):
        L.lsmc_plan_launch(self.handle, use_graph)

    def fetch(self) -> List[dict]:
        return [r.as_dict() for r in L.lsmc_plan_fetch(self.handle, self.n_results)]

    def fetch_scenarios(self):
        """Per result, {scenario kind: (price, near ties)} of the last launch
        (the revaluations the Greeks are differences of)."""
        prices, ties = L.lsmc_plan_fetch_scenarios(self.handle, self.n_results)
        return [{kind: (p[i], t[i]) for i, kind in enumerate(L.LSMC_SC_KINDS) if p[i] == p[i]}
                for p, t in zip(prices, ties)]

    def info(self):
        return L.lsmc_plan_get_info(self.handle)

    def set_timing(self, enable: bool = True):
        L.lsmc_plan_set_timing(self.handle, enable)

    def kernel_times(self):
        """(ms per kernel [setup, forward, backward, greeks], launches)."""
        return L.lsmc_plan_kernel_times(self.handle)

    def device_results(self):
        return L.lsmc_plan_device_results(self.handle)

    def close(self):
        if self.handle:
            L.lsmc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
