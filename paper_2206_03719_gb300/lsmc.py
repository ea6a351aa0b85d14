"""ctypes binding of liblsmc.so (include/lsmc.h): argument marshalling only.

Every function of the C ABI is exposed under its C name with the same
arguments.  All computation runs in the library's CUDA kernels; if the
library has not been built (see paper_2206_03719_gb300.build) loading fails
with an error instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

LSMC_ABI_VERSION = 1
LSMC_OK, LSMC_PENDING = 0, 1
LSMC_EINVAL, LSMC_ENOMEM, LSMC_EBUSY, LSMC_ETIMEOUT = -1, -2, -3, -4
LSMC_ECUDA, LSMC_ENOTIMPL, LSMC_ENOTFOUND, LSMC_ENODEV = -5, -6, -7, -8
LSMC_PUT, LSMC_CALL = 0, 1
LSMC_AMERICAN, LSMC_EUROPEAN = 0, 1
LSMC_SCHEME_QE, LSMC_SCHEME_FT_EULER = 0, 1
LSMC_BASIS_S2, LSMC_BASIS_SV2 = 0, 1
LSMC_FLAG_REGENERATE = 1
LSMC_FLAG_OUT_OF_SAMPLE = 2
LSMC_FLAG_STORE_FP16 = 4
LSMC_FLAG_STORE_BF16 = 8
LSMC_FP64, LSMC_MIXED, LSMC_DF = 0, 1, 2
LSMC_SUB_ITM_HALF = 0x8000
LSMC_GREEK_DELTA, LSMC_GREEK_GAMMA, LSMC_GREEK_VEGA = 1, 2, 4
LSMC_GREEK_RHO, LSMC_GREEK_THETA, LSMC_GREEK_ALL = 8, 16, 31

EXPORTS = [
    "lsmc_strerror", "lsmc_abi_version", "lsmc_create", "lsmc_destroy",
    "lsmc_set_stream", "lsmc_set_workspace", "lsmc_set_allocator", "lsmc_request_footprint",
    "lsmc_price_greeks", "lsmc_price_request", "lsmc_price_book", "lsmc_price_bounds",
    "lsmc_plan_create", "lsmc_plan_launch", "lsmc_plan_fetch",
    "lsmc_plan_device_results", "lsmc_plan_get_info", "lsmc_plan_layout_info", "lsmc_plan_destroy",
    "lsmc_plan_set_timing", "lsmc_plan_kernel_times", "lsmc_autotune",
    "lsmc_submit", "lsmc_poll", "lsmc_wait", "lsmc_ticket_times",
    "lsmc_philox", "lsmc_draws", "lsmc_paths", "lsmc_multi_asset_max", "lsmc_backward",
    "lsmc_backward_noalloc", "lsmc_device_allocations", "lsmc_set_wait_limit",
    "lsmc_set_backward_shape", "lsmc_set_serving_share", "lsmc_plan_fetch_scenarios",
    "lsmc_measure_peaks", "lsmc_check_report", "lsmc_exp", "lsmc_quantile",
]
# scenario kinds of a result's revaluations (lsmc_plan_fetch_scenarios)
LSMC_SC_KINDS = ("base", "S+", "S-", "Sg+", "Sg-", "v0+", "v0-", "r+", "r-", "T-", "T+")
(LSMC_SC_BASE, LSMC_SC_S_UP, LSMC_SC_S_DN, LSMC_SC_SG_UP, LSMC_SC_SG_DN, LSMC_SC_V0_UP,
 LSMC_SC_V0_DN, LSMC_SC_R_UP, LSMC_SC_R_DN, LSMC_SC_T_DN, LSMC_SC_T_UP) = range(11)
LSMC_SC_COUNT = len(LSMC_SC_KINDS)


class lsmc_heston(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("S0", "r", "q", "v0", "kappa", "theta", "xi", "rho")]


class lsmc_contract(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("style", ctypes.c_int32),
                ("K", ctypes.c_double), ("T", ctypes.c_double)]


class lsmc_bumps(ctypes.Structure):
    _fields_ = [("rel_dS", ctypes.c_double), ("rel_dS_gamma", ctypes.c_double),
                ("rel_dv0", ctypes.c_double), ("abs_dr", ctypes.c_double),
                ("abs_dT", ctypes.c_double), ("greek_mask", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class lsmc_result(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("price", "price_se", "delta", "gamma", "vega", "rho", "theta",
                 "european_price")] + [
        ("n_singular_solves", ctypes.c_uint32), ("n_revaluations", ctypes.c_uint32),
        ("status", ctypes.c_int32), ("n_near_ties", ctypes.c_uint32)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class lsmc_bounds(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("lower", "lower_se", "upper", "upper_se", "martingale_end",
                 "martingale_end_se", "dual_ms")] + [
        ("n_near_ties", ctypes.c_uint32), ("status", ctypes.c_int32)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class lsmc_peaks(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("fp64_tflops", "fp32_tflops", "xu_tops", "fp64_ms", "fp32_ms", "xu_ms")] + [
        ("sms", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if f[0] != "reserved"}


class lsmc_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("hbm_budget", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("queue_capacity", ctypes.c_uint32)]


class lsmc_request(ctypes.Structure):
    _fields_ = [("model", lsmc_heston), ("type", ctypes.c_int32),
                ("style", ctypes.c_int32), ("T", ctypes.c_double),
                ("strikes", ctypes.POINTER(ctypes.c_double)),
                ("n_strikes", ctypes.c_uint32), ("n_paths", ctypes.c_uint32),
                ("n_steps", ctypes.c_uint32), ("basis", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("bumps", lsmc_bumps), ("seed", ctypes.c_uint64),
                ("stream_id", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class lsmc_plan_info(ctypes.Structure):
    _fields_ = [("generated_path_steps", ctypes.c_uint64),
                ("lsmc_path_steps", ctypes.c_uint64),
                ("backward_jobs", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("kernels_per_launch", ctypes.c_uint32), ("n_results", ctypes.c_uint32),
                ("n_instances", ctypes.c_uint32), ("n_groups", ctypes.c_uint32),
                ("itm_path_steps", ctypes.c_uint64), ("h2d_bytes", ctypes.c_uint64),
                ("d2h_bytes", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False, path: str = None):
    """Load liblsmc.so (raises if it is missing and build_if_missing is False).
    path: another build of the library (e.g. the checked build) to load
    instead, only before the first load of the process."""
    global _lib
    with _lock:
        if _lib is not None:
            if path is not None and path != _lib._name:
                raise RuntimeError("another build of liblsmc.so is already loaded")
            return _lib
        path = path or _build.LIB_PATH
        if build_if_missing and path == _build.LIB_PATH:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(
                "liblsmc.so is not built (%s); run paper_2206_03719_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, sz, u32, u64, i32, dbl = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_int32, ctypes.c_double)
        sig = {
            "lsmc_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "lsmc_abi_version": ([], ctypes.c_int),
            "lsmc_create": ([P(vp), P(lsmc_config)], ctypes.c_int),
            "lsmc_destroy": ([vp], None),
            "lsmc_set_stream": ([vp, vp], ctypes.c_int),
            "lsmc_set_workspace": ([vp, vp, sz], ctypes.c_int),
            "lsmc_set_allocator": ([vp, ALLOC_FN, FREE_FN, vp], ctypes.c_int),
            "lsmc_request_footprint": ([vp, P(lsmc_request), P(sz)], ctypes.c_int),
            "lsmc_price_greeks": ([vp, P(lsmc_heston), P(lsmc_contract), u32, u32, i32,
                                   P(lsmc_bumps), u64, P(lsmc_result)], ctypes.c_int),
            "lsmc_price_request": ([vp, P(lsmc_request), P(lsmc_result)], ctypes.c_int),
            "lsmc_price_book": ([vp, P(lsmc_request), sz, P(lsmc_result)], ctypes.c_int),
            "lsmc_price_bounds": ([vp, P(lsmc_request), ctypes.c_uint32, ctypes.c_uint32,
                                   P(lsmc_bounds)], ctypes.c_int),
            "lsmc_plan_create": ([vp, P(lsmc_request), sz, P(vp)], ctypes.c_int),
            "lsmc_plan_launch": ([vp, i32], ctypes.c_int),
            "lsmc_plan_fetch": ([vp, P(lsmc_result)], ctypes.c_int),
            "lsmc_plan_device_results": ([vp, P(vp), P(sz)], ctypes.c_int),
            "lsmc_plan_get_info": ([vp, P(lsmc_plan_info)], ctypes.c_int),
            "lsmc_plan_layout_info": ([vp, P(lsmc_request), sz, u32, u32, P(lsmc_plan_info)],
                                      ctypes.c_int),
            "lsmc_plan_destroy": ([vp], None),
            "lsmc_plan_set_timing": ([vp, i32], ctypes.c_int),
            "lsmc_plan_kernel_times": ([vp, P(dbl), P(u32)], ctypes.c_int),
            "lsmc_autotune": ([vp, P(lsmc_request), sz, P(u32), P(u32), P(dbl)], ctypes.c_int),
            "lsmc_submit": ([vp, P(lsmc_request), P(u64)], ctypes.c_int),
            "lsmc_poll": ([vp, u64, P(lsmc_result)], ctypes.c_int),
            "lsmc_wait": ([vp, u64, P(lsmc_result), dbl], ctypes.c_int),
            "lsmc_ticket_times": ([vp, u64, P(dbl), P(dbl), P(dbl)], ctypes.c_int),
            "lsmc_philox": ([vp, u32, u32, vp, sz, vp], ctypes.c_int),
            "lsmc_draws": ([u64, u32, vp, vp, sz, i32, vp, vp], ctypes.c_int),
            "lsmc_multi_asset_max": ([P(lsmc_heston), u32, dbl, i32, i32, dbl, u32, u32, u64,
                                      u32, vp, vp], ctypes.c_int),
            "lsmc_paths": ([P(lsmc_heston), dbl, i32, i32, u32, u32, u64, u32, vp, vp, vp],
                           ctypes.c_int),
            "lsmc_backward": ([vp, vp, u32, u32, i32, P(lsmc_heston), P(lsmc_contract), i32,
                               vp, vp, vp, vp], ctypes.c_int),
            "lsmc_backward_noalloc": ([vp, vp, u32, u32, i32, P(lsmc_heston), P(lsmc_contract),
                                       i32, vp, vp, vp, vp], ctypes.c_int),
            "lsmc_device_allocations": ([P(u64)], ctypes.c_int),
            "lsmc_set_wait_limit": ([vp, dbl], ctypes.c_int),
            "lsmc_set_backward_shape": ([vp, u32, u32], ctypes.c_int),
            "lsmc_set_serving_share": ([vp, ctypes.c_double], ctypes.c_int),
            "lsmc_plan_fetch_scenarios": ([vp, P(dbl), P(u32), sz], ctypes.c_int),
            "lsmc_measure_peaks": ([i32, P(lsmc_peaks)], ctypes.c_int),
            "lsmc_check_report": ([P(u32), P(u32), i32], ctypes.c_int),
            "lsmc_exp": ([vp, vp, sz, i32, vp], ctypes.c_int),
            "lsmc_quantile": ([vp, vp, sz, i32, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


class LsmcError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = load().lsmc_strerror(status).decode()
        super().__init__("%s: %s (%d)" % (what, msg, status) if what else "%s (%d)" % (msg, status))


def check(status, what=""):
    if status < 0:
        raise LsmcError(status, what)
    return status


# ---- C-named wrappers (same names and arguments as include/lsmc.h) ---------
def lsmc_strerror(status):
    return load().lsmc_strerror(status).decode()


def lsmc_abi_version():
    return load().lsmc_abi_version()


def lsmc_create(config):
    ctx = ctypes.c_void_p()
    check(load().lsmc_create(ctypes.byref(ctx), ctypes.byref(config) if config else None),
          "lsmc_create")
    return ctx


def lsmc_destroy(ctx):
    load().lsmc_destroy(ctx)


def lsmc_set_stream(ctx, stream):
    return check(load().lsmc_set_stream(ctx, stream), "lsmc_set_stream")


# device memory callbacks: alloc(bytes, user) -> pointer, release(pointer, user)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def lsmc_set_allocator(ctx, alloc, release):
    """alloc(nbytes) -> int device pointer (0 on failure), release(ptr);
    returns the ctypes callbacks, which the caller keeps alive while the
    context exists.  alloc = release = None restores cudaMalloc."""
    if alloc is None:
        check(load().lsmc_set_allocator(ctx, ALLOC_FN(), FREE_FN(), None), "lsmc_set_allocator")
        return None
    a = ALLOC_FN(lambda n, user: alloc(n) or None)
    f = FREE_FN(lambda ptr, user: release(ptr))
    check(load().lsmc_set_allocator(ctx, a, f, None), "lsmc_set_allocator")
    return (a, f)


def lsmc_device_allocations():
    n = ctypes.c_uint64()
    check(load().lsmc_device_allocations(ctypes.byref(n)), "lsmc_device_allocations")
    return n.value


def lsmc_measure_peaks(device=0):
    out = lsmc_peaks()
    check(load().lsmc_measure_peaks(device, ctypes.byref(out)), "lsmc_measure_peaks")
    return out.as_dict()


def lsmc_check_report(reset=False):
    """(code, line) of the checked build's first out-of-range access (0, 0:
    none); LsmcError(LSMC_ENOTIMPL) from the ordinary build."""
    code, line = ctypes.c_uint32(), ctypes.c_uint32()
    check(load().lsmc_check_report(ctypes.byref(code), ctypes.byref(line), 1 if reset else 0),
          "lsmc_check_report")
    return code.value, line.value


def lsmc_set_wait_limit(ctx, seconds):
    return check(load().lsmc_set_wait_limit(ctx, seconds), "lsmc_set_wait_limit")


def lsmc_set_backward_shape(ctx, sub, ppt):
    return check(load().lsmc_set_backward_shape(ctx, sub, ppt), "lsmc_set_backward_shape")


def lsmc_set_serving_share(ctx, share):
    return check(load().lsmc_set_serving_share(ctx, share), "lsmc_set_serving_share")


def lsmc_set_workspace(ctx, ptr, nbytes):
    return check(load().lsmc_set_workspace(ctx, ptr, nbytes), "lsmc_set_workspace")


def lsmc_request_footprint(ctx, req):
    n = ctypes.c_size_t()
    check(load().lsmc_request_footprint(ctx, ctypes.byref(req), ctypes.byref(n)),
          "lsmc_request_footprint")
    return n.value


def lsmc_price_greeks(ctx, model, contract, n_paths, n_steps, basis, bumps, seed):
    out = lsmc_result()
    check(load().lsmc_price_greeks(ctx, ctypes.byref(model), ctypes.byref(contract), n_paths,
                                   n_steps, basis, ctypes.byref(bumps), seed,
                                   ctypes.byref(out)), "lsmc_price_greeks")
    return out


def lsmc_price_request(ctx, req):
    outs = (lsmc_result * req.n_strikes)()
    check(load().lsmc_price_request(ctx, ctypes.byref(req), outs), "lsmc_price_request")
    return list(outs)


def lsmc_price_book(ctx, reqs):
    arr = (lsmc_request * len(reqs))(*reqs)
    total = sum(r.n_strikes for r in reqs)
    outs = (lsmc_result * total)()
    check(load().lsmc_price_book(ctx, arr, len(reqs), outs), "lsmc_price_book")
    return list(outs)


def lsmc_price_bounds(ctx, req, n_outer, n_inner):
    outs = (lsmc_bounds * req.n_strikes)()
    check(load().lsmc_price_bounds(ctx, ctypes.byref(req), n_outer, n_inner, outs),
          "lsmc_price_bounds")
    return list(outs)


def lsmc_plan_create(ctx, reqs):
    arr = (lsmc_request * len(reqs))(*reqs)
    plan = ctypes.c_void_p()
    check(load().lsmc_plan_create(ctx, arr, len(reqs), ctypes.byref(plan)), "lsmc_plan_create")
    return plan


def lsmc_plan_launch(plan, use_graph=False):
    return check(load().lsmc_plan_launch(plan, 1 if use_graph else 0), "lsmc_plan_launch")


def lsmc_plan_fetch(plan, n_results):
    outs = (lsmc_result * n_results)()
    check(load().lsmc_plan_fetch(plan, outs), "lsmc_plan_fetch")
    return list(outs)


def lsmc_plan_fetch_scenarios(plan, n_results):
    """(prices, near_ties): lists of n_results rows of LSMC_SC_COUNT values."""
    prices = (ctypes.c_double * (n_results * LSMC_SC_COUNT))()
    ties = (ctypes.c_uint32 * (n_results * LSMC_SC_COUNT))()
    check(load().lsmc_plan_fetch_scenarios(plan, prices, ties, n_results),
          "lsmc_plan_fetch_scenarios")
    rows = lambda a: [list(a[k * LSMC_SC_COUNT:(k + 1) * LSMC_SC_COUNT]) for k in range(n_results)]
    return rows(prices), rows(ties)


def lsmc_plan_device_results(plan):
    p, n = ctypes.c_void_p(), ctypes.c_size_t()
    check(load().lsmc_plan_device_results(plan, ctypes.byref(p), ctypes.byref(n)),
          "lsmc_plan_device_results")
    return p.value, n.value


def lsmc_plan_get_info(plan):
    info = lsmc_plan_info()
    check(load().lsmc_plan_get_info(plan, ctypes.byref(info)), "lsmc_plan_get_info")
    return info


def lsmc_plan_layout_info(ctx, reqs, sub, ppt=0):
    """Counters of the plan these requests would get with this backward
    shape, computed on the host (ctx may be None)."""
    arr = (lsmc_request * len(reqs))(*reqs)
    info = lsmc_plan_info()
    check(load().lsmc_plan_layout_info(ctx, arr, len(reqs), sub, ppt, ctypes.byref(info)),
          "lsmc_plan_layout_info")
    return info


def lsmc_plan_set_timing(plan, enable=True):
    return check(load().lsmc_plan_set_timing(plan, 1 if enable else 0), "lsmc_plan_set_timing")


def lsmc_plan_kernel_times(plan):
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_uint32()
    check(load().lsmc_plan_kernel_times(plan, ms, ctypes.byref(n)), "lsmc_plan_kernel_times")
    return list(ms), n.value


def lsmc_autotune(ctx, reqs):
    """(sub-tiles per job, paths per lane, backward ms) of the fastest shape."""
    arr = (lsmc_request * len(reqs))(*reqs)
    sub, ppt, ms = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
    check(load().lsmc_autotune(ctx, arr, len(reqs), ctypes.byref(sub), ctypes.byref(ppt),
                               ctypes.byref(ms)), "lsmc_autotune")
    return sub.value, ppt.value, ms.value


def lsmc_plan_destroy(plan):
    load().lsmc_plan_destroy(plan)


def lsmc_submit(ctx, req):
    t = ctypes.c_uint64()
    check(load().lsmc_submit(ctx, ctypes.byref(req), ctypes.byref(t)), "lsmc_submit")
    return t.value


def lsmc_poll(ctx, ticket, n_strikes):
    outs = (lsmc_result * n_strikes)()
    st = check(load().lsmc_poll(ctx, ticket, outs), "lsmc_poll")
    return st, (list(outs) if st == LSMC_OK else None)


def lsmc_wait(ctx, ticket, n_strikes, timeout_s=-1.0):
    outs = (lsmc_result * n_strikes)()
    st = check(load().lsmc_wait(ctx, ticket, outs, timeout_s), "lsmc_wait")
    return st, (list(outs) if st == LSMC_OK else None)


def lsmc_ticket_times(ctx, ticket):
    s, a, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(load().lsmc_ticket_times(ctx, ticket, ctypes.byref(s), ctypes.byref(a),
                                   ctypes.byref(d)), "lsmc_ticket_times")
    return s.value, a.value, d.value


def lsmc_philox(d_ctr, key_lo, key_hi, d_out, n, stream=None):
    return check(load().lsmc_philox(d_ctr, key_lo, key_hi, d_out, n, stream), "lsmc_philox")


def lsmc_draws(seed, stream_id, d_path, d_step, n, precision, d_out, stream=None):
    return check(load().lsmc_draws(seed, stream_id, d_path, d_step, n, precision, d_out, stream),
                 "lsmc_draws")


def lsmc_exp(d_x, d_y, n, precision, stream=None):
    return check(load().lsmc_exp(d_x, d_y, n, precision, stream), "lsmc_exp")


def lsmc_quantile(d_u, d_z, n, precision, stream=None):
    return check(load().lsmc_quantile(d_u, d_z, n, precision, stream), "lsmc_quantile")


def lsmc_paths(model, T, scheme, precision, n_paths, n_steps, seed, stream_id, d_S, d_V,
               stream=None):
    return check(load().lsmc_paths(ctypes.byref(model), T, scheme, precision, n_paths, n_steps,
                                   seed, stream_id, d_S, d_V, stream), "lsmc_paths")


def lsmc_multi_asset_max(models, T, scheme, precision, rho_assets, n_paths, n_steps, seed,
                         stream_id, d_M, stream=None):
    """STAC-A2 path reduction into device memory d_M ((n_steps + 1) x n_paths)."""
    arr = (lsmc_heston * len(models))(*models)
    return check(load().lsmc_multi_asset_max(arr, len(models), T, scheme, precision, rho_assets,
                                             n_paths, n_steps, seed, stream_id, d_M, stream),
                 "lsmc_multi_asset_max")


def lsmc_backward(d_S, d_V, n_paths, n_steps, precision, model, contract, basis, d_out,
                  d_beta=None, d_n_singular=None, stream=None):
    return check(load().lsmc_backward(d_S, d_V, n_paths, n_steps, precision, ctypes.byref(model),
                                      ctypes.byref(contract), basis, d_out, d_beta, d_n_singular,
                                      stream), "lsmc_backward")


def lsmc_backward_noalloc(d_S, d_V, n_paths, n_steps, precision, model, contract, basis, d_out,
                          d_beta=None, d_n_singular=None, stream=None):
    return check(load().lsmc_backward_noalloc(d_S, d_V, n_paths, n_steps, precision,
                                              ctypes.byref(model), ctypes.byref(contract), basis,
                                              d_out, d_beta, d_n_singular, stream),
                 "lsmc_backward_noalloc")
