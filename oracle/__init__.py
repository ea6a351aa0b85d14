"""ctypes binding of the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark are the only callers.  The product package never imports
this module, and this module imports nothing from the product package.

`build()` compiles oracle.c with gcc (no FMA contraction) into
oracle/_build/liboracle.so; `lib()` loads it, building on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h")]
_lock = threading.Lock()
_lib = None

PUT, CALL = 0, 1
AMERICAN, EUROPEAN = 0, 1
QE, FT_EULER = 0, 1
BASIS_S2, BASIS_SV2 = 0, 1
GRID_F64, GRID_F32 = 0, 1
DELTA, GAMMA, VEGA, RHO, THETA = 1, 2, 4, 8, 16
SC_KINDS = ["base", "S+", "S-", "Sg+", "Sg-", "v0+", "v0-", "r+", "r-", "T-", "T+"]
KEY_PRICING = 1 << 62   # near-tie keys of the out-of-sample pricing pass
MAX_ALT_KEYS = 12


class Heston(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("S0", "r", "q", "v0", "kappa", "theta", "xi", "rho")]


class Bumps(ctypes.Structure):
    _fields_ = [("rel_dS", ctypes.c_double), ("rel_dS_gamma", ctypes.c_double),
                ("rel_dv0", ctypes.c_double), ("abs_dr", ctypes.c_double),
                ("abs_dT", ctypes.c_double), ("greek_mask", ctypes.c_uint32),
                ("pad_", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("price", "price_se", "delta", "gamma", "vega", "rho", "theta",
                 "european_price")] + [
        ("n_singular", ctypes.c_uint32), ("n_revaluations", ctypes.c_uint32),
        ("status", ctypes.c_int32), ("pad_", ctypes.c_int32)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if f[0] != "pad_"}


class TieCtl(ctypes.Structure):
    _fields_ = [("tie_rel", ctypes.c_double), ("ties", ctypes.POINTER(ctypes.c_uint64)),
                ("max_ties", ctypes.c_uint32), ("n_ties", ctypes.c_uint32),
                ("flips", ctypes.POINTER(ctypes.c_uint64)), ("n_flips", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    with _lock:
        stale = force or not os.path.exists(_SO) or any(
            os.path.getmtime(s) > os.path.getmtime(_SO) for s in _SRC)
        if stale:
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _SO + ".%d.tmp" % os.getpid()
            subprocess.check_call(
                ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                 "-shared", "-o", tmp, _SRC[0], "-lm", "-lpthread"])
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_philox_n.argtypes = [u32p, u32p, u32p, ctypes.c_size_t]
        L.orc_norm_inv_n.argtypes = [dp, dp, ctypes.c_size_t]
        L.orc_draws_n.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p, u32p,
                                  ctypes.c_size_t, ctypes.c_int, dp]
        L.orc_uniform_f64.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.orc_uniform_f64.restype = ctypes.c_double
        L.orc_uniform_f32.argtypes = [ctypes.c_uint32]
        L.orc_uniform_f32.restype = ctypes.c_double
        L.orc_norm_inv.argtypes = [ctypes.c_double]
        L.orc_norm_inv.restype = ctypes.c_double
        L.orc_qe_step.argtypes = [ctypes.POINTER(Heston)] + [ctypes.c_double] * 6 + [dp]
        L.orc_ft_step.argtypes = [ctypes.POINTER(Heston)] + [ctypes.c_double] * 5 + [dp]
        L.orc_paths.argtypes = [ctypes.POINTER(Heston), ctypes.c_double, ctypes.c_int,
                                ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_uint64, ctypes.c_uint32, dp, dp, ctypes.c_int]
        L.orc_path_one.argtypes = [ctypes.POINTER(Heston), ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_uint32, dp, dp]
        L.orc_multi_max.argtypes = [ctypes.POINTER(Heston), ctypes.c_uint32, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.c_uint32, dp, ctypes.c_int]
        L.orc_asset_path.argtypes = [ctypes.POINTER(Heston), ctypes.c_uint32, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_uint32, dp]
        L.orc_lsmc_oos.argtypes = [dp, dp, dp, dp, ctypes.c_uint32, ctypes.c_uint32] + \
            [ctypes.c_double] * 5 + [ctypes.c_int] * 3 + [dp, u32p]
        L.orc_price_greeks_ex.argtypes = [
            ctypes.POINTER(Heston), ctypes.c_int, ctypes.c_int, ctypes.c_double,
            dp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.POINTER(Bumps), ctypes.c_uint64,
            ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Result), dp]
        L.orc_dual_bound.argtypes = [
            ctypes.POINTER(Heston), ctypes.c_int, ctypes.c_double, dp, ctypes.c_uint32,
            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, dp]
        L.orc_round_f16.argtypes = [ctypes.c_double]
        L.orc_round_f16.restype = ctypes.c_double
        L.orc_round_bf16.argtypes = [ctypes.c_double]
        L.orc_round_bf16.restype = ctypes.c_double
        L.orc_round_n.argtypes = [dp, dp, ctypes.c_size_t, ctypes.c_int]
        L.orc_lsmc.argtypes = [dp, dp, ctypes.c_uint32, ctypes.c_uint32] + \
            [ctypes.c_double] * 5 + [ctypes.c_int] * 3 + \
            [dp, u32p, dp, ctypes.POINTER(ctypes.c_uint8)]
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.orc_lsmc_tie.argtypes = [dp, dp, ctypes.c_uint32, ctypes.c_uint32] + \
            [ctypes.c_double] * 5 + [ctypes.c_int] * 3 + [dp, u32p, ctypes.POINTER(TieCtl)]
        L.orc_greeks_from_values.argtypes = [ctypes.POINTER(Heston), ctypes.POINTER(Bumps),
                                             ctypes.POINTER(ctypes.c_int), dp, ctypes.c_int,
                                             ctypes.POINTER(Result)]
        L.orc_greeks_from_values.restype = None
        L.orc_scenario_alternatives.argtypes = [
            ctypes.POINTER(Heston), ctypes.c_int, ctypes.c_int, ctypes.c_double,
            ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, ctypes.POINTER(Bumps), ctypes.c_uint64, ctypes.c_uint32,
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, u64p,
            ctypes.c_uint32, dp, u64p, ctypes.c_uint32, u32p, ctypes.c_int]
        L.orc_scenarios.argtypes = [ctypes.POINTER(Heston), ctypes.c_double,
                                    ctypes.POINTER(Bumps), ctypes.POINTER(Heston),
                                    dp, ctypes.POINTER(ctypes.c_int)]
        L.orc_price_greeks.argtypes = [
            ctypes.POINTER(Heston), ctypes.c_int, ctypes.c_int, ctypes.c_double,
            dp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.POINTER(Bumps), ctypes.c_uint64,
            ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(Result), dp]
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def heston(**kw) -> Heston:
    return Heston(**kw)


def bumps(rel_dS=0.01, rel_dS_gamma=0.0, rel_dv0=0.01, abs_dr=1e-3,
          abs_dT=1.0 / 252.0, greek_mask=DELTA | GAMMA | VEGA) -> Bumps:
    return Bumps(rel_dS, rel_dS_gamma, rel_dv0, abs_dr, abs_dT, greek_mask, 0)


def philox(ctr, key):
    """ctr: (n, 4) uint32; key: (2,) uint32 -> (n, 4) uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    lib().orc_philox_n(_ptr(ctr, ctypes.c_uint32), _ptr(key, ctypes.c_uint32),
                       _ptr(out, ctypes.c_uint32), ctr.shape[0])
    return out


def uniform_f64(hi, lo):
    return lib().orc_uniform_f64(int(hi), int(lo))


def uniform_f32(w):
    return lib().orc_uniform_f32(int(w))


def norm_inv(u):
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    z = np.empty_like(u)
    lib().orc_norm_inv_n(_ptr(u, ctypes.c_double), _ptr(z, ctypes.c_double), u.size)
    return z


def draws(seed, stream, path, step, grid=GRID_F64):
    """(U_V, Z_V, Z_X) per (path, step): returns (n, 3) float64."""
    path = np.ascontiguousarray(path, dtype=np.uint32).reshape(-1)
    step = np.ascontiguousarray(step, dtype=np.uint32).reshape(-1)
    assert path.size == step.size
    out = np.empty((path.size, 3), dtype=np.float64)
    lib().orc_draws_n(seed, stream, _ptr(path, ctypes.c_uint32),
                      _ptr(step, ctypes.c_uint32), path.size, grid,
                      _ptr(out, ctypes.c_double))
    return out


def qe_step(model: Heston, dt, x, v, uV, zV, zX):
    out = (ctypes.c_double * 2)()
    lib().orc_qe_step(ctypes.byref(model), dt, x, v, uV, zV, zX, out)
    return out[0], out[1]


def ft_step(model: Heston, dt, x, v, zV, zX):
    out = (ctypes.c_double * 3)()
    lib().orc_ft_step(ctypes.byref(model), dt, x, v, zV, zX, out)
    return out[0], out[1], out[2]


def paths(model: Heston, T, scheme, P, N, seed, stream=0, grid=GRID_F64,
          n_threads=None):
    """S, V of shape (N + 1, P)."""
    S = np.empty((N + 1, P), dtype=np.float64)
    V = np.empty((N + 1, P), dtype=np.float64)
    rc = lib().orc_paths(ctypes.byref(model), T, scheme, grid, P, N, seed, stream,
                         _ptr(S, ctypes.c_double), _ptr(V, ctypes.c_double),
                         n_threads or default_threads())
    if rc != 0:
        raise ValueError("orc_paths rejected its arguments (%d)" % rc)
    return S, V


def multi_max(models, T, scheme, P, N, seed, stream=0, rho_assets=0.0, grid=GRID_F64,
              n_threads=None):
    """STAC-A2 path reduction: M of shape (N + 1, P), the largest of the
    assets' values per path and date (models: a sequence of Heston)."""
    arr = (Heston * len(models))(*models)
    M = np.empty((N + 1, P), dtype=np.float64)
    rc = lib().orc_multi_max(arr, len(models), T, scheme, grid, rho_assets, P, N, seed, stream,
                             _ptr(M, ctypes.c_double), n_threads or default_threads())
    if rc != 0:
        raise ValueError("orc_multi_max rejected its arguments (%d)" % rc)
    return M


def asset_path(model: Heston, asset, T, scheme, path, N, seed, stream=0, rho_assets=0.0,
               grid=GRID_F64):
    """S of one asset of one multi-asset path, length N + 1."""
    S = np.empty(N + 1, dtype=np.float64)
    rc = lib().orc_asset_path(ctypes.byref(model), asset, T, scheme, grid, rho_assets, path, N,
                              seed, stream, _ptr(S, ctypes.c_double))
    if rc != 0:
        raise ValueError("orc_asset_path rejected its arguments (%d)" % rc)
    return S


def path_one(model: Heston, T, scheme, path, N, seed, stream=0, grid=GRID_F64):
    """S, V of one path (index `path`), each of length N + 1."""
    S = np.empty(N + 1, dtype=np.float64)
    V = np.empty(N + 1, dtype=np.float64)
    rc = lib().orc_path_one(ctypes.byref(model), T, scheme, grid, path, N, seed, stream,
                            _ptr(S, ctypes.c_double), _ptr(V, ctypes.c_double))
    if rc != 0:
        raise ValueError("orc_path_one rejected its arguments (%d)" % rc)
    return S, V


def lsmc(S, V, S0, K, T, r, theta, type_=PUT, style=AMERICAN, basis=BASIS_S2,
         want_detail=False, tie_rel=None, flips=()):
    """Backward induction over given paths.  Returns a dict with price,
    price_se, european_price, continuation, n_singular and (optionally)
    beta (N, 6) and exercise (N, P).  tie_rel: also report the keys n P + p
    of the near-tie decisions (|h - c| <= tie_rel max(|c|, h)) as
    "near_ties"; flips: keys of decisions to take the other way."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    N = S.shape[0] - 1
    P = S.shape[1]
    out = (ctypes.c_double * 4)()
    ns = ctypes.c_uint32(0)
    if tie_rel is not None or len(flips):
        assert not want_detail
        cap = 4096
        ties = (ctypes.c_uint64 * cap)()
        fl = np.ascontiguousarray(sorted(int(k) for k in flips), dtype=np.uint64)
        ctl = TieCtl(-1.0 if tie_rel is None else tie_rel, ties, cap, 0,
                     _ptr(fl, ctypes.c_uint64) if fl.size else None, fl.size)
        rc = lib().orc_lsmc_tie(_ptr(S, ctypes.c_double), _ptr(V, ctypes.c_double), P, N,
                                S0, K, T, r, theta, type_, style, basis, out, ctypes.byref(ns),
                                ctypes.byref(ctl))
        if rc != 0:
            raise ValueError("orc_lsmc_tie rejected its arguments (%d)" % rc)
        return {"price": out[0], "price_se": out[1], "european_price": out[2],
                "continuation": out[3], "n_singular": ns.value,
                "near_ties": [ties[i] for i in range(min(ctl.n_ties, cap))],
                "n_near_ties": ctl.n_ties}
    beta = np.empty((N, 6), dtype=np.float64) if want_detail else None
    ex = np.empty((N, P), dtype=np.uint8) if want_detail else None
    rc = lib().orc_lsmc(_ptr(S, ctypes.c_double), _ptr(V, ctypes.c_double), P, N,
                        S0, K, T, r, theta, type_, style, basis, out,
                        ctypes.byref(ns),
                        _ptr(beta, ctypes.c_double) if want_detail else None,
                        _ptr(ex, ctypes.c_uint8) if want_detail else None)
    if rc != 0:
        raise ValueError("orc_lsmc rejected its arguments (%d)" % rc)
    d = {"price": out[0], "price_se": out[1], "european_price": out[2],
         "continuation": out[3], "n_singular": ns.value}
    if want_detail:
        d["beta"] = beta
        d["exercise"] = ex
    return d


def lsmc_oos(SA, VA, SB, VB, S0, K, T, r, theta, type_=PUT, style=AMERICAN, basis=BASIS_S2):
    """Out-of-sample estimate: the policy of the regressions on (SA, VA)
    applied to (SB, VB).  Returns a dict like lsmc."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (SA, VA, SB, VB)]
    N, P = arrs[0].shape[0] - 1, arrs[0].shape[1]
    out = (ctypes.c_double * 4)()
    ns = ctypes.c_uint32(0)
    rc = lib().orc_lsmc_oos(*[_ptr(a, ctypes.c_double) for a in arrs], P, N, S0, K, T, r,
                            theta, type_, style, basis, out, ctypes.byref(ns))
    if rc != 0:
        raise ValueError("orc_lsmc_oos rejected its arguments (%d)" % rc)
    return {"price": out[0], "price_se": out[1], "european_price": out[2],
            "continuation": out[3], "n_singular": ns.value}


def scenarios(model: Heston, T, b: Bumps):
    models = (Heston * 11)()
    Ts = (ctypes.c_double * 11)()
    kinds = (ctypes.c_int * 11)()
    n = lib().orc_scenarios(ctypes.byref(model), T, ctypes.byref(b), models, Ts, kinds)
    if n < 0:
        raise ValueError("orc_scenarios rejected its arguments (%d)" % n)
    return [(SC_KINDS[kinds[i]], models[i], Ts[i]) for i in range(n)]


STORE_NATIVE, STORE_F16, STORE_BF16 = 0, 1, 2


def round_store(x, store):
    """x (array of doubles) rounded to nearest, ties to even, to binary16
    (store = STORE_F16) or bfloat16 (STORE_BF16), returned as doubles."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().orc_round_n(_ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double), x.size, int(store))
    return y


def dual_bound(model: Heston, strikes, T, P, N, n_outer, n_inner, *, type_=PUT, scheme=QE,
               grid=GRID_F64, basis=BASIS_S2, seed=42, stream=0, n_threads=None):
    """Lower (out-of-sample) and dual upper bounds of the American price per
    strike: list of dicts lower, lower_se, upper, upper_se, pi_N, pi_N_se."""
    strikes = np.ascontiguousarray(strikes, dtype=np.float64).reshape(-1)
    out = np.empty(6 * strikes.size, dtype=np.float64)
    rc = lib().orc_dual_bound(ctypes.byref(model), type_, T, _ptr(strikes, ctypes.c_double),
                              strikes.size, P, N, scheme, grid, basis, seed, stream, n_outer,
                              n_inner, n_threads or default_threads(), _ptr(out, ctypes.c_double))
    if rc != 0:
        raise ValueError("orc_dual_bound rejected its arguments (%d)" % rc)
    names = ("lower", "lower_se", "upper", "upper_se", "pi_N", "pi_N_se")
    return [dict(zip(names, out[6 * k: 6 * k + 6])) for k in range(strikes.size)]


def greeks_from_values(model: Heston, b: Bumps, kinds, values):
    """Price and Greeks from revaluation prices: kinds (names of SC_KINDS)
    and values, one per scenario of the table."""
    n = len(kinds)
    k = (ctypes.c_int * n)(*[SC_KINDS.index(x) for x in kinds])
    v = (ctypes.c_double * n)(*values)
    res = Result()
    lib().orc_greeks_from_values(ctypes.byref(model), ctypes.byref(b), k, v, n,
                                 ctypes.byref(res))
    return res.as_dict()


def scenario_alternatives(model: Heston, K, T, P, N, sc, *, type_=PUT, style=AMERICAN,
                          scheme=QE, grid=GRID_F64, basis=BASIS_S2, b: Bumps | None = None,
                          seed=42, stream=0, out_of_sample=False, store=STORE_NATIVE,
                          tie_rel=1e-9, keys=(), n_threads=None):
    """Revaluation `sc` (index into the scenario table) of strike K as
    price_greeks simulates it: (prices, near_ties) with prices[i] the price
    when the decisions of `keys` whose bit is set in i (bit j = the j-th
    smallest key) are taken the other way, and near_ties the keys of the
    plain run's near-tie decisions at tie_rel."""
    b = b or bumps()
    keys = sorted(int(x) for x in keys)
    assert len(keys) <= MAX_ALT_KEYS
    kk = (ctypes.c_uint64 * max(1, len(keys)))(*keys)
    out = (ctypes.c_double * (1 << len(keys)))()
    cap = 4096
    ties = (ctypes.c_uint64 * cap)()
    nt = ctypes.c_uint32(0)
    rc = lib().orc_scenario_alternatives(
        ctypes.byref(model), type_, style, T, K, P, N, scheme, grid, basis, ctypes.byref(b),
        seed, stream, 1 if out_of_sample else 0, int(store), sc, tie_rel, kk, len(keys), out,
        ties, cap, ctypes.byref(nt), n_threads or default_threads())
    if rc != 0:
        raise ValueError("orc_scenario_alternatives rejected its arguments (%d)" % rc)
    return list(out), [ties[i] for i in range(min(nt.value, cap))]


def price_greeks(model: Heston, strikes, T, P, N, *, type_=PUT, style=AMERICAN,
                 scheme=QE, grid=GRID_F64, basis=BASIS_S2, b: Bumps | None = None,
                 seed=42, stream=0, n_threads=None, want_scenarios=False,
                 out_of_sample=False, store=STORE_NATIVE):
    """Price and Greeks for each strike (list of dicts); out_of_sample: the
    policy of the regressions on `stream` priced on stream ^ 0x80000000;
    store: STORE_F16 / STORE_BF16 for a 16-bit path store (exp(x) and v
    rounded to the format, a rate bump reading the base simulation's
    values times exp(+-dr t_n))."""
    b = b or bumps()
    strikes = np.ascontiguousarray(strikes, dtype=np.float64).reshape(-1)
    nk = strikes.size
    res = (Result * nk)()
    scen = np.empty(11 * nk, dtype=np.float64)
    rc = lib().orc_price_greeks_ex(ctypes.byref(model), type_, style, T,
                                   _ptr(strikes, ctypes.c_double), nk, P, N, scheme,
                                   grid, basis, ctypes.byref(b), seed, stream,
                                   1 if out_of_sample else 0, int(store),
                                   n_threads or default_threads(), res,
                                   _ptr(scen, ctypes.c_double))
    if rc != 0:
        raise ValueError("orc_price_greeks rejected its arguments (%d)" % rc)
    out = [res[i].as_dict() for i in range(nk)]
    if want_scenarios:
        n_sc = out[0]["n_revaluations"]
        return out, scen[: n_sc * nk].reshape(n_sc, nk)
    return out
