"""Helpers shared by the GPU parity tests."""
import math

import numpy as np
import pytest

import oracle
from paper_2206_03719_gb300 import workloads

_GREEK = {"delta": oracle.DELTA, "gamma": oracle.GAMMA, "vega": oracle.VEGA,
          "rho": oracle.RHO, "theta": oracle.THETA}
KEYS = ("price", "delta", "gamma", "vega", "rho", "theta", "european_price")


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def oracle_for(wl, grid=oracle.GRID_F64, n_threads=None):
    mask = 0
    for g in wl.greeks:
        mask |= _GREEK[g]
    b = oracle.bumps(rel_dS=wl.rel_dS, rel_dS_gamma=wl.rel_dS_gamma, rel_dv0=wl.rel_dv0,
                     abs_dr=wl.abs_dr, abs_dT=wl.abs_dT, greek_mask=mask)
    return oracle.price_greeks(
        oracle.heston(**wl.model), wl.strikes, wl.T, wl.n_paths, wl.n_steps,
        type_=oracle.PUT if wl.option == "put" else oracle.CALL,
        style=oracle.AMERICAN if wl.style == "american" else oracle.EUROPEAN,
        scheme=oracle.QE if wl.scheme == "qe" else oracle.FT_EULER, grid=grid,
        basis=oracle.BASIS_S2 if wl.basis == "s2" else oracle.BASIS_SV2, b=b, seed=wl.seed,
        stream=wl.stream, n_threads=n_threads, out_of_sample=wl.out_of_sample,
        store={"native": oracle.STORE_NATIVE, "fp16": oracle.STORE_F16,
               "bf16": oracle.STORE_BF16}[wl.store])


FP64_TOL = 1e-10     # FP64 GPU vs FP64 oracle on identical streams
FLIP_TOL = 1e-4      # the same when near-tie exercise decisions occurred


def parity_tol(n_near_ties):
    """1e-10 when no exercise decision was within rounding reach of its
    threshold (then both implementations must take the same decisions);
    otherwise decisions may legitimately differ and each difference moves a
    price at first order: the bound falls back to 1e-4."""
    return FP64_TOL if int(n_near_ties) == 0 else FLIP_TOL


def rel_err(a, b):
    """|a - b| / max(|b|, 1e-12); NaN on both sides counts as equal."""
    if math.isnan(b) and math.isnan(a):
        return 0.0
    return abs(a - b) / max(abs(b), 1e-12)


# central-difference denominators of the Greeks for 1% / 2% S bumps, 1% v0,
# 1e-3 r and 1/252 T bumps with S0 = 100, v0 = 0.04: rounding noise of the
# scenario prices, divided by these, is the floor below which a Greek
# difference carries no information
_DENOM = {"delta": 2.0, "gamma": 1.0, "vega": 8e-4, "rho": 2e-3, "theta": 2.0 / 252}


def assert_close(got, ref, tol, keys=KEYS, what=""):
    errs = {}
    scale = max(abs(ref.get("price", 1.0)), 1e-2)
    for k in keys:
        # a Greek is compared relative to itself or, when it is much smaller
        # than the price differences it is made of, to price / denominator
        floor = scale / _DENOM.get(k, 1.0)
        e = abs(got[k] - ref[k]) / max(abs(ref[k]), floor) if not (
            math.isnan(got[k]) and math.isnan(ref[k])) else 0.0
        errs[k] = e
        assert e <= tol, "%s %s: got %.15g ref %.15g rel %.3g" % (what, k, got[k], ref[k], e)
    return errs
