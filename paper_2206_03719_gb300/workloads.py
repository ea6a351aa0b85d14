"""Seeded synthetic workloads shared by the tests, the smoke check and the
benchmark.

This module holds only input descriptions and seeded generators of inputs
(contract books, request arrival times).  It contains none of the method's
arithmetic and imports neither the CUDA binding nor the oracle, so both sides
of every parity test take their inputs from here.

The paper measures on the licensed STAC-A2 workload (Table 1: 5-50 assets,
126-1260 daily steps, 25k paths); these single-asset Heston books stand in
for it with its step counts and path counts of the same order.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Heston dynamics of the single-asset American put workloads
HESTON_BASE = dict(S0=100.0, r=0.02, q=0.0, v0=0.04, kappa=1.5, theta=0.04,
                   xi=0.3, rho=-0.7)

ALL_GREEKS = ("delta", "gamma", "vega", "rho", "theta")


@dataclasses.dataclass
class Workload:
    """One pricing request: Heston model, a contract family sharing one path
    set (several strikes), simulation size and bump specification."""
    name: str
    model: dict
    strikes: List[float]
    T: float
    n_paths: int
    n_steps: int
    option: str = "put"          # "put" | "call"
    style: str = "american"      # "american" | "european"
    basis: str = "s2"            # "s2" = {1,S,S^2}; "sv2" = {1,S,S^2,v,Sv,v^2}
    scheme: str = "qe"           # "qe" (Andersen) | "ft_euler"
    precision: str = "fp64"      # "fp64" | "mixed"
    greeks: tuple = ("delta", "gamma", "vega")
    rel_dS: float = 0.01
    rel_dS_gamma: float = 0.0    # 0: gamma shares the delta pair
    rel_dv0: float = 0.01
    abs_dr: float = 1e-3
    abs_dT: float = 1.0 / 252.0
    seed: int = 42
    stream: int = 0
    regenerate: bool = False     # no path store: regenerate segments from checkpoints
    out_of_sample: bool = False  # price the regression policy on independent paths
    store: str = "native"        # path store element: "native", "fp16" or "bf16"

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)

    @property
    def n_scenarios(self) -> int:
        g = set(self.greeks)
        gamma_shares = self.rel_dS_gamma in (0.0, self.rel_dS)
        n = 1
        if "delta" in g or ("gamma" in g and gamma_shares):
            n += 2
        if "gamma" in g and not gamma_shares:
            n += 2
        n += 2 * sum(1 for k in ("vega", "rho", "theta") if k in g)
        return n

    @property
    def generated_path_steps(self) -> int:
        return self.n_scenarios * self.n_paths * self.n_steps

    @property
    def lsmc_path_steps(self) -> int:
        return self.generated_path_steps * len(self.strikes)

    @property
    def n_greeks(self) -> int:
        return len(self.strikes) * len(self.greeks)


# American put, 4096 paths x 32 exercise dates, basis {1,S,S^2}, FP64,
# price + delta/gamma/vega by central 1% bumps (5 revaluations)
SMALL_FP64 = Workload(
    name="american-put-heston-4096x32-fp64", model=dict(HESTON_BASE),
    strikes=[100.0], T=1.0, n_paths=4096, n_steps=32, basis="s2",
    greeks=("delta", "gamma", "vega"), rel_dS=0.01, rel_dS_gamma=0.0)

# American puts K in {80..120}, 131072 paths x 252 steps, basis
# {1,S,S^2,v,Sv,v^2}, FP64, all five Greeks (11 revaluations per strike)
PAPER_FP64 = Workload(
    name="american-put-heston-131072x252-5strikes-fp64",
    model=dict(HESTON_BASE), strikes=[80.0, 90.0, 100.0, 110.0, 120.0], T=1.0,
    n_paths=131072, n_steps=252, basis="sv2", greeks=ALL_GREEKS,
    rel_dS=0.01, rel_dS_gamma=0.02)

# the same book at 1,048,576 paths with FP32 paths and FP64 reductions
LARGE_MIXED = PAPER_FP64.replace(
    name="american-put-heston-1048576x252-5strikes-mixed", n_paths=1048576,
    precision="mixed")


def book(n_contracts: int = 512, seed: int = 2206_03719,
         paths_lo: int = 4096, paths_hi: int = 262144,
         steps=(50, 100, 252, 500), tile: int = 128,
         precision: str = "mixed") -> List[Workload]:
    """Uneven book of American puts and calls with per-contract Heston
    parameters (numpy PCG64 draws): K ~ U[70,130], T ~ U[0.25,2],
    kappa ~ U[0.5,3], theta ~ U[0.02,0.09], xi ~ U[0.1,0.6],
    rho ~ U[-0.9,-0.3], paths log-uniform in [4k, 256k] rounded to a multiple
    of `tile`, steps drawn from `steps`; all five Greeks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_contracts):
        K = float(rng.uniform(70.0, 130.0))
        T = float(rng.uniform(0.25, 2.0))
        kappa = float(rng.uniform(0.5, 3.0))
        theta = float(rng.uniform(0.02, 0.09))
        xi = float(rng.uniform(0.1, 0.6))
        rho = float(rng.uniform(-0.9, -0.3))
        lp = rng.uniform(math.log(paths_lo), math.log(paths_hi))
        P = int(round(math.exp(lp) / tile)) * tile
        P = min(max(P, paths_lo), paths_hi)
        N = int(steps[int(rng.integers(0, len(steps)))])
        opt = "put" if rng.integers(0, 2) == 0 else "call"
        model = dict(HESTON_BASE, kappa=kappa, theta=theta, xi=xi, rho=rho)
        out.append(Workload(
            name="book-%03d" % i, model=model, strikes=[K], T=T, n_paths=P,
            n_steps=N, option=opt, basis="s2", greeks=ALL_GREEKS,
            rel_dS=0.01, rel_dS_gamma=0.02, precision=precision, seed=42,
            stream=i))
    return out


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int = 7,
                     max_requests: Optional[int] = None) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps, seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t > duration_s or (max_requests and len(out) >= max_requests):
            break
        out.append(t)
    return np.asarray(out)


# ---- STAC-A2 path reduction: the paper's problem sizes (Table 1) ------------
# (assets, daily dates) at 25,000 paths; one trading day per date, so the
# horizon is dates / 252 years.
STAC_SIZES = {"tiny": (5, 126), "small": (10, 126), "medium": (20, 252),
              "large": (30, 504), "huge": (50, 1260)}
STAC_PATHS = 25_000


def stac_models(n_assets: int, seed: int = 2022):
    """Heston models of the assets of a STAC-A2 path reduction (the paper's
    per-asset configurations are not published): drawn with numpy PCG64 --
    S0 ~ U[80, 120], q ~ U[0, 0.03], v0 ~ U[0.01, 0.09], kappa ~ U[0.5, 3],
    theta ~ U[0.02, 0.09], xi ~ U[0.1, 0.8], rho ~ U[-0.9, -0.3], r = 0.02."""
    rng = np.random.default_rng(seed)
    return [dict(S0=float(rng.uniform(80, 120)), r=0.02, q=float(rng.uniform(0, 0.03)),
                 v0=float(rng.uniform(0.01, 0.09)), kappa=float(rng.uniform(0.5, 3.0)),
                 theta=float(rng.uniform(0.02, 0.09)), xi=float(rng.uniform(0.1, 0.8)),
                 rho=float(rng.uniform(-0.9, -0.3)))
            for _ in range(n_assets)]
