"""Writes the stored expected values of tests/golden/ by running the FP64
oracle (oracle/) on the seeded synthetic workloads.  Nothing else is called:
every number in the JSON files comes from the oracle.

    python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

_ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
from paper_2206_03719_gb300 import workloads  # noqa: E402

_GREEK = {"delta": oracle.DELTA, "gamma": oracle.GAMMA, "vega": oracle.VEGA,
          "rho": oracle.RHO, "theta": oracle.THETA}


def run_oracle(wl, grid=oracle.GRID_F64, n_threads=None):
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
        stream=wl.stream, n_threads=n_threads, want_scenarios=True)


# the book and serving subsets: seeded contract indices of the uneven book
# (512 contracts) and the first requests of the served stream, whose oracle
# values state the error of the batched and served forms
BOOK_SUBSET = sorted(int(i) for i in
                     __import__("numpy").random.default_rng(32).choice(512, 32, replace=False))
SERVING_SUBSET = list(range(32))


def _contract_results(wls):
    out = []
    for wl in wls:
        t = time.time()
        res = run_oracle(wl)[0][0]
        out.append({"name": wl.name, "results": res, "seconds": time.time() - t})
    return out


SUBSETS = {
    "book_subset": lambda: [workloads.book(n_contracts=512)[i] for i in BOOK_SUBSET],
    "serving_subset": lambda: workloads.book(n_contracts=max(SERVING_SUBSET) + 1,
                                             seed=99)[:len(SERVING_SUBSET)],
}

GOLDEN = {
    # American puts K = 80..120, 131072 paths x 252 steps, SV2 basis, QE, all Greeks
    "paper_fp64": workloads.PAPER_FP64,
    # the same book under full-truncation Euler
    "paper_fp64_ft": workloads.PAPER_FP64.replace(scheme="ft_euler"),
}


def main(names):
    here = os.path.dirname(os.path.abspath(__file__))
    for name in names or list(GOLDEN) + list(SUBSETS):
        if name in SUBSETS:
            t = time.time()
            wls = SUBSETS[name]()
            out = {"indices": BOOK_SUBSET if name == "book_subset" else SERVING_SUBSET,
                   "source": "oracle/oracle.c (FP64)",
                   "contracts": _contract_results(wls)}
            with open(os.path.join(here, name + ".json"), "w") as f:
                json.dump(out, f, indent=1)
            print(name, "%.1f s" % (time.time() - t))
            continue
        wl = GOLDEN[name]
        t = time.time()
        res, scen = run_oracle(wl)
        # the revaluations behind each strike's Greeks, by scenario kind
        kinds = [k for k, _, _ in oracle.scenarios(
            oracle.heston(**wl.model), wl.T,
            oracle.bumps(rel_dS=wl.rel_dS, rel_dS_gamma=wl.rel_dS_gamma, rel_dv0=wl.rel_dv0,
                         abs_dr=wl.abs_dr, abs_dT=wl.abs_dT,
                         greek_mask=sum(_GREEK[g] for g in wl.greeks)))]
        for k, r in enumerate(res):
            r["scenarios"] = {kind: float(scen[s][k]) for s, kind in enumerate(kinds)}
        out = {"workload": wl.name, "scheme": wl.scheme, "n_paths": wl.n_paths,
               "n_steps": wl.n_steps, "strikes": wl.strikes, "source": "oracle/oracle.c (FP64)",
               "results": res}
        with open(os.path.join(here, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, "%.1f s" % (time.time() - t))


if __name__ == "__main__":
    main(sys.argv[1:])
