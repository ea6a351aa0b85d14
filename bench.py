"""Benchmark: Heston / Longstaff-Schwartz price + full Greeks on one GB300.

One step = the whole path of the workload (Philox + normals + Heston paths
for every path group, Longstaff-Schwartz over every scenario x strike,
estimator and finite-difference Greeks) for the American-put book of
131,072 paths x 252 steps, strikes {80, 90, 100, 110, 120}, basis
{1, S, S^2, v, Sv, v^2}, 11 revaluations per strike, FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Under torchrun (N > 1) every rank prices its own
replica of the workload on its own random stream (replicas only: the path
needs no exchange) and rank 0 reports the units of all ranks over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

_ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, _ROOT)

from paper_2206_03719_gb300 import workloads  # noqa: E402

GOLDEN = os.path.join(_ROOT, "tests", "golden", "paper_fp64.json")
GOLDEN_BOOK = os.path.join(_ROOT, "tests", "golden", "book_subset.json")
GOLDEN_SERVING = os.path.join(_ROOT, "tests", "golden", "serving_subset.json")
PEAKS = os.path.join(_ROOT, "MEASURED_PEAKS.json")
# algorithmic work of the stepper (forward pass), counted from the formulas
# of the scheme (a fused multiply-add counts 2 flops; elementary functions --
# division, square root, exponential, logarithm -- counted apart, each one
# evaluation on the special-function unit in single precision):
#   per simulated path-step, shared by the contract's path groups: the two
#   uniforms (2 flops each), 1 - U (1), two normal quantiles (a degree-8
#   polynomial, 18 flops, and one logarithm each)                -> 41 flops, 2 functions
#   per path group, QE: m and s^2 (4), m^2, the branch test and its
#   quadratic-branch arithmetic (11 with the two divisions' products), the
#   log-price step (9), S0 exp(x) (2); two divisions, three square roots and
#   one exponential                                              -> 26 flops, 6 functions
#   per path group, full-truncation Euler: 11 flops, one square root, plus
#   S0 exp(x) (2 flops, one exponential)                         -> 13 flops, 2 functions
#   stored per path group: exp(x) and, with the SV2 basis, v.
# measured peaks of this run (set by main before the side measurements)
RUN = {"peaks": {}, "hbm_gbs": None}
STEP_SHARED = {"flops": 41, "functions": 2}
STEP_GROUP = {"qe": {"flops": 26, "functions": 6}, "ft_euler": {"flops": 13, "functions": 2}}
# algorithmic FP64 operations of the backward pass (a fused multiply-add
# counts as two):
#   every (instance, path, date): S = scale*E, payoff, discount      -> 3
#   in-the-money moment sums (SV2): x, w, 12 monomial products,
#     15 monomial adds, 5 products + 6 adds for X^T y                 -> 40
#   in-the-money exercise test at the next date: S, payoff, x, w,
#     5 multiply-adds for the continuation value, compare             -> 15
BWD_FLOPS_ALL = 3
BWD_FLOPS_ITM = 40 + 15
# DRAM bytes of one FP64 backward launch on the 131,072-path book, from an
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the same
# kernel at 98,304 paths (3.110958e9 + 0.348644e9 bytes) scaled by the path
# count (the path store and cash flows grow in proportion).  Valid only for
# the kernel source and the tile shape it was taken with (sub-tiles per job
# with LSMC_SUB_ITM_HALF, paths per lane): reported as null once the code of
# backward.cu changes (code_sha256_16) or the bench runs another shape.
BWD_TRAFFIC = {"bytes": (3.110957824e9 + 0.348643840e9) * 131072 / 98304,
               "source_sha256_16": "9312333d9ec49f23",
               "shape": (32 | 0x8000, 2),
               "capture": "profiles/backward_kernel_fp64_98304x252.md (traffic capture), "
                          "scaled by 131072/98304"}


def code_sha256_16(path):
    """The first 16 hex digits of the SHA-256 of a source file's code: every
    line with its // comment and trailing blanks removed, blank lines
    dropped (so edits of comments alone keep the hash)."""
    lines = []
    for line in open(path, encoding="utf-8"):
        code = line.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="paper_fp64",
                    choices=["paper_fp64", "large_mixed", "paper_mixed", "paper_df", "small",
                             "book_subset"],
                    help="book_subset serves --cpu-full only")
    ap.add_argument("--paths", type=int, default=0,
                    help="override the path count (profiling of a smaller case)")
    ap.add_argument("--sub", type=int, default=0,
                    help="backward sub-tiles per job; 0 = pick by the autotuner")
    ap.add_argument("--ppt", type=int, default=0,
                    help="backward paths per lane with --sub (0 = the precision's default)")
    ap.add_argument("--itm-half", action="store_true",
                    help="with --sub: half the sub-tiles per job for strikes in the money at S0")
    ap.add_argument("--regenerate", action="store_true",
                    help="no path store: regenerate segments from saved states")
    ap.add_argument("--out-of-sample", action="store_true",
                    help="price the regression policy on independent paths")
    ap.add_argument("--store", default="native", choices=["native", "fp16", "bf16"],
                    help="element type of the path store")
    ap.add_argument("--extra", default="",
                    help="run only this side measurement and print it (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--peaks", action="store_true",
                    help="print the measured pipe throughputs (lsmc_measure_peaks) and exit")
    ap.add_argument("--cpu-full", action="store_true",
                    help="time the FP64 oracle once on the whole workload (all paths) and exit")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the precision-split, book and serving measurements")
    return ap.parse_args()


def pick_workload(name):
    if name == "small":
        return workloads.SMALL_FP64
    if name == "paper_fp64":
        return workloads.PAPER_FP64
    if name == "paper_df":
        return workloads.PAPER_FP64.replace(precision="df",
                                            name="american-put-heston-131072x252-5strikes-df")
    if name == "paper_mixed":
        return workloads.PAPER_FP64.replace(precision="mixed",
                                            name="american-put-heston-131072x252-5strikes-mixed")
    return workloads.LARGE_MIXED


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_workload(wl, rank):
    """The workload rank `rank` prices: the same request on its own random
    stream (stream id + rank), an independent Monte Carlo replica of the same
    size.  Rank 0 keeps the stream the stored oracle values were taken on."""
    if rank == 0:
        return wl
    return wl.replace(stream=wl.stream + rank)


def max_over_ranks(ms, dist, device):
    """The slowest rank's step time (every rank gets it); ms itself alone."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, ms_max):
    """Units all ranks processed per second of the slowest rank's step."""
    return world * units_per_rank / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def oracle_sample_rate(wl, sample_paths, threads=None):
    """Time the FP64 oracle on the workload with sample_paths paths; return
    (seconds, Greeks/s scaled to the full path count, cores used)."""
    sys.path.insert(0, os.path.join(_ROOT, "tests"))
    import oracle
    from golden.make_golden import run_oracle  # noqa: E402
    oracle.build()
    n_threads = threads or (os.cpu_count() or 1)
    sample = wl.replace(n_paths=sample_paths, precision="fp64")
    t0 = time.perf_counter()
    run_oracle(sample, n_threads=n_threads)
    dt = time.perf_counter() - t0
    scale = wl.n_paths / sample_paths  # the oracle's cost is linear in paths
    return dt, wl.n_greeks / (dt * scale), n_threads


def groups_of(wl):
    """Simulations after folding the bumps onto path groups: the base one,
    v0 +/- and T -/+ (S and r bumps share the base simulation)."""
    return 1 + 2 * ("vega" in wl.greeks) + 2 * ("theta" in wl.greeks)


def stepper_roofline(wl, fwd_ms, peaks, hbm_gbs):
    """Roofline fractions of one forward launch: the FMA pipe (basic
    flops of the formulas), the special-function unit (elementary functions;
    single precision only -- in double they run on the FMA pipe) and DRAM (the
    rows stored), each achieved over its measured peak, and their maximum."""
    groups = groups_of(wl)
    path_steps = wl.n_paths * wl.n_steps
    g = STEP_GROUP[wl.scheme]
    flops = path_steps * (STEP_SHARED["flops"] + groups * g["flops"])
    funcs = path_steps * (STEP_SHARED["functions"] + groups * g["functions"])
    value = 4 if wl.precision == "mixed" else 8
    stored = path_steps * groups * value * (2 if wl.basis == "sv2" else 1)
    t = fwd_ms / 1e3
    single = wl.precision == "mixed"
    # float pairs run the same formulas on the FP32 pipes (about ten FP32
    # instructions per operation), their elementary functions in software
    fp32 = wl.precision in ("mixed", "df")
    fma_peak = peaks.get("fp32_tflops" if fp32 else "fp64_tflops")
    out = {"kernel": "forward_kernel", "workload": wl.name, "precision": wl.precision,
           "kernel_ms": fwd_ms, "simulated_path_steps": path_steps * groups,
           "fma": {"achieved": flops / t / 1e12, "peak": fma_peak, "unit": "TFLOP/s",
                   "pipe": "FP32" if fp32 else "FP64", "flops_per_path_step":
                   STEP_SHARED["flops"] + groups * g["flops"]},
           "dram": {"achieved": stored / t / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                    "bytes_per_path_step": stored / path_steps}}
    if single:
        out["xu"] = {"achieved": funcs / t / 1e12, "peak": peaks.get("xu_tops"), "unit": "Tops/s",
                     "functions_per_path_step": STEP_SHARED["functions"] + groups * g["functions"]}
    else:
        out["elementary_functions_per_path_step"] = (STEP_SHARED["functions"] +
                                                     groups * g["functions"])
    fr = {}
    for k in ("fma", "xu", "dram"):
        if k in out and out[k]["peak"]:
            out[k]["frac"] = out[k]["achieved"] / out[k]["peak"]
            fr[k] = out[k]["frac"]
    out["frac"] = max(fr.values()) if fr else None
    out["bound"] = max(fr, key=fr.get) if fr else None
    return out


def subset_errors(results_by_index, gold_path):
    """Largest relative error, per price and Greek, of results (contract
    index -> result dict) against the oracle values stored for a subset."""
    if not os.path.exists(gold_path):
        return None
    gold = json.load(open(gold_path))
    worst, n = {}, 0
    for i, c in zip(gold["indices"], gold["contracts"]):
        g = results_by_index.get(i)
        if g is None:
            continue
        n += 1
        for k in ("price", "delta", "gamma", "vega", "rho", "theta"):
            worst[k] = max(worst.get(k, 0.0), abs(g[k] - c["results"][k]) /
                           max(abs(c["results"][k]), 1e-12))
    if not n:
        return None
    return {"contracts_compared": n, "max_rel_err_vs_oracle": worst,
            "within_1e-4": all(v <= 1e-4 for v in worst.values())}


def max_rel_err(got, gold):
    worst = 0.0
    for g, r in zip(got, gold):
        for k in ("price", "delta", "gamma", "vega", "rho", "theta"):
            if r[k] is None or (isinstance(r[k], float) and math.isnan(r[k])):
                continue
            worst = max(worst, abs(g[k] - r[k]) / max(abs(r[k]), 1e-12))
    return worst


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # a sixteen-chunk sample per step keeps every host thread of the oracle's
    # forward pass busy, so the rate per path is that of the whole workload
    sample_paths = min(wl.n_paths, 16384)
    times = []
    for i in range(args.warmup + args.steps):
        dt, rate, cores = oracle_sample_rate(wl, sample_paths)
        if i >= args.warmup:
            times.append(dt)
    mean = sum(times) / len(times)
    scale = wl.n_paths / sample_paths
    value = wl.n_greeks / (mean * scale)
    sample = ("FP64 oracle (oracle/oracle.c) on %d of the %d paths per step, all %d strikes and "
              "%d revaluations, extrapolated linearly in paths" % (
                  sample_paths, wl.n_paths, len(wl.strikes), wl.n_scenarios))
    line = {
        "impl": "reference", "metric": "Greeks/s", "value": value, "unit": "Greeks/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n_paths": wl.n_paths, "n_steps": wl.n_steps,
                   "strikes": wl.strikes, "revaluations": wl.n_scenarios,
                   "scheme": wl.scheme, "basis": wl.basis},
        "cpu_baseline": {"value": value, "unit": "Greeks/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Greeks/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)



def measure_precision(api, L, torch, wl, reps=3):
    """Greeks/s of a workload in a reduced or emulated precision and its
    error against the FP64 GPU path (itself checked against the oracle) on
    the same random stream."""
    need = L.lsmc_request_footprint(None, api.Request(wl).c)
    need64 = L.lsmc_request_footprint(None, api.Request(wl, precision="fp64").c)
    out = {"workload": wl.name, "precision": wl.precision, "n_paths": wl.n_paths}
    with api.Context(workspace_bytes=max(need, need64) + (256 << 20)) as ctx:
        ctx.autotune([wl])
        plan = ctx.plan([wl])
        for _ in range(3):
            plan.launch()
        plan.fetch()
        plan.set_timing(True)
        for _ in range(reps):
            plan.launch()
        got = plan.fetch()
        kms, launches = plan.kernel_times()
        plan.close()
        ref = ctx.price(wl, precision="fp64")
    errs = {}
    for g, r in zip(got, ref):
        for k in ("price", "delta", "gamma", "vega", "rho", "theta"):
            e = abs(g[k] - r[k]) / max(abs(r[k]), 1e-12)
            errs[k] = max(errs.get(k, 0.0), e)
    ms = sum(kms) / max(1, launches)
    fwd_ms = kms[1] / max(1, launches)
    groups = groups_of(wl)
    out.update({"greeks_per_s": wl.n_greeks / (ms / 1e3), "ms_per_step": ms,
                "forward_simulated_path_steps_per_s": wl.n_paths * wl.n_steps * groups / (fwd_ms / 1e3),
                "generated_path_steps_per_s": wl.generated_path_steps / (ms / 1e3),
                "lsmc_path_steps_per_s": wl.lsmc_path_steps / (ms / 1e3),
                "kernel_ms": {"forward": kms[1] / max(1, launches),
                              "backward": kms[2] / max(1, launches)},
                "max_rel_err_vs_fp64_gpu": errs,
                "all_within_1e-4": all(v <= 1e-4 for v in errs.values()),
                "stepper_roofline": stepper_roofline(wl, fwd_ms, RUN["peaks"], RUN["hbm_gbs"])})
    return out


def measure_variants(api, L, torch, reps=3):
    """The paper-size book in regenerate mode (no path store) and out of
    sample (policy priced on independent paths), FP64 and float pairs:
    device time per step, device bytes, and the change against the default."""
    out = {}
    for prec in ("fp64", "df"):
        base = workloads.PAPER_FP64.replace(precision=prec)
        for tag, wl in (("default", base), ("regenerate", base.replace(regenerate=True)),
                        ("out_of_sample", base.replace(out_of_sample=True))):
            need = L.lsmc_request_footprint(None, api.Request(wl).c)
            with api.Context(workspace_bytes=need + (256 << 20)) as ctx:
                plan = ctx.plan([wl])
                for _ in range(2):
                    plan.launch()
                plan.fetch()
                plan.set_timing(True)
                for _ in range(reps):
                    plan.launch()
                res = plan.fetch()
                kms, n = plan.kernel_times()
                info = plan.info()
                plan.close()
            ms = sum(kms) / max(1, n)
            out["%s_%s" % (prec, tag)] = {"ms_per_step": ms, "greeks_per_s": wl.n_greeks / (ms / 1e3),
                                          "device_bytes": int(info.device_bytes),
                                          "price_k100": res[2]["price"], "price_se_k100": res[2]["price_se"]}
    return out


# The paper's deviation of half-precision arithmetic from double on its
# multi-asset path reduction, by number of time steps (its table of data
# types; context only: here only the path store is 16-bit)
PAPER_HALF_DEVIATION_PCT = {126: 0.06, 252: 0.38, 504: 1.01, 1260: 11.14, 2520: 14.65}


def measure_store16(api, L, torch, reps=2, paths=65536):
    """The 16-bit path store against the full-precision store on the same
    random streams, for the paper's step counts: largest relative deviation
    of the price and of each Greek over the five strikes, device time and
    path-store bytes.  Float-pair arithmetic (within 1e-11 of FP64), so the
    deviations are the store's; plus FP64 and MIXED timings at their
    headline sizes."""
    keys = ("price", "delta", "gamma", "vega", "rho", "theta")

    def run(wl):
        need = L.lsmc_request_footprint(None, api.Request(wl).c)
        with api.Context(workspace_bytes=need + (256 << 20)) as ctx:
            plan = ctx.plan([wl])
            for _ in range(2):
                plan.launch()
            plan.fetch()
            plan.set_timing(True)
            for _ in range(reps):
                plan.launch()
            res = plan.fetch()
            kms, n = plan.kernel_times()
            bytes_ = int(plan.info().device_bytes)
            plan.close()
        return res, sum(kms) / max(1, n), bytes_

    def dev(a, b):
        return {k: max(abs(x[k] - y[k]) / max(abs(y[k]), 1e-12) for x, y in zip(a, b))
                for k in keys}

    out = {"paths": paths, "arithmetic": "df", "by_steps": {}}
    for N in sorted(PAPER_HALF_DEVIATION_PCT):
        base = workloads.PAPER_FP64.replace(precision="df", n_paths=paths, n_steps=N)
        ref, ms0, b0 = run(base)
        row = {"native": {"ms": ms0, "device_bytes": b0,
                          "price_se_k100": ref[2]["price_se"]},
               "paper_half_arith_deviation_pct": PAPER_HALF_DEVIATION_PCT[N]}
        for fmt in ("fp16", "bf16"):
            got, ms, b = run(base.replace(store=fmt))
            d = dev(got, ref)
            row[fmt] = {"ms": ms, "device_bytes": b, "max_rel_dev": d,
                        "price_dev_pct": 100.0 * d["price"],
                        "price_dev_in_se_k100": abs(got[2]["price"] - ref[2]["price"]) /
                                                ref[2]["price_se"]}
        out["by_steps"][str(N)] = row
    for tag, wl in (("fp64_paper", workloads.PAPER_FP64),
                    ("mixed_large", workloads.LARGE_MIXED)):
        _, ms0, b0 = run(wl)
        _, ms1, b1 = run(wl.replace(store="fp16"))
        out[tag] = {"native_ms": ms0, "fp16_ms": ms1, "native_bytes": b0, "fp16_bytes": b1}
    return out


def measure_dual(api, L, torch):
    """Lower (out-of-sample) and dual upper bounds of the paper-size book's
    five strikes (base scenario), with the dual pass's device time; inner
    path-steps counted as the most the inner paths can take,
    n_outer n_inner N (N + 1) / 2 (they stop early when every strike's rule
    has exercised)."""
    out = {}
    for prec, n_outer, n_inner in (("df", 1024, 128), ("fp64", 256, 128), ("mixed", 1024, 128),
                                   ("df", 8192, 64)):
        wl = workloads.PAPER_FP64.replace(precision=prec)
        need = L.lsmc_request_footprint(None, api.Request(wl).c)
        with api.Context(workspace_bytes=need + (512 << 20)) as ctx:
            ctx.price_bounds(wl, 64, 8)  # warm-up (module load, allocator)
            b = ctx.price_bounds(wl, n_outer, n_inner)
        N = wl.n_steps
        steps = n_outer * n_inner * N * (N + 1) / 2
        out["%s_%dx%d" % (prec, n_outer, n_inner)] = {
            "dual_ms": b[0]["dual_ms"],
            "inner_path_steps_per_s_at_most": steps / (b[0]["dual_ms"] / 1e3),
            "strikes": [{"K": K, "lower": x["lower"], "lower_se": x["lower_se"],
                         "upper": x["upper"], "upper_se": x["upper_se"],
                         "gap": x["upper"] - x["lower"],
                         "martingale_end": x["martingale_end"],
                         "martingale_end_se": x["martingale_end_se"],
                         "n_near_ties": x["n_near_ties"]} for K, x in zip(wl.strikes, b)]}
    return out


def measure_book(api, L, torch, n_contracts=512, chunk=128, precision="mixed"):
    """Uneven book (512 contracts, all bump scenarios, in the given precision)
    in launches of `chunk` contracts, each captured once in a CUDA
    graph and replayed; device time summed over the chunks (each chunk holds
    its own paths, so chunks run one after another within a workspace of the
    largest chunk's size)."""
    book = workloads.book(n_contracts=n_contracts, precision=precision)
    chunks = [book[i:i + chunk] for i in range(0, len(book), chunk)]
    need = max(sum(L.lsmc_request_footprint(None, api.Request(w).c) for w in c) for c in chunks)
    greeks = sum(w.n_greeks for w in book)
    gen = sum(w.generated_path_steps for w in book)
    lsmc = sum(w.lsmc_path_steps for w in book)
    total_ms = 0.0
    results = {}
    with api.Context(workspace_bytes=need + (512 << 20)) as ctx:
        subs = []
        for ci, c in enumerate(chunks):
            sub, ppt, _ = ctx.autotune(c)
            subs.append([sub & ~L.LSMC_SUB_ITM_HALF, ppt, bool(sub & L.LSMC_SUB_ITM_HALF)])
            p = ctx.plan(c)
            p.launch(use_graph=True)  # capture and warm
            p.fetch()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(ctx.stream)
            p.launch(use_graph=True)
            ev1.record(ctx.stream)
            for j, r in enumerate(p.fetch()):
                results[ci * chunk + j] = r
            total_ms += ev0.elapsed_time(ev1)
            p.close()
    return {"contracts": n_contracts, "launch_chunks": len(chunks), "device_ms": total_ms,
            "error": subset_errors(results, GOLDEN_BOOK),
            "greeks_per_s": greeks / (total_ms / 1e3),
            "generated_path_steps_per_s": gen / (total_ms / 1e3),
            "lsmc_path_steps_per_s": lsmc / (total_ms / 1e3),
            "precision": precision, "graph": True, "autotuned_shape_sub_ppt_itmhalf": subs}


# The paper's STAC-A2 runtimes (Table A1, Alveo U280 multi-kernel, total
# runtime including transfers and host reordering; and the 2 x 24-core Xeon
# CPU reference, Table 2), milliseconds: context for the path reduction, not
# the same measurement.
PAPER_STAC_MS = {"fpga_fp64": [75.97, 141.39, 592.79, 1971.64, 10644.86],
                 "fpga_fp32": [46.11, 82.01, 341.82, 1178.14, 5838.23],
                 "cpu_fp64": [369.07, 638.67, 1551.90, 4558.11, 15561.09]}


def measure_stac(api, L, torch, reps=3):
    """STAC-A2 path reduction (Heston QE paths of every asset, exp, max over
    assets per path and date) at the paper's five problem sizes, 25,000
    paths, in FP64, float pairs and FP32: device time per run (CUDA events),
    elements (path x asset x date) per second."""
    out = {}
    stream = torch.cuda.Stream()
    for i, (name, (A, N)) in enumerate(workloads.STAC_SIZES.items()):
        P = workloads.STAC_PATHS
        models = [L.lsmc_heston(**m) for m in workloads.stac_models(A)]
        row = {"assets": A, "dates": N, "paths": P, "elements": A * N * P}
        for prec, tag, dt, width in ((L.LSMC_FP64, "fp64", torch.float64, 1),
                                     (L.LSMC_DF, "df", torch.float32, 2),
                                     (L.LSMC_MIXED, "fp32", torch.float32, 1)):
            M = torch.empty((N + 1) * P * width, dtype=dt, device="cuda")
            with torch.cuda.stream(stream):
                L.lsmc_multi_asset_max(models, N / 252.0, L.LSMC_SCHEME_QE, prec, 0.0, P, N,
                                       2022, 0, M.data_ptr(), stream.cuda_stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    L.lsmc_multi_asset_max(models, N / 252.0, L.LSMC_SCHEME_QE, prec, 0.0, P, N,
                                           2022, 0, M.data_ptr(), stream.cuda_stream)
                e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[tag] = {"ms": ms, "elements_per_s": A * N * P / (ms / 1e3)}
            del M
        row["paper_context_ms"] = {k: v[i] for k, v in PAPER_STAC_MS.items()}
        out[name] = row
    return out


def measure_serving(api, L, torch, rate=200.0, window_s=8.0, warm_s=2.0, serial_n=32,
                    precision="mixed", max_inflight=16, saturation=0, max_batch=0, share=0.0):
    """Poisson stream of book-distributed requests with continuous batching
    (up to `max_inflight` launches on the device at once, each pricing the
    requests admitted together, admitted by workspace bytes), and the first
    `serial_n` of the same requests solved one at a time in plain FP64 on the
    same GPU."""
    arrivals = workloads.poisson_arrivals(rate, warm_s + window_s, seed=11)
    reqs = workloads.book(n_contracts=len(arrivals), seed=99, precision=precision)
    with api.Context(workspace_bytes=48 << 30, max_inflight=max_inflight,
                     precision=precision, max_batch=max_batch) as srv:
        srv.set_serving_share(share)
        t0 = time.perf_counter()
        tickets = []
        for t_arr, w in zip(arrivals, reqs):
            now = time.perf_counter() - t0
            if t_arr > now:
                time.sleep(t_arr - now)
            tickets.append((t_arr, w, srv.submit(w)))
        ok = 0
        served_results = {}
        for i, (_, w, t) in enumerate(tickets):
            st, res = srv.wait(t, len(w.strikes), 300.0)
            ok += st == L.LSMC_OK
            if st == L.LSMC_OK:
                served_results[i] = res[0].as_dict()
        wall = time.perf_counter() - t0
        times = [L.lsmc_ticket_times(srv.ctx, t) for _, _, t in tickets]
    lat = [d - s for (t_arr, _, _), (s, a, d) in zip(tickets, times) if t_arr >= warm_s]
    lat.sort()
    pct = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))] * 1e3 if lat else None
    greeks = sum(w.n_greeks for t_arr, w, _ in tickets if t_arr >= warm_s)
    first_done = min(s for s, a, d in times)
    last_done = max(d for s, a, d in times)
    served = {"rate_per_s": rate, "window_s": window_s, "warm_s": warm_s,
              "requests": len(tickets), "ok": ok,
              "p50_ms": pct(0.50), "p99_ms": pct(0.99), "mean_ms": 1e3 * sum(lat) / max(1, len(lat)),
              "greeks_per_s": sum(w.n_greeks for _, w, _ in tickets) / (last_done - first_done),
              "precision": precision, "max_inflight": max_inflight,
              "max_batch": max_batch or 64, "backward_share": share or 1.0 / max_inflight,
              "error": subset_errors(served_results, GOLDEN_SERVING)}
    if saturation:
        # capacity: a burst far above what the device can serve, all submitted
        # at once; sustained Greeks/s from the first submission to the last
        # completion
        burst = workloads.book(n_contracts=saturation, seed=1234, precision=precision)
        with api.Context(workspace_bytes=48 << 30, max_inflight=max_inflight,
                         precision=precision) as srv:
            srv.set_serving_share(share)
            srv.price(burst[0])  # module load
            t0 = time.perf_counter()
            ts = [srv.submit(w) for w in burst]
            done = sum(srv.wait(t, 1, 600.0)[0] == L.LSMC_OK for t in ts)
            dt = time.perf_counter() - t0
        served["saturation"] = {"requests": saturation, "ok": done, "seconds": dt,
                                "greeks_per_s": sum(w.n_greeks for w in burst) / dt,
                                "requests_per_s": saturation / dt}
    # the same requests, one at a time, plain FP64
    serial = reqs[:serial_n]
    need = max(L.lsmc_request_footprint(None, api.Request(w, precision="fp64").c) for w in serial)
    with api.Context(workspace_bytes=need + (256 << 20)) as ctx:
        ctx.price(serial[0], precision="fp64")
        t0 = time.perf_counter()
        per = []
        for w in serial:
            t1 = time.perf_counter()
            ctx.price(w, precision="fp64")
            per.append(time.perf_counter() - t1)
        dt = time.perf_counter() - t0
    per.sort()
    served["serial_fp64"] = {"requests": len(serial), "greeks_per_s": sum(w.n_greeks for w in serial) / dt,
                             "p50_ms": per[len(per) // 2] * 1e3, "p99_ms": per[-1] * 1e3}
    return served


def extra_jobs():
    """The measurements reported beside the headline (name, function)."""
    df_paper = workloads.PAPER_FP64.replace(
        precision="df", name="american-put-heston-131072x252-5strikes-df")
    df_large = workloads.LARGE_MIXED.replace(
        precision="df", name="american-put-heston-1048576x252-5strikes-df")
    jobs = (("precision_split", lambda *a: {
                "df_paper": measure_precision(*a, df_paper),
                "df_large": measure_precision(*a, df_large),
                "mixed_large": measure_precision(*a, workloads.LARGE_MIXED)}),
            ("book", lambda *a: {"df": measure_book(*a, precision="df"),
                                 "mixed": measure_book(*a, precision="mixed"),
                                 "fp64": measure_book(*a, precision="fp64")}),
            ("stac_a2_path_reduction", lambda *a: measure_stac(*a)),
            ("regenerate_and_out_of_sample", lambda *a: measure_variants(*a)),
            ("store16_precision_study", lambda *a: measure_store16(*a)),
            ("dual_upper_bound", lambda *a: measure_dual(*a)),
            ("serving", lambda *a: {"df": measure_serving(*a, precision="df", max_inflight=8,
                                                          saturation=400),
                                    "mixed": measure_serving(*a, precision="mixed",
                                                             max_inflight=4, saturation=800)}),
            # not in the default run: the long window (10 s warm-up, 60 s
            # measured) and the slot counts side by side
            ("serving_long", lambda *a: {
                "df_%d" % k: measure_serving(*a, precision="df", max_inflight=k, warm_s=10.0,
                                             window_s=60.0) for k in (4, 8)}),
            # not in the default run: latency against offered load (requests/s)
            ("serving_curve", lambda *a: dict(
                [("df_%d" % r, measure_serving(*a, rate=float(r), precision="df", max_inflight=8,
                                               serial_n=1)) for r in (50, 100, 200, 300)] +
                [("mixed_%d" % r, measure_serving(*a, rate=float(r), precision="mixed",
                                                  max_inflight=4, serial_n=1))
                 for r in (200, 400, 800)])))
    return jobs


def within_1e4_summary(line, acc, value):
    """Greeks/s of every form measured in this run whose prices and Greeks
    are within 1e-4 relative of the FP64 oracle (the forms outside the bound
    are listed apart, with their error)."""
    ok, out = {}, {}
    if acc is not None:
        (ok if acc <= 1e-4 else out)["fp64_headline"] = value
    ps = line.get("precision_split") or {}
    for k, v in ps.items() if isinstance(ps, dict) else []:
        if isinstance(v, dict) and "greeks_per_s" in v:
            # error against the FP64 GPU path, which matches the oracle at 1e-10
            (ok if v.get("all_within_1e-4") else out)["precision_split." + k] = v["greeks_per_s"]
    for sect in ("book", "serving"):
        d = line.get(sect) or {}
        for k, v in d.items() if isinstance(d, dict) else []:
            if isinstance(v, dict) and "greeks_per_s" in v:
                e = v.get("error")
                if e is None:
                    continue
                (ok if e["within_1e-4"] else out)["%s.%s" % (sect, k)] = v["greeks_per_s"]
    best = max(ok, key=ok.get) if ok else None
    return {"forms": ok, "best": best, "best_greeks_per_s": ok.get(best),
            "outside_1e-4": out}


def run_cpu_full(wl, name):
    """The FP64 oracle once on the whole workload (every path, strike and
    revaluation) on all host cores: a full-size CPU baseline.  name
    "book_subset": the 32 seeded contracts of the uneven book whose oracle
    values are stored, one after another."""
    import oracle
    sys.path.insert(0, os.path.join(_ROOT, "tests"))
    from golden.make_golden import BOOK_SUBSET, run_oracle  # noqa: E402
    oracle.build()
    n = os.cpu_count() or 1
    if name == "book_subset":
        book = workloads.book(n_contracts=512)
        wls = [book[i] for i in BOOK_SUBSET]
        t0 = time.perf_counter()
        for w in wls:
            run_oracle(w.replace(precision="fp64"), n_threads=n)
        dt = time.perf_counter() - t0
        print(json.dumps({"cpu_full": {"workload": "book subset (%d contracts)" % len(wls),
                                       "seconds": dt, "cores": n,
                                       "greeks_per_s": sum(w.n_greeks for w in wls) / dt,
                                       "lsmc_path_steps_per_s":
                                           sum(w.lsmc_path_steps for w in wls) / dt}}),
              flush=True)
        return
    t0 = time.perf_counter()
    res, _ = run_oracle(wl.replace(precision="fp64"), n_threads=n)
    dt = time.perf_counter() - t0
    acc = None
    if os.path.exists(GOLDEN) and wl.n_paths == workloads.PAPER_FP64.n_paths and wl.scheme == "qe":
        acc = max_rel_err(res, json.load(open(GOLDEN))["results"])
    print(json.dumps({"cpu_full": {"workload": wl.name, "seconds": dt, "cores": n,
                                   "greeks_per_s": wl.n_greeks / dt,
                                   "lsmc_path_steps_per_s": wl.lsmc_path_steps / dt,
                                   "max_rel_err_vs_stored_oracle": acc}}), flush=True)


def main():
    args = parse()
    if args.workload == "book_subset" and not args.cpu_full:
        sys.exit("--workload book_subset serves --cpu-full only")
    wl = pick_workload(args.workload)
    if args.paths:
        wl = wl.replace(n_paths=args.paths, name=wl.name + "-paths%d" % args.paths)
    if args.regenerate:
        wl = wl.replace(regenerate=True, name=wl.name + "-regenerate")
    if args.out_of_sample:
        wl = wl.replace(out_of_sample=True, name=wl.name + "-out-of-sample")
    if args.store != "native":
        wl = wl.replace(store=args.store, name=wl.name + "-store-" + args.store)
    if args.impl == "reference":
        run_reference(args, wl)
        return
    if args.cpu_full:
        run_cpu_full(wl, args.workload)
        return
    rank, world, local = dist_env()
    wl = replica_workload(wl, rank)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2206_03719_gb300 import api, build
    from paper_2206_03719_gb300 import lsmc as L
    build.build()
    # the roofline denominators: HBM copy bandwidth from the pool's measured
    # peaks, the arithmetic pipes measured here (timed probes, before any
    # timed region)
    mp = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    RUN["hbm_gbs"] = mp.get("hbm_gbs")
    RUN["peaks"] = L.lsmc_measure_peaks(local)
    if args.peaks:
        print(json.dumps({"peaks": RUN["peaks"], "hbm_gbs": RUN["hbm_gbs"]}))
        return
    if args.extra:
        # one of the side measurements alone (profiling runs)
        print(json.dumps({"extra": args.extra, "result": dict(extra_jobs())[args.extra](api, L, torch)}))
        return
    req = api.Request(wl)
    need = L.lsmc_request_footprint(None, req.c)
    ctx = api.Context(workspace_bytes=need + (256 << 20))
    if args.sub:
        # a fixed backward shape (profiling runs) instead of the autotuner's
        tuned_sub = args.sub | (L.LSMC_SUB_ITM_HALF if args.itm_half else 0)
        ctx.set_backward_shape(tuned_sub, args.ppt)
        tuned_ppt = args.ppt or None
    else:
        tuned_sub, tuned_ppt, _ = ctx.autotune([wl])
    plan = ctx.plan([wl])
    info = plan.info()
    stream = ctx.stream

    for _ in range(args.warmup):
        plan.launch()
    first = plan.fetch()
    plan.set_timing(True)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        plan.launch()
    end.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = start.elapsed_time(end) / args.steps
    kms, launches = plan.kernel_times()
    res = plan.fetch()
    info = plan.info()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(world, wl.n_greeks, ms_max)

    plan.close()
    # end to end through the public call with host buffers
    e2e = None
    if not args.no_e2e:
        times = []
        for i in range(max(2, min(args.steps, 3)) + 1):
            barrier()
            t0 = time.perf_counter()
            out = L.lsmc_price_request(ctx.ctx, req.c)
            times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(sorted(times[1:])[len(times[1:]) // 2] * 1e3, dist, "cuda") / 1e3
        e2e = {"value": job_throughput(world, wl.n_greeks, e2e_s * 1e3), "unit": "Greeks/s",
               "h2d_bytes_per_step": int(info.h2d_bytes),
               "d2h_bytes_per_step": int(info.d2h_bytes),
               "ms_per_step": e2e_s * 1e3,
               "path": "lsmc_price_request: validate, plan, upload, launch, read back"}

    ctx.close()
    extras = {}
    if not args.no_extras and not args.paths and args.workload == "paper_fp64" and world == 1:
        jobs = [j for j in extra_jobs() if j[0] != "serving_long"]
        for name, fn in jobs:
            torch.cuda.empty_cache()
            try:
                extras[name] = fn(api, L, torch)
            except Exception as e:  # report, do not hide, a failed extra
                extras[name] = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank != 0:
        return

    # accuracy against the stored FP64 oracle values of this workload
    acc = None
    if os.path.exists(GOLDEN) and wl.n_paths == workloads.PAPER_FP64.n_paths and wl.scheme == "qe":
        gold = json.load(open(GOLDEN))["results"]
        acc = max_rel_err(res, gold)

    fp64_peak = RUN["peaks"].get("fp64_tflops")
    bwd_ms = kms[2] / max(1, launches)
    fwd_ms = kms[1] / max(1, launches)
    itm = info.itm_path_steps
    flops = BWD_FLOPS_ALL * info.lsmc_path_steps + BWD_FLOPS_ITM * itm
    achieved = flops / (bwd_ms / 1e3) / 1e12
    fp64 = wl.precision == "fp64"
    traffic = None
    src = os.path.join(_ROOT, "paper_2206_03719_gb300", "csrc", "backward.cu")
    if fp64 and wl.n_paths == workloads.PAPER_FP64.n_paths and os.path.exists(src):
        if (code_sha256_16(src) == BWD_TRAFFIC["source_sha256_16"] and
                (tuned_sub, tuned_ppt) == BWD_TRAFFIC["shape"]):
            traffic = BWD_TRAFFIC["bytes"]
    roofline = {
        "kernel": "backward_kernel (Longstaff-Schwartz moments, solve, exercise)",
        "bound": "alu", "achieved": achieved,
        "peak": fp64_peak if fp64 else None, "unit": "TFLOP/s",
        "frac": achieved / fp64_peak if fp64 and fp64_peak else None,
        "peak_source": "measured: FP64 fused multiply-add probe (lsmc_measure_peaks, "
                       "%.1f ms on every SM) in this run" % RUN["peaks"].get("fp64_ms", 0.0),
        "traffic": traffic,
        "traffic_source": BWD_TRAFFIC["capture"] if traffic else None,
        # the path store read once (E and v rows of every path group and date)
        "path_store_bytes": wl.n_paths * wl.n_steps * 2 * 8 *
                            (1 + 2 * ("vega" in wl.greeks) + 2 * ("theta" in wl.greeks)),
        "kernel_ms": {"setup": kms[0] / max(1, launches), "forward": fwd_ms,
                      "backward": bwd_ms, "greeks": kms[3] / max(1, launches)},
        "measured_peaks": dict(RUN["peaks"], hbm_gbs=RUN["hbm_gbs"]),
        # the stepper of this workload; the single-precision stepper at
        # 1,048,576 paths joins it from the precision split below
        "stepper": {"headline": stepper_roofline(wl, fwd_ms, RUN["peaks"], RUN["hbm_gbs"])},
    }
    cpu = None
    if not args.no_cpu_baseline:
        # the whole workload once on every host core (about 25 s on 16 Arm
        # cores for the paper-size book); one thread on a 1,024-path sample
        dt, rate, cores = oracle_sample_rate(wl, wl.n_paths)
        dt1, rate1, _ = oracle_sample_rate(wl, 1024, threads=1)
        cpu = {"value": rate, "unit": "Greeks/s", "cores": cores, "kind": "oracle",
               "sample": "full: the FP64 oracle on the whole workload (%d paths x %d steps, "
                         "%d strikes, %d revaluations) once, %.1f s; its forward pass splits "
                         "paths over the threads, its backward pass strikes"
                         % (wl.n_paths, wl.n_steps, len(wl.strikes), wl.n_scenarios, dt),
               "single_thread": {"value": rate1, "unit": "Greeks/s", "cores": 1,
                                 "sample": "1024 paths (%.1f s), scaled linearly" % dt1}}
    line = {
        "metric": "Greeks/s", "value": value, "unit": "Greeks/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32+f64", "df": "f32x2+f64"}[wl.precision], "data": "synthetic",
        "config": {"workload": wl.name, "n_paths": wl.n_paths, "n_steps": wl.n_steps,
                   "strikes": wl.strikes, "greeks": list(wl.greeks),
                   "revaluations": wl.n_scenarios, "scheme": wl.scheme, "basis": wl.basis,
                   "precision": wl.precision, "parallelism": "replicas" if world > 1 else "single",
                   "backward_subtiles_per_job": tuned_sub & ~L.LSMC_SUB_ITM_HALF,
                   "backward_itm_strikes_half_subtiles": bool(tuned_sub & L.LSMC_SUB_ITM_HALF),
                   "backward_paths_per_lane": tuned_ppt,
                   "l2": "path store %.2f GB per step exceeds L2" % (info.device_bytes / 1e9)},
        "path_steps_per_s": {"generated": job_throughput(world, wl.generated_path_steps, ms_max),
                             "lsmc": job_throughput(world, wl.lsmc_path_steps, ms_max)},
        "max_rel_err_vs_oracle": acc,
        "accuracy_ok": (acc is not None and acc <= 1e-4) if acc is not None else None,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(info.kernels_per_launch) * args.steps,
        "clocks": clocks,
        "device_bytes": int(info.device_bytes),
    }
    line.update(extras)
    ps = extras.get("precision_split") or {}
    if isinstance(ps, dict) and "mixed_large" in ps and "stepper_roofline" in ps["mixed_large"]:
        roofline["stepper"]["mixed_1048576"] = ps["mixed_large"]["stepper_roofline"]
    line["greeks_per_s_within_1e-4"] = within_1e4_summary(line, acc, value)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
