"""The benchmark's host-side accounting on CPU: the path-group count its
roofline uses against the library's own planner, the stepper roofline's
bytes and bound, whole-job throughput, the source hash that keeps a stored
traffic figure honest, the error of a stored-subset comparison, and which
forms count as within 1e-4."""
import json
import math

import pytest

import bench
from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import build as B
from paper_2206_03719_gb300 import lsmc as L

PAPER = workloads.PAPER_FP64


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


@pytest.mark.parametrize("greeks", [(), ("delta",), ("delta", "gamma"), ("vega",), ("rho",),
                                    ("theta",), ("vega", "theta"), workloads.ALL_GREEKS])
def test_group_count_is_the_planners(lib, greeks):
    wl = PAPER.replace(greeks=greeks)
    assert bench.groups_of(wl) == api.plan_layout([wl], 8, 4).n_groups


def test_stepper_roofline_bytes_and_bound():
    peaks = {"fp64_tflops": 1.0, "fp32_tflops": 80.0, "xu_tops": 10.0}
    r = bench.stepper_roofline(PAPER, 27.5, peaks, 6675.5)
    # five path groups, E and v rows of doubles
    assert r["dram"]["bytes_per_path_step"] == 5 * 2 * 8
    assert r["simulated_path_steps"] == 5 * PAPER.n_paths * PAPER.n_steps
    assert r["fma"]["pipe"] == "FP64" and "xu" not in r
    assert r["frac"] == max(r["fma"]["frac"], r["dram"]["frac"])
    assert r["bound"] == "fma"
    mixed = bench.stepper_roofline(workloads.LARGE_MIXED, 2.95, peaks, 6675.5)
    assert mixed["dram"]["bytes_per_path_step"] == 5 * 2 * 4
    assert mixed["fma"]["pipe"] == "FP32" and "xu" in mixed
    fr = {k: mixed[k]["frac"] for k in ("fma", "xu", "dram")}
    assert mixed["frac"] == max(fr.values()) and mixed["bound"] == max(fr, key=fr.get)
    # achieved bytes over the kernel time
    stored = 5 * 2 * 4 * workloads.LARGE_MIXED.n_paths * workloads.LARGE_MIXED.n_steps
    assert math.isclose(mixed["dram"]["achieved"], stored / 2.95e-3 / 1e9)


def test_throughput_counts_every_rank():
    assert bench.job_throughput(4, 25, 1000.0) == 100.0
    assert bench.job_throughput(1, 25, 250.0) == 100.0


def test_source_hash_ignores_comments_only(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {  // twice\n  return 2 * x;\n}\n")
    h = bench.code_sha256_16(str(a))
    a.write_text("// a new header line\nint f(int x) {  // doubled\n\n  return 2 * x;   \n}\n")
    assert bench.code_sha256_16(str(a)) == h
    a.write_text("int f(int x) {\n  return 3 * x;\n}\n")
    assert bench.code_sha256_16(str(a)) != h


def test_subset_errors_and_max_rel_err(tmp_path):
    keys = ("price", "delta", "gamma", "vega", "rho", "theta")
    gold = {"indices": [3, 7],
            "contracts": [{"results": {k: 1.0 for k in keys}},
                          {"results": {k: -2.0 for k in keys}}]}
    path = tmp_path / "gold.json"
    path.write_text(json.dumps(gold))
    got = {3: {k: 1.0 for k in keys}, 7: dict({k: -2.0 for k in keys}, gamma=-2.0002)}
    e = bench.subset_errors(got, str(path))
    assert e["contracts_compared"] == 2
    assert math.isclose(e["max_rel_err_vs_oracle"]["gamma"], 1e-4)
    assert e["max_rel_err_vs_oracle"]["price"] == 0.0
    got[7]["gamma"] = -2.01
    assert not bench.subset_errors(got, str(path))["within_1e-4"]
    assert bench.subset_errors({}, str(path)) is None
    assert bench.subset_errors(got, str(tmp_path / "missing.json")) is None
    # NaN reference values (Greeks not asked for) are skipped
    ref = [dict({k: 1.0 for k in keys}, rho=float("nan"))]
    assert math.isclose(bench.max_rel_err([dict({k: 1.0 for k in keys}, delta=1.5)], ref), 0.5)


def test_only_forms_within_1e4_compete():
    line = {"precision_split": {"df_paper": {"greeks_per_s": 849.0, "all_within_1e-4": True},
                                "mixed_large": {"greeks_per_s": 309.0, "all_within_1e-4": False}},
            "book": {"df": {"greeks_per_s": 1659.0, "error": {"within_1e-4": True}},
                     "mixed": {"greeks_per_s": 5383.0, "error": {"within_1e-4": False}},
                     "fp64": {"greeks_per_s": 367.0, "error": None}},
            "serving": {}}
    s = bench.within_1e4_summary(line, 4.5e-11, 319.1)
    assert s["best"] == "book.df" and s["best_greeks_per_s"] == 1659.0
    assert set(s["forms"]) == {"fp64_headline", "precision_split.df_paper", "book.df"}
    assert set(s["outside_1e-4"]) == {"precision_split.mixed_large", "book.mixed"}
    # a headline outside the bound does not count either
    assert "fp64_headline" in bench.within_1e4_summary({}, 2e-4, 1.0)["outside_1e-4"]
