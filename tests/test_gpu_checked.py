"""The checked build (LSMC_CHECKED): every global-memory access of the
forward, backward (with its per-request hand-over to host-mapped memory),
out-of-sample, dual-bound, Greeks and path-reduction kernels is tested
against the byte ranges its launch owns (the plan's allocation, a stage
call's arrays, the serving slot's mapped arrays); an access outside them
would be skipped and recorded, never performed.  On small cases of every
kernel family the checked build must record nothing and give the ordinary
build's results bit for bit (the checks add branches, not arithmetic).

compute-sanitizer is closed on this machine; this build is the library's own
substitute.  One build of the library per process, so the checked one runs
in a child process."""
import json
import math
import subprocess
import sys
import os

import pytest

from gpu_common import torch_cuda

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Runs every case with the build given on the command line ("checked" or
# "ordinary") and prints the results and the check report as JSON.
CASES = r'''
import json, sys
import torch
from paper_2206_03719_gb300 import build
from paper_2206_03719_gb300 import lsmc as L
if sys.argv[1] == "checked":
    L.load(path=build.build(checked=True))
else:
    L.load(path=build.build())
from paper_2206_03719_gb300 import api, workloads

out, reports = {}, {}
def report(name):
    if sys.argv[1] == "checked":
        reports[name] = L.lsmc_check_report(reset=True)

base = workloads.SMALL_FP64.replace(n_paths=3001, n_steps=17, basis="sv2",
                                    greeks=workloads.ALL_GREEKS, rel_dS_gamma=0.02,
                                    strikes=[92.0, 100.0, 107.0])
with api.Context(workspace_bytes=1 << 30) as ctx:
    for prec in ("fp64", "df", "mixed"):
        out["price_" + prec] = ctx.price(base, precision=prec); report("price_" + prec)
    out["regenerate"] = ctx.price(base.replace(regenerate=True)); report("regenerate")
    out["out_of_sample"] = ctx.price(base.replace(out_of_sample=True), precision="df")
    report("out_of_sample")
    out["store_fp16"] = ctx.price(base.replace(store="fp16")); report("store_fp16")
    out["ft_euler_call"] = ctx.price(base.replace(scheme="ft_euler", option="call", basis="s2"))
    report("ft_euler_call")
    out["european"] = ctx.price(base.replace(style="european")); report("european")
    book = workloads.book(n_contracts=3, paths_hi=9000, steps=(8, 13), precision="fp64")
    out["book"] = ctx.price_book(book); report("book")
    out["bounds_fp64"] = ctx.price_bounds(base.replace(greeks=()), 40, 24)
    report("bounds_fp64")
    out["bounds_df"] = ctx.price_bounds(base.replace(greeks=()), 33, 40, precision="df")
    report("bounds_df")
# served: results handed over per request through host-mapped memory
with api.Context(workspace_bytes=1 << 30, max_inflight=1) as srv:
    ws = [base.replace(n_steps=9), base.replace(n_steps=17, strikes=[95.0]),
          base.replace(n_steps=5, precision="df")]
    ts = [srv.submit(w) for w in ws]
    out["served"] = [[r.as_dict() for r in srv.wait(t, len(w.strikes), 120.0)[1]]
                     for t, w in zip(ts, ws)]
report("served")
# stage calls on caller arrays
P, N = 2500, 9
m = L.lsmc_heston(**workloads.HESTON_BASE)
S = torch.empty((N + 1, P), dtype=torch.float64, device="cuda")
V = torch.empty((N + 1, P), dtype=torch.float64, device="cuda")
L.lsmc_paths(m, 0.75, L.LSMC_SCHEME_QE, L.LSMC_FP64, P, N, 7, 1, S.data_ptr(), V.data_ptr())
torch.cuda.synchronize(); report("paths")
res = torch.zeros(5, dtype=torch.float64, device="cuda")
beta = torch.zeros((N, 6), dtype=torch.float64, device="cuda")
c = L.lsmc_contract(L.LSMC_PUT, L.LSMC_AMERICAN, 101.0, 0.75)
L.lsmc_backward(S.data_ptr(), V.data_ptr(), P, N, L.LSMC_FP64, m, c, L.LSMC_BASIS_SV2,
                res.data_ptr(), beta.data_ptr())
torch.cuda.synchronize(); report("backward")
out["backward"] = res.cpu().tolist() + beta.cpu().flatten().tolist()
L.lsmc_backward_noalloc(S.data_ptr(), V.data_ptr(), P, N, L.LSMC_FP64, m, c, L.LSMC_BASIS_SV2,
                        res.data_ptr(), beta.data_ptr())
torch.cuda.synchronize(); report("backward_noalloc")
out["backward_noalloc"] = res.cpu().tolist() + beta.cpu().flatten().tolist()
out["paths"] = [float(S.sum()), float(V.sum()), float(S[N, P - 1]), float(V[N, 0])]
M = torch.empty((N + 1) * 777, dtype=torch.float64, device="cuda")
models = [L.lsmc_heston(**x) for x in workloads.stac_models(3)]
L.lsmc_multi_asset_max(models, 0.5, L.LSMC_SCHEME_QE, L.LSMC_FP64, 0.3, 777, N, 3, 0,
                       M.data_ptr())
torch.cuda.synchronize(); report("multi_max")
out["multi_max"] = [float(M.sum()), float(M[-1])]

def plain(x):
    if isinstance(x, list):
        return [plain(y) for y in x]
    if hasattr(x, "as_dict"):
        return x.as_dict() if not isinstance(x, dict) else x
    return x
print("JSON" + json.dumps({"out": plain(out), "reports": reports}))
'''


def _run(which):
    r = subprocess.run([sys.executable, "-c", CASES, which], cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("JSON")][-1]
    return json.loads(line[4:])


def _same(a, b):
    if isinstance(a, dict):  # (the dual pass's device time is a timing, not a result)
        return a.keys() == b.keys() and all(_same(a[k], b[k]) for k in a if k != "dual_ms")
    if isinstance(a, list):
        return len(a) == len(b) and all(_same(x, y) for x, y in zip(a, b))
    if isinstance(a, float) and math.isnan(a):
        return isinstance(b, float) and math.isnan(b)
    return a == b


def test_checked_build_records_nothing_and_matches_the_ordinary_build():
    torch_cuda()
    checked = _run("checked")
    ordinary = _run("ordinary")
    bad = {k: v for k, v in checked["reports"].items() if tuple(v) != (0, 0)}
    assert not bad, "accesses outside their ranges (code, line): %s" % bad
    assert len(checked["reports"]) >= 14
    for k in ordinary["out"]:
        assert _same(checked["out"][k], ordinary["out"][k]), k
