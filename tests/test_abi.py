"""The C ABI without a GPU: the library loads, exports every entry point
include/lsmc.h declares, its structs have the header's layout, and host-side
validation works (CPU only; no kernel is launched)."""
import ctypes
import os
import re
import subprocess
import sys
import tempfile

import pytest

from paper_2206_03719_gb300 import build as B
from paper_2206_03719_gb300 import lsmc as L
from paper_2206_03719_gb300 import api, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsmc.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsmc_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(L.EXPORTS) == declared


def test_every_struct_field_sits_where_the_header_puts_it(tmp_path):
    # the binding's ctypes structures field by field against the compiler's
    # offsetof (a swap of two fields of one size keeps every size and would
    # pass a size check alone)
    structs = (L.lsmc_heston, L.lsmc_contract, L.lsmc_bumps, L.lsmc_result, L.lsmc_config,
               L.lsmc_request, L.lsmc_plan_info, L.lsmc_bounds)
    fields = [(t.__name__, f[0]) for t in structs for f in t._fields_]
    src = tmp_path / "offsets.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lsmc.h"\nint main(void) {\n' +
                   "".join('  printf("%%zu\\n", offsetof(%s, %s));\n' % f for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "offsets"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    offs = [int(x) for x in subprocess.check_output([str(exe)]).decode().split()]
    assert offs == [getattr(getattr(L, t), f).offset for t, f in fields]


def _prototypes():
    """{name: (return type, [parameter declarations])} of the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"(const\s+char\s*\*|int|void)\s+(lsmc_\w+)\s*\(", text):
        depth, i = 1, m.end()
        while depth:
            depth += {"(": 1, ")": -1}.get(text[i], 0)
            i += 1
        params, depth, cur = [], 0, ""
        for ch in text[m.end():i - 1]:
            if ch == "," and depth == 0:
                params.append(cur.strip())
                cur = ""
                continue
            depth += {"(": 1, ")": -1}.get(ch, 0)
            cur += ch
        params.append(cur.strip())
        out[m.group(2)] = (m.group(1).replace(" ", ""), [p for p in params if p not in ("", "void")])
    return out


def _c_class(decl):
    if "*" in decl or "[" in decl or "(" in decl:
        return "ptr"
    ty = decl.split()[-2] if len(decl.split()) > 1 else decl
    return {"int": ("int", 4), "int32_t": ("int", 4), "uint32_t": ("int", 4),
            "uint64_t": ("int", 8), "int64_t": ("int", 8), "size_t": ("int", 8),
            "double": ("float", 8), "float": ("float", 4)}[ty]


def _ctypes_class(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, (ctypes._Pointer, ctypes._CFuncPtr)):
        return "ptr"
    return ("float" if t._type_ in "fd" else "int", ctypes.sizeof(t))


def test_every_binding_signature_matches_its_prototype(lib):
    # argument count, and per argument pointer or scalar of the same kind
    # and width, of every entry point as the binding declares it to ctypes
    protos = _prototypes()
    assert sorted(protos) == sorted(L.EXPORTS)
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        assert len(fn.argtypes) == len(params), name
        for decl, t in zip(params, fn.argtypes):
            assert _c_class(decl) == _ctypes_class(t), (name, decl, t)
        assert {"int": ctypes.c_int, "void": None, "constchar*": ctypes.c_char_p}[ret] == \
            fn.restype, name


def test_binding_constants_equal_the_header(tmp_path):
    # every named constant of the header (enum members and #defines), as the
    # C compiler evaluates it, equals the binding's constant of that name
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    names = set(re.findall(r"#define (LSMC_[A-Z0-9_]+) \S", text))
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        names |= set(re.findall(r"\b(LSMC_[A-Z0-9_]+)\b(?!\s*\()", body))
    names = sorted(names)
    assert {"LSMC_SUB_ITM_HALF", "LSMC_GREEK_ALL", "LSMC_SC_T_UP", "LSMC_SC_COUNT"} <= set(names)
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "lsmc.h"\nint main(void) {\n' +
                   "".join('  printf("%%s %%lld\\n", "%s", (long long)(%s));\n' % (n, n)
                           for n in names) + "  return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    for line in subprocess.check_output([str(exe)]).decode().split("\n"):
        if line:
            name, value = line.split()
            assert getattr(L, name) == int(value), name


def test_no_cpu_fallback_and_no_oracle_in_the_product():
    # without its library the binding refuses to load (a fresh interpreter,
    # so no library is cached) ...
    code = ("from paper_2206_03719_gb300 import lsmc as L\n"
            "L.load(path='/nonexistent/liblsmc.so')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode != 0 and "liblsmc.so is not built" in r.stderr
    # ... and no file of the package reaches the oracle (test infrastructure)
    pkg = os.path.join(ROOT, "paper_2206_03719_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cpp", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f), encoding="utf-8").read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|oracle\.h|orc_", text,
                                     flags=re.M), f
    # nor does the oracle reach the package: it shares no code with the CUDA path
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f), encoding="utf-8").read()
            assert not re.search(r"paper_2206_03719_gb300|lsmc\.h|csrc", text), f


def test_abi_version_and_strerror(lib):
    assert L.lsmc_abi_version() == L.LSMC_ABI_VERSION == 1
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8):
        assert L.lsmc_strerror(code) not in ("", "unknown status")
    assert L.lsmc_strerror(12345) == "unknown status"


def test_struct_layouts_match_header(lib, tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "lsmc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lsmc_heston), sizeof(lsmc_contract),
         sizeof(lsmc_bumps), sizeof(lsmc_result), sizeof(lsmc_config), sizeof(lsmc_request),
         sizeof(lsmc_plan_info), sizeof(lsmc_bounds));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(lsmc_request, strikes), offsetof(lsmc_request, bumps),
         offsetof(lsmc_request, seed), offsetof(lsmc_result, n_singular_solves),
         offsetof(lsmc_config, hbm_budget));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    sizes, offs = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)]).decode().split("\n")[:2]]
    assert sizes == [ctypes.sizeof(t) for t in (L.lsmc_heston, L.lsmc_contract, L.lsmc_bumps,
                                                   L.lsmc_result, L.lsmc_config, L.lsmc_request,
                                                   L.lsmc_plan_info, L.lsmc_bounds)]
    assert offs == [L.lsmc_request.strikes.offset, L.lsmc_request.bumps.offset,
                    L.lsmc_request.seed.offset, L.lsmc_result.n_singular_solves.offset,
                    L.lsmc_config.hbm_budget.offset]


def test_footprint_and_validation_on_host(lib):
    req = api.Request(workloads.PAPER_FP64)
    n = L.lsmc_request_footprint(None, req.c)
    # 5 path groups x (S and v) x 252 x 131072 doubles dominate
    assert n > 5 * 2 * 252 * 131072 * 8
    mixed = api.Request(workloads.PAPER_FP64, precision="mixed")
    assert L.lsmc_request_footprint(None, mixed.c) < n
    bad = [
        dict(model=dict(workloads.HESTON_BASE, xi=0.0)),                # QE needs xi > 0
        dict(model=dict(workloads.HESTON_BASE, rho=1.5)),
        dict(model=dict(workloads.HESTON_BASE, S0=float("nan"))),
        dict(strikes=[-1.0]),
        dict(T=0.0),
        dict(n_paths=0),
        dict(rel_dS=0.0),
        dict(abs_dT=2.0),
    ]
    for kw in bad:
        r = api.Request(workloads.PAPER_FP64.replace(**kw))
        with pytest.raises(L.LsmcError) as e:
            L.lsmc_request_footprint(None, r.c)
        assert e.value.status == L.LSMC_EINVAL, kw
    # FT-Euler accepts xi = 0
    ft = api.Request(workloads.PAPER_FP64.replace(model=dict(workloads.HESTON_BASE, xi=0.0)),
                     scheme="ft_euler")
    assert L.lsmc_request_footprint(None, ft.c) > 0


def test_create_without_a_device_reports_enodev(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = ctypes.c_void_p()
    cfg = L.lsmc_config(0, 0, 0, 0, 0, 0, 0)
    assert lib.lsmc_create(ctypes.byref(ctx), ctypes.byref(cfg)) == L.LSMC_ENODEV
    assert not ctx.value


def test_stage_entry_points_reject_bad_arguments_before_launch(lib):
    assert lib.lsmc_philox(None, 0, 0, None, 5, None) == L.LSMC_EINVAL
    assert lib.lsmc_draws(1, 0, None, None, 3, 0, None, None) == L.LSMC_EINVAL
    assert lib.lsmc_draws(1, 0, None, None, 0, 7, None, None) == L.LSMC_EINVAL
    m = L.lsmc_heston(100, 0.02, 0, 0.04, 1.5, 0.04, 0.3, -0.7)
    assert lib.lsmc_paths(ctypes.byref(m), 1.0, 0, 0, 16, 4, 1, 0, None, None, None) == L.LSMC_EINVAL
    assert lib.lsmc_create(None, None) == L.LSMC_EINVAL


def test_allocator_and_bounds_entry_points_reject_bad_arguments(lib):
    # no context, or only one of the two callbacks: refused before anything runs
    alloc = L.ALLOC_FN(lambda n, user: None)
    release = L.FREE_FN(lambda p, user: None)
    assert lib.lsmc_set_allocator(None, alloc, release, None) == L.LSMC_EINVAL
    assert lib.lsmc_set_allocator(None, L.ALLOC_FN(), L.FREE_FN(), None) == L.LSMC_EINVAL
    out = L.lsmc_bounds()
    assert lib.lsmc_price_bounds(None, None, 16, 16, ctypes.byref(out)) == L.LSMC_EINVAL


def test_option_and_diagnostic_entry_points_on_host(lib):
    # context options and the per-scenario fetch refuse a missing context or
    # plan; the allocation count needs no device and starts at zero here
    assert lib.lsmc_set_wait_limit(None, 1.0) == L.LSMC_EINVAL
    assert lib.lsmc_set_backward_shape(None, 4, 4) == L.LSMC_EINVAL
    assert lib.lsmc_set_serving_share(None, 0.5) == L.LSMC_EINVAL
    prices = (ctypes.c_double * L.LSMC_SC_COUNT)()
    assert lib.lsmc_plan_fetch_scenarios(None, prices, None, 1) == L.LSMC_EINVAL
    assert lib.lsmc_device_allocations(None) == L.LSMC_EINVAL
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert L.lsmc_device_allocations() == 0
    assert L.LSMC_SC_KINDS[0] == "base" and L.LSMC_SC_COUNT == 11


def test_request_flags_on_host(lib):
    # footprints follow the flags (16-bit rows, no path store), and the flag
    # rules are checked before anything is allocated
    fp = lambda wl: L.lsmc_request_footprint(None, api.Request(wl).c)
    base = workloads.PAPER_FP64
    rows = 5 * 2 * 252 * 131072  # path groups x (E, v) x dates x paths
    native = fp(base)
    half = fp(base.replace(store="fp16"))
    assert fp(base.replace(store="bf16")) == half
    assert native - half >= rows * (8 - 2)
    assert fp(base.replace(regenerate=True)) < native - rows * 8 * 3 // 4
    assert fp(base.replace(regenerate=True, store="fp16")) < half
    assert fp(base.replace(out_of_sample=True)) >= native
    for flags in (16, 1 << 31, L.LSMC_FLAG_STORE_FP16 | L.LSMC_FLAG_STORE_BF16):
        r = api.Request(base)
        r.c.flags = flags
        with pytest.raises(L.LsmcError) as e:
            L.lsmc_request_footprint(None, r.c)
        assert e.value.status == L.LSMC_EINVAL, flags


def test_path_groups_follow_the_bumps_on_host(lib):
    # spot and rate bumps reuse the base simulation's rows (S0 scales the
    # stored exp(x); a rate bump shifts every log price by +-dr t), while the
    # v0 and maturity bumps are simulations of their own: one path group for
    # price, delta, gamma and rho, two more each for vega and theta
    base = workloads.PAPER_FP64
    rows = 2 * 252 * 131072 * 8  # E and v rows of one path group
    groups = {}
    for g in [(), ("delta", "gamma", "rho"), ("vega",), ("theta",), workloads.ALL_GREEKS]:
        n = L.lsmc_request_footprint(None, api.Request(base.replace(greeks=g)).c)
        groups[g] = n // rows
    assert groups[()] == groups[("delta", "gamma", "rho")] == 1
    assert groups[("vega",)] == groups[("theta",)] == 3
    assert groups[workloads.ALL_GREEKS] == 5


def test_exp_stage_entry_rejects_bad_arguments(lib):
    assert lib.lsmc_exp(None, None, 4, 0, None) == L.LSMC_EINVAL
    assert lib.lsmc_exp(None, None, 0, 7, None) == L.LSMC_EINVAL
    assert lib.lsmc_quantile(None, None, 4, 0, None) == L.LSMC_EINVAL
    assert lib.lsmc_quantile(None, None, 0, 7, None) == L.LSMC_EINVAL
    assert lib.lsmc_quantile(None, None, 0, L.LSMC_DF, None) == L.LSMC_ENOTIMPL
