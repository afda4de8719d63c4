"""The C ABI library loads and exports every entry point the header declares (CPU only);
host-side helpers of the cost model agree with the paper's closed forms."""
import os
import re

import pytest

import oracle.formulas as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ns():
    import __graft_entry__ as g
    g._build_module().build()
    import paper_2606_22482_gb300 as ns
    return ns


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ns_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_header_symbols_exported(ns):
    import ctypes
    lib = ctypes.CDLL(ns._abi.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 25
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert set(ns._abi.SIGNATURES) == declared


def test_tune_default(ns):
    t = ns.tune_default()
    assert (t.TM, t.TK, t.tau_tile, t.group) == (16, 16, ns.NS_TAU_INF, 4)


def test_cost_helpers_match_closed_forms(ns):
    for p_res, p_tc, r in [(1e9, 1e12, 1.0), (3e9, 6e12, 2.0), (5e10, 1e11, 1.0)]:
        assert ns.lib.ns_cost_alpha(p_res, p_tc, r) == pytest.approx(F.alpha(p_res, p_tc, r), rel=1e-15)
    for a, tm, tk in [(0.002, 16, 16), (0.1, 16, 16), (0.25, 64, 32), (1.0, 16, 16), (0.0, 16, 16)]:
        assert ns.lib.ns_cost_tau(a, tm, tk) == F.tau_tile(a, tm, tk)
    assert ns.lib.ns_skew(2.0, 1.0) == F.skew(2.0, 1.0)
    assert ns.lib.ns_skew(1.0, 3.0) == F.skew(1.0, 3.0)


def test_argument_errors_without_a_device(ns):
    # entry points reject missing arguments before any CUDA call, with a message
    import ctypes
    lib = ns.lib
    assert lib.ns_spmm_plan(None, 32, ns.NS_F32, None, None, None) == 1      # NS_ERR_INVALID
    assert b"NULL" in lib.ns_last_error()
    assert lib.ns_batch_autotune(None, 0, None, ns.NS_F32, None, None, None, None, None, None) == 1
    assert lib.ns_plan_destroy(None) == 0
    t = ns.tune_default()
    t.TM = 24                                                              # not 16, 32 or 64
    c = ns._abi.Csr(4, 4, 0, None, None, None, 1)
    rp = (ctypes.c_int32 * 5)()
    c.rowptr = ctypes.cast(rp, ctypes.c_void_p)
    h = ctypes.c_void_p()
    assert lib.ns_spmm_plan(ctypes.byref(c), 32, ns.NS_F32, ctypes.byref(t), None, ctypes.byref(h)) == 1
    assert b"tune" in lib.ns_last_error()


def test_static_rejects_zero_columns_before_any_device_call(ns):
    # a CSR with nonzeros but no columns cannot be valid, and B has no row to gather: the
    # allocation-free entry point refuses it on the host instead of launching
    import ctypes
    lib = ns.lib
    rp = (ctypes.c_int32 * 5)(0, 1, 2, 3, 3)
    ci = (ctypes.c_int32 * 3)(0, 0, 0)
    vv = (ctypes.c_float * 3)(1.0, 1.0, 1.0)
    cbuf = (ctypes.c_float * 64)()
    c = ns._abi.Csr(4, 0, 3, ctypes.cast(rp, ctypes.c_void_p), ctypes.cast(ci, ctypes.c_void_p),
                    ctypes.cast(vv, ctypes.c_void_p), 1)
    rc = lib.ns_spmm_csr_static(ctypes.byref(c), None, 8, ctypes.cast(cbuf, ctypes.c_void_p), 8, 8,
                                ns.NS_F32, None)
    assert rc == 1                                                          # NS_ERR_INVALID
    assert b"n = 0" in lib.ns_last_error()


def test_header_export_names_match_library_and_binding(ns):
    # the names ns_plan_export accepts, as listed in the header, are the ones the library's
    # lookup table holds and the ones the binding knows
    src = open(os.path.join(ROOT, "include", "ns_spmm.h")).read()
    m = re.search(r"Names:(.*?)\.", src, re.S)
    listed = m.group(1).replace("*", " ").split()
    api = open(os.path.join(ROOT, "paper_2606_22482_gb300", "csrc", "ns_api.cu")).read()
    table = re.findall(r"^\s*A\((\w+),", api, re.M)
    assert listed == table
    assert tuple(listed) == tuple(ns.PLAN_ARRAYS)


_CTYPE = {"int32_t": "c_int", "int64_t": "c_long", "double": "c_double", "ns_dtype_t": "c_int",
          "ns_tune_t": "Tune"}


def _header_structs():
    """Field lists (name, C type) of every `typedef struct { ... } name;` in the header."""
    src = open(os.path.join(ROOT, "include", "ns_spmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, re.S):
        fields = []
        for decl in m.group(1).split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            tm = re.match(r"(const\s+)?([\w]+)\s*(\**)\s*(.*)$", decl)
            ctype, ptr, rest = tm.group(2), tm.group(3), tm.group(4)
            for name in rest.split(","):
                name = name.strip()
                p = ptr + ("*" * (len(name) - len(name.lstrip("*"))))
                name = name.lstrip("*").strip()
                arr = re.match(r"(\w+)\[(\d+)\]", name)
                if arr:
                    name = arr.group(1)
                fields.append((name, "ptr" if p else ctype))
        out[m.group(2)] = fields
    return out


@pytest.mark.parametrize("cname,pyname", [("ns_plan_stats_t", "PlanStats"), ("ns_req_stats_t", "ReqStats"),
                                          ("ns_request_t", "Request"), ("ns_serve_cfg_t", "ServeCfg"),
                                          ("ns_tune_t", "Tune")])
def test_binding_structs_match_header(ns, cname, pyname):
    # the ctypes mirrors of the header's structs: same fields, same order, same widths
    import ctypes
    hdr = _header_structs()[cname]
    py = getattr(ns._abi, pyname)._fields_
    assert [n for n, _ in hdr] == [n for n, _ in py], (cname, hdr, py)
    for (n, ct), (_, pt) in zip(hdr, py):
        if ct == "ptr":
            assert ctypes.sizeof(pt) == ctypes.sizeof(ctypes.c_void_p), n
        elif ct in ("int32_t", "ns_dtype_t"):
            assert ctypes.sizeof(pt) == 4, n
        elif ct == "int64_t":
            assert ctypes.sizeof(pt) == 8, n
        elif ct == "double":
            assert pt is ctypes.c_double, n
        elif ct == "ns_tune_t":
            assert pt is ns._abi.Tune, n
