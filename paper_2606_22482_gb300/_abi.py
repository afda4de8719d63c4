"""ctypes declarations of include/ns_spmm.h (loaded once; raises if the library is missing)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libns_spmm.so")

NS_F32 = 0
NS_BF16 = 1
NS_TAU_INF = 2147483647

STATUS = {0: "NS_OK", 1: "NS_ERR_INVALID", 2: "NS_ERR_UNSUPPORTED", 3: "NS_ERR_OOM",
          4: "NS_ERR_CUDA", 5: "NS_ERR_TIMEOUT", 6: "NS_ERR_AGAIN", 7: "NS_ERR_TOO_LARGE",
          8: "NS_ERR_NOT_FOUND"}

TUNE_FIELDS = ("TM", "TK", "tau_tile", "tau_row", "tau_col", "col_order", "chunk_nnz",
               "absorb_cap", "group", "cost_tc", "cost_res", "l2_hints", "TN", "reorder")


class NsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class Tune(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in TUNE_FIELDS]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f in TUNE_FIELDS}


class PlanStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "m", "n", "nnz", "K", "b_bf16", "TM", "TK", "m_aic", "n_win", "n_dtiles", "n_dwin",
        "n_dvals", "n_res", "n_rl", "T", "n_chunks", "n_split", "n_slots", "n_items", "device_bytes")]


class RebalanceReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("tau", ctypes.c_int32 * 16), ("dt_tc_ms", ctypes.c_double * 16),
                ("dt_res_ms", ctypes.c_double * 16), ("skew", ctypes.c_double * 16)]


class TuneReport(ctypes.Structure):
    _fields_ = [("p_res", ctypes.c_double), ("p_tc", ctypes.c_double), ("alpha0", ctypes.c_double),
                ("best_ms", ctypes.c_double), ("trials", ctypes.c_int32), ("plan_runs", ctypes.c_double)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("max_graphs", ctypes.c_int32), ("tune", Tune)]


class Request(ctypes.Structure):
    _fields_ = [("graph_id", ctypes.c_int32), ("K", ctypes.c_int32), ("b_dtype", ctypes.c_int32),
                ("B", ctypes.c_void_p), ("C", ctypes.c_void_p), ("t_arrival", ctypes.c_double)]


class ReqStats(ctypes.Structure):
    _fields_ = [("t_admit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("status", ctypes.c_int32), ("plan_built", ctypes.c_int32),
                ("t_planned", ctypes.c_double), ("t_h2d", ctypes.c_double), ("t_exec", ctypes.c_double),
                ("t_d2h", ctypes.c_double)]


# every exported symbol of include/ns_spmm.h with (restype, argtypes)
P = ctypes.c_void_p
I32, I64, D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "ns_tune_default": (None, [ctypes.POINTER(Tune)]),
    "ns_spmm_plan": (ctypes.c_int, [ctypes.POINTER(Csr), I32, I32, ctypes.POINTER(Tune), P, ctypes.POINTER(P)]),
    "ns_spmm_execute": (ctypes.c_int, [P, P, I64, P, I64, P]),
    "ns_spmm_host": (ctypes.c_int, [ctypes.POINTER(Csr), P, I32, I32, P, ctypes.POINTER(Tune), P]),
    "ns_release_cache": (ctypes.c_int, []),
    "ns_plan_stats": (ctypes.c_int, [P, ctypes.POINTER(PlanStats)]),
    "ns_plan_array_info": (ctypes.c_int, [P, ctypes.c_char_p, ctypes.POINTER(I64), ctypes.POINTER(I32)]),
    "ns_plan_export": (ctypes.c_int, [P, ctypes.c_char_p, P, I64]),
    "ns_plan_destroy": (ctypes.c_int, [P]),
    "ns_batch_plan": (ctypes.c_int, [ctypes.POINTER(Csr), I32, ctypes.POINTER(I32), I32, ctypes.POINTER(Tune), P, ctypes.POINTER(P)]),
    "ns_batch_execute": (ctypes.c_int, [P, ctypes.POINTER(P), ctypes.POINTER(P), P]),
    "ns_batch_stats": (ctypes.c_int, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    "ns_batch_destroy": (ctypes.c_int, [P]),
    "ns_batch_autotune": (ctypes.c_int, [ctypes.POINTER(Csr), I32, ctypes.POINTER(I32), I32, ctypes.POINTER(Tune),
                                         ctypes.POINTER(P), ctypes.POINTER(P), P, ctypes.POINTER(Tune),
                                         ctypes.POINTER(ctypes.c_double)]),
    "ns_autotune": (ctypes.c_int, [ctypes.POINTER(Csr), I32, I32, P, ctypes.POINTER(Tune), ctypes.POINTER(TuneReport)]),
    "ns_cost_alpha": (D, [D, D, D]),
    "ns_cost_tau": (I32, [D, I32, I32]),
    "ns_skew": (D, [D, D]),
    "ns_rebalance": (ctypes.c_int, [ctypes.POINTER(Csr), I32, I32, P, ctypes.c_int64, P, ctypes.c_int64, P,
                                    ctypes.POINTER(Tune), D, I32, ctypes.POINTER(Tune),
                                    ctypes.POINTER(RebalanceReport)]),
    "ns_rebalance_next": (I32, [I32, I32, I32, D, D, D, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "ns_serve_create": (ctypes.c_int, [ctypes.POINTER(ServeCfg), ctypes.POINTER(P)]),
    "ns_serve_register_graph": (ctypes.c_int, [P, ctypes.POINTER(Csr), ctypes.POINTER(I32)]),
    "ns_serve_submit": (ctypes.c_int, [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "ns_serve_poll": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ReqStats)]),
    "ns_serve_now": (D, []),
    "ns_serve_destroy": (ctypes.c_int, [P]),
    "ns_spmm_csr_static": (ctypes.c_int, [ctypes.POINTER(Csr), P, I64, P, I64, I32, I32, P]),
    "ns_last_error": (ctypes.c_char_p, []),
    "ns_launch_count": (I64, []),
    "ns_device_ok": (I32, []),
    "ns_inject_alloc_failure": (ctypes.c_int, [I32]),
    "ns_plan_inject_status": (ctypes.c_int, [P, I32]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libns_spmm.so not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    missing = []
    for name, (res, args) in SIGNATURES.items():
        try:
            f = getattr(lib, name)
        except AttributeError:
            missing.append(name)
            continue
        f.restype = res
        f.argtypes = args
    lib.missing_symbols = missing
    return lib


lib = _load()


def check(code: int) -> None:
    if code != 0:
        raise NsError(code, lib.ns_last_error().decode(errors="replace"))


def tune_default() -> Tune:
    t = Tune()
    lib.ns_tune_default(ctypes.byref(t))
    return t
