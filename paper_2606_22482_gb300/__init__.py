"""Python binding of libns_spmm (GB300 hybrid tensor-core / CUDA-core SpMM).

Argument marshalling only: every step of planning and execution runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  The names mirror the C ABI in
``include/ns_spmm.h``; importing fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _abi
from ._abi import (NS_F32, NS_BF16, NS_TAU_INF, NsError, Tune, PlanStats, lib, check,
                   tune_default)

__all__ = ["NS_F32", "NS_BF16", "NS_TAU_INF", "NsError", "Tune", "PlanStats", "Plan", "rebalance",
           "spmm_plan", "spmm_execute", "spmm_host", "tune_default", "launch_count", "lib",
           "batch_autotune",
           "PLAN_ARRAYS"]

PLAN_ARRAYS = ("aic_rows", "win_rows", "win_dptr", "dwin", "dwin_absorb", "dtile_cols",
               "dtile_bits", "dtile_voff", "dtile_vals", "dtile_x", "res_rowptr", "res_col", "res_val",
               "rl_rows", "rl_start", "chunk_b", "chunk_k0", "row_split", "split_row",
               "split_np", "split_slot", "split_base", "queue", "item_cost")


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _csr_struct(A, device: bool) -> tuple[_abi.Csr, list]:
    """ns_csr_t from a dict with torch tensors (device) or numpy arrays (host); keeps refs."""
    keep = []
    if device:
        rp, ci, v = A["rowptr"], A["colidx"], A["vals"]
        for t, dt in ((rp, "int32"), (ci, "int32"), (v, "float32")):
            if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != f"torch.{dt}":
                raise NsError(1, f"device CSR arrays must be contiguous CUDA {dt} tensors")
        ptrs = (rp.data_ptr(), ci.data_ptr(), v.data_ptr())
        keep += [rp, ci, v]
        nnz = int(ci.numel())
    else:
        rp = np.ascontiguousarray(A["rowptr"], dtype=np.int32)
        ci = np.ascontiguousarray(A["colidx"], dtype=np.int32)
        v = np.ascontiguousarray(A["vals"], dtype=np.float32)
        keep += [rp, ci, v]
        ptrs = (rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        nnz = int(ci.size)
    c = _abi.Csr(int(A["m"]), int(A["n"]), nnz, ctypes.c_void_p(ptrs[0]), ctypes.c_void_p(ptrs[1]),
                 ctypes.c_void_p(ptrs[2]), 1 if device else 0)
    return c, keep


class Plan:
    """An execution plan (owns its device arrays until closed)."""

    def __init__(self, handle, keep, K: int, dtype: int):
        self._h = handle
        self._keep = keep
        self.K = K
        self.dtype = dtype

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        st = PlanStats()
        check(lib.ns_plan_stats(self._h, ctypes.byref(st)))
        return {f: int(getattr(st, f)) for f, _ in PlanStats._fields_}

    def export(self, name: str) -> np.ndarray:
        cnt = ctypes.c_int64()
        es = ctypes.c_int32()
        check(lib.ns_plan_array_info(self._h, name.encode(), ctypes.byref(cnt), ctypes.byref(es)))
        if name == "dtile_vals":
            dt = np.uint16 if es.value == 2 else np.float32
        elif name == "dtile_x":
            dt = np.uint16
        elif name == "dtile_bits":
            dt = np.uint32
        elif name == "res_val":
            dt = np.float32
        elif name == "item_cost":
            dt = np.int64
        else:
            dt = np.int32
        out = np.empty(int(cnt.value), dtype=dt)
        check(lib.ns_plan_export(self._h, name.encode(), out.ctypes.data_as(ctypes.c_void_p),
                                 out.nbytes))
        return out

    def inject_status(self, bits: int) -> None:
        """ns_plan_inject_status: OR status bits (2 timeout, 4 bad index) into the device word."""
        check(lib.ns_plan_inject_status(self._h, int(bits)))

    def execute(self, B, C, stream=None) -> None:
        """C := A @ B on the device (B: n x K float32 or bfloat16 tensor, C: m x K float32)."""
        spmm_execute(self, B, C, stream)

    def close(self) -> None:
        if self._h:
            check(lib.ns_plan_destroy(self._h))
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def spmm_plan(A: dict, K: int, b_dtype: int = NS_F32, tune: Tune | None = None, *,
              device: bool | None = None, stream=None) -> Plan:
    """ns_spmm_plan.  ``A`` holds torch CUDA tensors (device CSR, referenced by the plan) or
    numpy arrays (host CSR, copied)."""
    if device is None:
        device = hasattr(A["rowptr"], "is_cuda") and A["rowptr"].is_cuda
    c, keep = _csr_struct(A, device)
    h = ctypes.c_void_p()
    check(lib.ns_spmm_plan(ctypes.byref(c), int(K), int(b_dtype),
                           ctypes.byref(tune) if tune is not None else None,
                           _stream_handle(stream), ctypes.byref(h)))
    return Plan(h, keep if device else None, int(K), int(b_dtype))


def spmm_execute(plan: Plan, B, C, stream=None) -> None:
    """ns_spmm_execute with torch CUDA tensors."""
    import torch
    if not (B.is_cuda and C.is_cuda) or C.dtype != torch.float32:
        raise NsError(1, "B and C must be CUDA tensors, C float32")
    if (plan.dtype == NS_BF16) != (B.dtype == torch.bfloat16):
        raise NsError(1, "B dtype does not match the plan")
    ldb = B.stride(0) if B.dim() == 2 else plan.K
    ldc = C.stride(0) if C.dim() == 2 else plan.K
    check(lib.ns_spmm_execute(plan.handle, ctypes.c_void_p(B.data_ptr()), int(ldb),
                              ctypes.c_void_p(C.data_ptr()), int(ldc), _stream_handle(stream)))


def spmm_host(A: dict, B: np.ndarray, C: np.ndarray, b_dtype: int = NS_F32,
              tune: Tune | None = None, stream=None) -> None:
    """ns_spmm_host: C = A @ B with every operand in host memory (copies inside the call)."""
    c, keep = _csr_struct(A, False)
    K = int(B.shape[1])
    assert C.dtype == np.float32 and C.flags["C_CONTIGUOUS"] and B.flags["C_CONTIGUOUS"]
    check(lib.ns_spmm_host(ctypes.byref(c), ctypes.c_void_p(B.ctypes.data), K, int(b_dtype),
                           ctypes.c_void_p(C.ctypes.data),
                           ctypes.byref(tune) if tune is not None else None,
                           _stream_handle(stream)))


def inject_alloc_failure(after: int) -> None:
    """ns_inject_alloc_failure: the allocation after `after` more successful ones fails (-1: off)."""
    check(lib.ns_inject_alloc_failure(int(after)))


def launch_count() -> int:
    return int(lib.ns_launch_count())


def autotune(A: dict, K: int, b_dtype: int = NS_F32, stream=None, report: bool = False,
             plan_runs: float = 0.0):
    """ns_autotune on a device CSR: returns the chosen Tune (and the dry-run report if asked).

    ``plan_runs``: executions per plan over which plan time is amortised (0 = 200)."""
    c, keep = _csr_struct(A, True)
    t = Tune()
    rep = _abi.TuneReport()
    rep.plan_runs = float(plan_runs)
    check(lib.ns_autotune(ctypes.byref(c), int(K), int(b_dtype), _stream_handle(stream),
                          ctypes.byref(t), ctypes.byref(rep)))
    if report:
        return t, {f: getattr(rep, f) for f, _ in _abi.TuneReport._fields_}
    return t


def rebalance(A: dict, K: int, b_dtype: int, B, C, start: Tune | None = None, eps: float = 0.05,
              max_iter: int = 10, stream=None):
    """ns_rebalance (Section 5.3): bisect tau on per-class finish times until Skew <= 1 + eps.

    A is a device CSR, B and C CUDA tensors (C receives A @ B).  Returns (tune, report dict with
    the per-iteration tau, class spans in ms and skew)."""
    c, keep = _csr_struct(A, True)
    out = Tune()
    rep = _abi.RebalanceReport()
    check(lib.ns_rebalance(ctypes.byref(c), int(K), int(b_dtype), ctypes.c_void_p(B.data_ptr()),
                           int(B.stride(0)), ctypes.c_void_p(C.data_ptr()), int(C.stride(0)),
                           _stream_handle(stream), ctypes.byref(start) if start is not None else None,
                           float(eps), int(max_iter), ctypes.byref(out), ctypes.byref(rep)))
    n = rep.iterations
    report = {"iterations": n, "converged": bool(rep.converged), "tau": list(rep.tau[:n]),
              "dt_tc_ms": list(rep.dt_tc_ms[:n]), "dt_res_ms": list(rep.dt_res_ms[:n]),
              "skew": list(rep.skew[:n])}
    return out, report


def batch_autotune(As: list, Ks: list, b_dtype: int, Bs: list, Cs: list, start: Tune | None = None,
                   stream=None) -> tuple:
    """ns_batch_autotune: the chunk size W timed on the whole batch; returns (Tune, best_ms)."""
    structs, keep = [], []
    for A in As:
        c, k = _csr_struct(A, True)
        structs.append(c)
        keep.append(k)
    arr = (_abi.Csr * len(structs))(*structs)
    ks = (ctypes.c_int32 * len(Ks))(*[int(k) for k in Ks])
    bp = (ctypes.c_void_p * len(Bs))(*[b.data_ptr() for b in Bs])
    cp = (ctypes.c_void_p * len(Cs))(*[c.data_ptr() for c in Cs])
    out = Tune()
    ms = ctypes.c_double()
    check(lib.ns_batch_autotune(arr, len(structs), ks, int(b_dtype),
                                ctypes.byref(start) if start is not None else None, bp, cp,
                                _stream_handle(stream), ctypes.byref(out), ctypes.byref(ms)))
    return out, ms.value


class Batch:
    """ns_batch_*: many SpMMs in one persistent launch replayed from a CUDA graph."""

    def __init__(self, As: list, Ks: list, b_dtype: int = NS_F32, tune: Tune | None = None,
                 stream=None):
        structs, self._keep = [], []
        for A in As:
            c, keep = _csr_struct(A, True)
            structs.append(c)
            self._keep.append(keep)
        arr = (_abi.Csr * len(structs))(*structs)
        ks = (ctypes.c_int32 * len(Ks))(*[int(k) for k in Ks])
        self._h = ctypes.c_void_p()
        self.Ks = [int(k) for k in Ks]
        self.dtype = int(b_dtype)
        check(lib.ns_batch_plan(arr, len(structs), ks, int(b_dtype),
                                ctypes.byref(tune) if tune is not None else None,
                                _stream_handle(stream), ctypes.byref(self._h)))

    def execute(self, Bs: list, Cs: list, stream=None) -> None:
        n = len(Bs)
        bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in Bs])
        cp = (ctypes.c_void_p * n)(*[c.data_ptr() for c in Cs])
        check(lib.ns_batch_execute(self._h, bp, cp, _stream_handle(stream)))

    def stats(self) -> dict:
        ni, ng = ctypes.c_int64(), ctypes.c_int64()
        check(lib.ns_batch_stats(self._h, ctypes.byref(ni), ctypes.byref(ng)))
        return {"n_items": ni.value, "n_graphs": ng.value}

    def close(self) -> None:
        if self._h:
            lib.ns_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """ns_serve_*: continuous batching of SpMM requests (host operands, device-resident plans)."""

    def __init__(self, hbm_budget_bytes: int = 8 << 30, max_inflight: int = 64,
                 max_queue: int = 4096, max_graphs: int = 1024, tune: Tune | None = None):
        cfg = _abi.ServeCfg()
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.max_inflight = int(max_inflight)
        cfg.max_queue = int(max_queue)
        cfg.max_graphs = int(max_graphs)
        cfg.tune = tune if tune is not None else tune_default()
        self._h = ctypes.c_void_p()
        check(lib.ns_serve_create(ctypes.byref(cfg), ctypes.byref(self._h)))
        self._graphs = []
        self._live = {}

    def register(self, A: dict) -> int:
        c, keep = _csr_struct(A, False)
        gid = ctypes.c_int32()
        check(lib.ns_serve_register_graph(self._h, ctypes.byref(c), ctypes.byref(gid)))
        return int(gid.value)

    def submit(self, graph_id: int, B: np.ndarray, C: np.ndarray, b_dtype: int = NS_F32,
               t_arrival: float | None = None) -> int:
        """Queue C = A_g @ B; B (uint16 BF16 bits or float32) and C (float32) stay alive until done."""
        r = _abi.Request()
        r.graph_id = int(graph_id)
        r.K = int(B.shape[1])
        r.b_dtype = int(b_dtype)
        r.B = ctypes.c_void_p(B.ctypes.data)
        r.C = ctypes.c_void_p(C.ctypes.data)
        r.t_arrival = float(t_arrival if t_arrival is not None else now())
        t = ctypes.c_uint64()
        check(lib.ns_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._live[int(t.value)] = (B, C)
        return int(t.value)

    def poll(self, ticket: int):
        """(done, stats dict or None); raises NsError if the request failed."""
        done = ctypes.c_int()
        st = _abi.ReqStats()
        try:
            check(lib.ns_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(st)))
        finally:
            if done.value:
                self._live.pop(ticket, None)
        if not done.value:
            return False, None
        return True, {f: getattr(st, f) for f, _ in _abi.ReqStats._fields_}

    def close(self) -> None:
        if self._h:
            lib.ns_serve_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def now() -> float:
    """The serving clock (seconds), for request arrival stamps."""
    return float(lib.ns_serve_now())
