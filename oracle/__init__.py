"""FP64 CPU oracle for the hybrid SpMM -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
legs may import this package.  The product library never loads it, and it never loads the
product library: the two share no code, header or constant table.

* :func:`spmm` -- the definition of SpMM (Section 5.1): ``C[i,:] = sum_p vals[p] * B[col[p],:]``
  in float64, ascending p, A and B widened to double first (BF16 B widened exactly).
* :func:`plan` -- the CPU reference partition (Sections 5.2.2 and 6.1, Eq. 1-5): kept rows,
  row windows, compacted dense tiles (bitmaps and packed values) and the residual CSR, which
  the device planner must reproduce bit for bit.  How the execute kernel schedules the
  partition (residual chunks, split rows, work-list order) is not part of it.
* :func:`bf16_rne` -- round-to-nearest-even FP32 -> BF16 on the bit pattern (dense-tile values
  of the BF16 form).

Helpers for the paper's closed forms used by the tests live in :mod:`oracle.formulas`; the
pure-Python brute-force planner that pins :func:`plan` on tiny inputs is
:mod:`oracle.bruteforce`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ns_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

TAU_INF = 2147483647

TUNE_FIELDS = ("TM", "TK", "tau_tile", "tau_row", "tau_col", "col_order", "reorder")

DEFAULT_TUNE = dict(TM=16, TK=16, tau_tile=TAU_INF, tau_row=0, tau_col=0, col_order=0, reorder=0)

PLAN_ARRAYS = ("aic_rows", "win_rows", "win_dptr", "dtile_cols", "dtile_bits", "dtile_voff",
               "dtile_vals", "res_rowptr", "res_col", "res_val")
PLAN_SCALARS = ("m", "n", "nnz", "K", "b_bf16", "TM", "TK", "m_aic", "n_win", "n_dtiles",
                "n_dwin", "n_dvals", "n_res")


class _Tune(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in TUNE_FIELDS]


def build(force: bool = False) -> str:
    """Compile ns_oracle.c with the host C compiler (plain -O2, no vendor code)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.orc_spmm_rows.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P, P,
                                      ctypes.c_int32, ctypes.c_int64, P, ctypes.c_int64, P]
        lib.orc_spmm_rows.restype = ctypes.c_int
        lib.orc_plan_build.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.POINTER(_Tune),
                                       ctypes.POINTER(ctypes.c_void_p)]
        lib.orc_plan_build.restype = ctypes.c_int
        lib.orc_plan_free.argtypes = [P]
        lib.orc_plan_scalar.argtypes = [P, ctypes.c_char_p]
        lib.orc_plan_scalar.restype = ctypes.c_int64
        lib.orc_plan_array.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
        lib.orc_plan_array.restype = ctypes.c_int
        lib.orc_f32_to_bf16_array.argtypes = [P, ctypes.c_int64, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def bf16_rne(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 bit patterns (uint16), round to nearest even on the bit pattern."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib.orc_f32_to_bf16_array(_ptr(x), x.size, _ptr(out))
    return out


def spmm(A: dict, B: np.ndarray, *, rows: np.ndarray | None = None, b_bf16: bool = False,
         threads: int = 1) -> np.ndarray:
    """Float64 ``A @ B`` restricted to ``rows`` (all rows by default).

    ``B`` is float32 (n x K) or, with ``b_bf16``, uint16 BF16 bit patterns (n x K).
    ``threads`` > 1 splits the rows over a thread pool (the C call releases the GIL); each row
    is still summed by one thread in ascending order, so the result does not depend on it.
    """
    lib = _load()
    m, n = int(A["m"]), int(A["n"])
    rowptr = np.ascontiguousarray(A["rowptr"], dtype=np.int32)
    colidx = np.ascontiguousarray(A["colidx"], dtype=np.int32)
    vals = np.ascontiguousarray(A["vals"], dtype=np.float32)
    B = np.ascontiguousarray(B)
    if b_bf16:
        assert B.dtype == np.uint16
    else:
        assert B.dtype == np.float32
    K = int(B.shape[1]) if B.ndim == 2 else 0
    if rows is None:
        rows = np.arange(m, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty((len(rows), K), dtype=np.float64)

    def run(r0: int, r1: int) -> int:
        sub = rows[r0:r1]
        return lib.orc_spmm_rows(m, n, K, _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(B),
                                 1 if b_bf16 else 0, K, _ptr(sub), r1 - r0,
                                 ctypes.c_void_p(out.ctypes.data + r0 * K * 8))

    if threads <= 1 or len(rows) < 2 * threads:
        rc = run(0, len(rows))
        if rc:
            raise ValueError("oracle spmm: invalid input")
        return out
    step = (len(rows) + threads * 8 - 1) // (threads * 8)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        rcs = list(ex.map(lambda r0: run(r0, min(len(rows), r0 + step)),
                          range(0, len(rows), step)))
    if any(rcs):
        raise ValueError("oracle spmm: invalid input")
    return out


class PlanError(ValueError):
    pass


def plan(A: dict, K: int, *, b_bf16: bool = False, **tune) -> dict:
    """CPU reference partition of A.  Returns a dict of scalars and numpy arrays.

    Keyword arguments override :data:`DEFAULT_TUNE`; any other key raises ``TypeError``.
    Raises :class:`PlanError` for an invalid CSR (unsorted / duplicate / out-of-range column,
    non-monotone row pointers) or tune.
    """
    lib = _load()
    t = dict(DEFAULT_TUNE)
    unknown = set(tune) - set(DEFAULT_TUNE)
    if unknown:
        raise TypeError(f"not a partition parameter: {sorted(unknown)}")
    t.update(tune)
    tu = _Tune(*[int(t[f]) for f in TUNE_FIELDS])
    rowptr = np.ascontiguousarray(A["rowptr"], dtype=np.int32)
    colidx = np.ascontiguousarray(A["colidx"], dtype=np.int32)
    vals = np.ascontiguousarray(A["vals"], dtype=np.float32)
    h = ctypes.c_void_p()
    rc = lib.orc_plan_build(int(A["m"]), int(A["n"]), _ptr(rowptr), _ptr(colidx), _ptr(vals),
                            int(K), 1 if b_bf16 else 0, ctypes.byref(tu), ctypes.byref(h))
    if rc == 1:
        raise PlanError("invalid CSR or tune")
    if rc != 0:
        raise MemoryError("oracle plan: allocation failed")
    try:
        out = {s: int(lib.orc_plan_scalar(h, s.encode())) for s in PLAN_SCALARS}
        for name in PLAN_ARRAYS:
            p = ctypes.c_void_p()
            cnt = ctypes.c_int64()
            es = ctypes.c_int32()
            if lib.orc_plan_array(h, name.encode(), ctypes.byref(p), ctypes.byref(cnt),
                                  ctypes.byref(es)):
                raise KeyError(name)
            if name == "dtile_vals":
                dt = np.uint16 if es.value == 2 else np.float32
            elif name == "dtile_bits":
                dt = np.uint32
            elif name == "res_val":
                dt = np.float32
            else:
                dt = np.int32
            n_el = int(cnt.value)
            if n_el == 0:
                out[name] = np.zeros(0, dtype=dt)
            else:
                buf = (ctypes.c_char * (n_el * es.value)).from_address(p.value)
                out[name] = np.frombuffer(buf, dtype=dt).copy()
        out["tune"] = t
        return out
    finally:
        lib.orc_plan_free(h)


def rel_frobenius(c_test: np.ndarray, c_ref: np.ndarray) -> float:
    """||c_test - c_ref||_F / ||c_ref||_F in float64 (inf if c_ref == 0 and c_test != 0)."""
    d = np.linalg.norm(np.asarray(c_test, dtype=np.float64) - c_ref)
    r = np.linalg.norm(c_ref)
    if r == 0.0:
        return 0.0 if d == 0.0 else float("inf")
    return float(d / r)
