"""CPU oracle for C = A*B on CSR (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg import this package. The product path never does: it has no CPU fallback.

The arithmetic lives in ``spgemm_oracle.c`` (plain C, a dense sparse
accumulator evaluating Eq. row_wise, double-double sums); this file compiles it
with gcc and marshals numpy arrays through ctypes.

Functions and the passage each follows:
  row_flops  -- per-row product count of Gustavson's first pass
                ("Window Distribution Phase": count the FMAs of each row).
  row_nnz    -- nnz(C_i) of the selected rows: the number of distinct columns
                j with at least one product a_ik*b_kj (Eq. row_wise), the
                structure half of spgemm without the values.
  spgemm     -- C = A*B by Eq. inner_product / Eq. row_wise; structure = every
                (i, j) hit by a product; values exact-then-rounded; the scale
                s_ij = sum |a_ik||b_kj| for tolerance checks.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: x86_64 and aarch64)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_row_flops.argtypes = [I64, P, P, P, P]
        lib.oracle_row_flops.restype = None
        lib.oracle_count.argtypes = [I64, P, I64, P, P, P, P, P]
        lib.oracle_count.restype = I64
        lib.oracle_fill_f64.argtypes = [I64, P, I64] + [P] * 10
        lib.oracle_fill_f64.restype = ctypes.c_int
        lib.oracle_fill_i64.argtypes = [I64, P, I64] + [P] * 9
        lib.oracle_fill_i64.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


@dataclasses.dataclass
class OracleResult:
    """Rows of C (all rows, or the selected ones in the given order)."""
    row_ptr: np.ndarray   # int64[nsel+1]
    col_idx: np.ndarray   # int32[nnz], ascending within each row
    val: np.ndarray       # float64 (exact sum, rounded) or int64 (exact_int)
    abs: np.ndarray | None  # float64 s_ij = sum |a_ik||b_kj| (None for exact_int)


def _arrays(A, B):
    a_rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    a_ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    b_rp = np.ascontiguousarray(B.row_ptr, dtype=np.int64)
    b_ci = np.ascontiguousarray(B.col_idx, dtype=np.int32)
    return a_rp, a_ci, b_rp, b_ci


def row_flops(A, B) -> np.ndarray:
    lib = _load()
    a_rp, a_ci, b_rp, _ = _arrays(A, B)
    out = np.zeros(A.rows, dtype=np.int64)
    lib.oracle_row_flops(A.rows, _p(a_rp), _p(a_ci), _p(b_rp), _p(out))
    return out


def row_nnz(A, B, rows=None) -> np.ndarray:
    """nnz(C_i) for all rows (rows=None) or for the listed rows of A, in order."""
    if A.cols != B.rows:
        raise ValueError("shape mismatch: A.cols != B.rows")
    lib = _load()
    a_rp, a_ci, b_rp, b_ci = _arrays(A, B)
    sel = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nsel = A.rows if sel is None else sel.size
    nnz = np.zeros(nsel, dtype=np.int64)
    if lib.oracle_count(nsel, _p(sel), B.cols, _p(a_rp), _p(a_ci), _p(b_rp), _p(b_ci), _p(nnz)) < 0:
        raise MemoryError("oracle_count")
    return nnz


def spgemm(A, B, rows=None, exact_int: bool = False) -> OracleResult:
    """C = A*B for all rows (rows=None) or for the listed rows of A, in order."""
    if A.cols != B.rows:
        raise ValueError("shape mismatch: A.cols != B.rows")
    lib = _load()
    a_rp, a_ci, b_rp, b_ci = _arrays(A, B)
    sel = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nsel = A.rows if sel is None else sel.size
    nnz = np.zeros(nsel, dtype=np.int64)
    total = lib.oracle_count(nsel, _p(sel), B.cols, _p(a_rp), _p(a_ci), _p(b_rp), _p(b_ci), _p(nnz))
    if total < 0:
        raise MemoryError("oracle_count")
    out_rp = np.zeros(nsel + 1, dtype=np.int64)
    np.cumsum(nnz, out=out_rp[1:])
    out_ci = np.zeros(max(total, 1), dtype=np.int32)
    if exact_int:
        av = np.ascontiguousarray(A.val).astype(np.int64)
        bv = np.ascontiguousarray(B.val).astype(np.int64)
        if not (np.array_equal(av, A.val) and np.array_equal(bv, B.val)):
            raise ValueError("exact_int needs integer-valued inputs")
        out_val = np.zeros(max(total, 1), dtype=np.int64)
        rc = lib.oracle_fill_i64(nsel, _p(sel), B.cols, _p(a_rp), _p(a_ci), _p(av), _p(b_rp),
                                 _p(b_ci), _p(bv), _p(out_rp), _p(out_ci), _p(out_val))
        ab = None
    else:
        av = np.ascontiguousarray(A.val, dtype=np.float64)
        bv = np.ascontiguousarray(B.val, dtype=np.float64)
        out_val = np.zeros(max(total, 1), dtype=np.float64)
        ab = np.zeros(max(total, 1), dtype=np.float64)
        rc = lib.oracle_fill_f64(nsel, _p(sel), B.cols, _p(a_rp), _p(a_ci), _p(av), _p(b_rp),
                                 _p(b_ci), _p(bv), _p(out_rp), _p(out_ci), _p(out_val), _p(ab))
        ab = ab[:total]
    if rc != 0:
        raise MemoryError("oracle_fill")
    return OracleResult(out_rp, out_ci[:total], out_val[:total], ab)
