"""The oracle over many rows at once: contiguous row ranges evaluated by the
unchanged oracle in a pool of threads (the oracle's C calls release the
interpreter lock, so the ranges run on all host cores), then joined in row
order. Test plumbing only: no SpGEMM arithmetic here."""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

import oracle


def _ranges(n: int, parts: int):
    step = max(1, -(-n // parts))
    return [np.arange(s, min(n, s + step), dtype=np.int64) for s in range(0, n, step)]


def spgemm_rows(A, B, rows=None, workers: int | None = None, exact_int: bool = False):
    """oracle.spgemm(A, B, rows) computed in row chunks on all host cores."""
    sel = np.arange(A.rows, dtype=np.int64) if rows is None else np.asarray(rows, dtype=np.int64)
    workers = workers or min(32, os.cpu_count() or 1)
    if sel.size == 0:
        return oracle.spgemm(A, B, rows=sel, exact_int=exact_int)
    chunks = [sel[r] for r in _ranges(sel.size, 4 * workers)]
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        parts = list(ex.map(lambda c: oracle.spgemm(A, B, rows=c, exact_int=exact_int), chunks))
    lens = np.concatenate([np.diff(p.row_ptr) for p in parts])
    rp = np.zeros(sel.size + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    ci = np.concatenate([p.col_idx for p in parts])
    val = np.concatenate([p.val for p in parts])
    ab = None if exact_int else np.concatenate([p.abs for p in parts])
    return oracle.OracleResult(rp, ci, val, ab)


def row_nnz(A, B, rows=None, workers: int | None = None) -> np.ndarray:
    """oracle.row_nnz(A, B, rows) computed in row chunks on all host cores."""
    sel = np.arange(A.rows, dtype=np.int64) if rows is None else np.asarray(rows, dtype=np.int64)
    workers = workers or min(32, os.cpu_count() or 1)
    if sel.size == 0:
        return np.zeros(0, dtype=np.int64)
    chunks = [sel[r] for r in _ranges(sel.size, 4 * workers)]
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        parts = list(ex.map(lambda c: oracle.row_nnz(A, B, rows=c), chunks))
    return np.concatenate(parts)
