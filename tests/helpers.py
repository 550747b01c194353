"""Small input builders and checks shared by the tests (no SpGEMM arithmetic)."""
from __future__ import annotations

import numpy as np

from paper_2105_14156_gb300.rmat import Csr, csr_from_coo, stream_key, uniform


def random_csr(rows, cols, density, seed, values="f64", sort_cols=True, dup_frac=0.0):
    """Random CSR with uniform positions; optional unsorted columns and duplicates."""
    k = stream_key(seed, 77)
    nz = int(round(density * rows * cols))
    if rows == 0 or cols == 0:
        nz = 0
    u = uniform(k, np.arange(2 * nz + 8, dtype=np.uint64))
    pos = np.floor(u[:nz] * rows * cols).astype(np.int64) if nz else np.zeros(0, np.int64)
    pos = np.unique(pos)
    r, c = pos // max(cols, 1), pos % max(cols, 1)
    if dup_frac > 0 and r.size:
        nd = max(1, int(dup_frac * r.size))
        r = np.concatenate([r, r[:nd]])
        c = np.concatenate([c, c[:nd]])
    order = np.lexsort((c, r))
    r, c = r[order], c[order]
    rp = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=rows), out=rp[1:])
    ci = c.astype(np.int32)
    if not sort_cols:
        # reverse each row's column order
        for i in range(rows):
            ci[rp[i]:rp[i + 1]] = ci[rp[i]:rp[i + 1]][::-1].copy()
    nnz = ci.size
    kv = stream_key(seed, 78)
    uv = uniform(kv, np.arange(nnz, dtype=np.uint64))
    if values == "f64":
        v = 2.0 * uv - 1.0
    elif values == "f32":
        v = (2.0 * uv - 1.0).astype(np.float32)
    elif values == "int":
        v = np.floor(uv * 9.0).astype(np.float64) - 4.0   # integers -4..4 (zeros included)
    else:
        raise ValueError(values)
    return Csr(rows, cols, rp, ci, v)


def to_dense(M: Csr, dtype=np.float64):
    """Dense value matrix (duplicates summed) and structural count matrix."""
    D = np.zeros((M.rows, M.cols), dtype=dtype)
    S = np.zeros((M.rows, M.cols), dtype=np.int64)
    for i in range(M.rows):
        for e in range(M.row_ptr[i], M.row_ptr[i + 1]):
            D[i, M.col_idx[e]] += M.val[e]
            S[i, M.col_idx[e]] += 1
    return D, S


def identity(n, dtype=np.float64):
    return Csr(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n, dtype=dtype))


def permutation(perm, dtype=np.float64):
    """P with P[i, perm[i]] = 1, so (P B)[i,:] = B[perm[i], :]."""
    n = len(perm)
    return Csr(n, n, np.arange(n + 1, dtype=np.int64), np.asarray(perm, dtype=np.int32), np.ones(n, dtype=dtype))


def diagonal(d):
    n = len(d)
    return Csr(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.asarray(d))


def sorted_rows(M: Csr):
    """Copy of M with each row sorted by column (values carried)."""
    ci = M.col_idx.copy()
    v = M.val.copy()
    for i in range(M.rows):
        s, e = M.row_ptr[i], M.row_ptr[i + 1]
        o = np.argsort(ci[s:e], kind="stable")
        ci[s:e] = ci[s:e][o]
        v[s:e] = v[s:e][o]
    return Csr(M.rows, M.cols, M.row_ptr.copy(), ci, v)
