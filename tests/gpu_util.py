"""Helpers of the GPU parity tests: run the CUDA path, compare with the oracle."""
from __future__ import annotations

import numpy as np

import oracle

# Tolerances of the values, per entry: |c - c*| <= TOL * s_ij with
# s_ij = sum_k |a_ik||b_kj| (c* is the oracle's exact-then-rounded sum).
TOL = {np.dtype(np.float32): 1e-5, np.dtype(np.float64): 1e-12}


def gpu_spgemm(handle, A, B, dtype=None, **params):
    from paper_2105_14156_gb300 import smash
    if params:
        handle.set_params(**params)
    dA = smash.to_device(A, dtype=dtype)
    dB = smash.to_device(B, dtype=dtype)
    C = handle.spgemm(dA, dB, check=True)
    return C.to_host()


def assert_matches_oracle(C, A, B, exact: bool = False, rows=None, ref=None):
    """Structure bit-exact; values exact (integer-valued data) or within TOL*s_ij.
    ref: the oracle's result for these rows, when already computed."""
    if ref is None:
        ref = oracle.spgemm(A, B, rows=rows)
    if rows is None:
        assert np.array_equal(C.row_ptr, ref.row_ptr), "row_ptr differs"
        assert np.array_equal(C.col_idx, ref.col_idx), "col_idx differs"
        got = C.val.astype(np.float64)
    else:
        ci, vals = [], []
        for i in rows:
            s, e = C.row_ptr[i], C.row_ptr[i + 1]
            ci.append(C.col_idx[s:e])
            vals.append(C.val[s:e])
        lens = np.array([c.size for c in ci])
        assert np.array_equal(lens, np.diff(ref.row_ptr)), "sampled row lengths differ"
        ci = np.concatenate(ci) if ci else np.zeros(0, np.int32)
        assert np.array_equal(ci, ref.col_idx), "sampled col_idx differ"
        got = (np.concatenate(vals) if vals else np.zeros(0)).astype(np.float64)
    if exact:
        assert np.array_equal(got, ref.val), "values differ (exact case)"
    else:
        tol = TOL[np.dtype(C.val.dtype)]
        err = np.abs(got - ref.val)
        bad = err > tol * ref.abs + 1e-300
        assert not bad.any(), "max err/s = %g" % np.max(err / np.maximum(ref.abs, 1e-300))
    return ref


def rel_frobenius(C, ref) -> float:
    d = C.val.astype(np.float64) - ref.val
    return float(np.linalg.norm(d) / max(np.linalg.norm(ref.val), 1e-300))


def device_rows(C, rows):
    """Rows of a device CSR (torch tensors) copied to the host one by one, as a
    host Csr over only those rows (row_ptr of the selection)."""
    from paper_2105_14156_gb300.rmat import Csr
    rp = C.row_ptr.cpu().numpy()
    ci, vals = [], []
    for i in rows:
        s, e = int(rp[i]), int(rp[i + 1])
        ci.append(C.col_idx[s:e].cpu().numpy())
        vals.append(C.val[s:e].cpu().numpy())
    lens = np.array([c.size for c in ci], dtype=np.int64)
    srp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=srp[1:])
    vdt = vals[0].dtype if vals else np.float32
    return Csr(len(rows), C.cols, srp,
               np.concatenate(ci) if ci else np.zeros(0, np.int32),
               np.concatenate(vals) if vals else np.zeros(0, vdt))
