"""Throughput and roofline bookkeeping for SpGEMM (no kernels, no oracle).

Byte model, after Eq. ai_spgemm: every CSR array of A, B and C is moved once,
  bytes(M) = rowptr_bytes * (rows + 1) + (index_bytes + value_bytes) * nnz(M),
and A and B count separately even when they are the same matrix.
Work model, after Eq. ai_cf: flop = number of products a_ik*b_kj (the paper
counts one FMA per product); cf = flop / nnz(C). "Useful GFLOP/s" counts the
multiply and the add of each product: 2 * products / seconds.
"""
from __future__ import annotations


def csr_bytes(rows: int, nnz: int, value_bytes: int, index_bytes: int = 4, rowptr_bytes: int = 8) -> int:
    return rowptr_bytes * (rows + 1) + (index_bytes + value_bytes) * nnz


def compression_factor(products: int, nnz_c: int) -> float:
    """cf = flop / nnz(C) (Eq. ai_cf)."""
    return products / nnz_c if nnz_c else float("nan")


def arithmetic_intensity(nnz_a: int, nnz_b: int, nnz_c: int, cf: float, b: int) -> float:
    """Upper bound of Eq. ai_spgemm: nnz(C)*cf / ((nnz(A)+nnz(B)+nnz(C)) * b)."""
    return nnz_c * cf / ((nnz_a + nnz_b + nnz_c) * b)


def spgemm_bytes(a_rows, a_nnz, b_rows, b_nnz, c_rows, c_nnz, value_bytes: int) -> int:
    return (csr_bytes(a_rows, a_nnz, value_bytes) + csr_bytes(b_rows, b_nnz, value_bytes)
            + csr_bytes(c_rows, c_nnz, value_bytes))


def useful_gflops(products: int, seconds: float) -> float:
    return 2.0 * products / seconds / 1e9
