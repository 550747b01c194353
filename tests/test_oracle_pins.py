"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a transposed operand, a wrong index, an unsorted row, a lost duplicate, a
rounding that is not exact) fails at least one of them:
  * dense brute force (triple loop over the definition, Eq. inner_product) on
    small rectangular matrices, exact in int64, and exact rationals for float64;
  * identity, permutation and diagonal products, whose result is known exactly;
  * closed forms: total flop = sum_k colcount_A(k) * rowlen_B(k); nnz(C_i) <=
    min(flop_i, ncols); all-ones blocks; one-nonzero-per-row B;
  * scipy.sparse as an independent library routine (no cancellation inputs).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2105_14156_gb300.rmat import Csr, rmat, GRAPH500_ABCD
from tests.helpers import diagonal, identity, permutation, random_csr, sorted_rows, to_dense


def dense_brute(A: Csr, B: Csr):
    """Triple loop over Eq. inner_product on dense copies: c_ij = sum_k a_ik b_kj."""
    DA, SA = to_dense(A, np.int64 if A.val.dtype.kind in "iu" else np.float64)
    DB, SB = to_dense(B, DA.dtype)
    m, K = DA.shape
    n = DB.shape[1]
    C = np.zeros((m, n), dtype=DA.dtype)
    P = np.zeros((m, n), dtype=np.int64)
    for i in range(m):
        for j in range(n):
            s = 0
            p = 0
            for k in range(K):
                s += DA[i, k] * DB[k, j]
                p += SA[i, k] * SB[k, j]
            C[i, j] = s
            P[i, j] = p
    return C, P


def csr_result_to_dense(res, m, n, dtype):
    D = np.zeros((m, n), dtype=dtype)
    Sm = np.zeros((m, n), dtype=bool)
    for i in range(m):
        cols = res.col_idx[res.row_ptr[i]:res.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0), "row not strictly ascending"
        D[i, cols] = res.val[res.row_ptr[i]:res.row_ptr[i + 1]]
        Sm[i, cols] = True
    return D, Sm


@pytest.mark.parametrize("m,k,n,da,db,seed", [
    (7, 5, 9, 0.4, 0.3, 1), (16, 16, 16, 0.2, 0.25, 2), (24, 40, 13, 0.1, 0.3, 3),
    (1, 30, 30, 0.5, 0.2, 4), (30, 1, 30, 0.5, 0.5, 5), (30, 30, 1, 0.3, 0.5, 6),
])
def test_brute_force_int_exact(m, k, n, da, db, seed):
    A = random_csr(m, k, da, seed, values="int", dup_frac=0.2)
    B = random_csr(k, n, db, seed + 100, values="int", sort_cols=False, dup_frac=0.1)
    A = Csr(A.rows, A.cols, A.row_ptr, A.col_idx, A.val.astype(np.int64))
    B = Csr(B.rows, B.cols, B.row_ptr, B.col_idx, B.val.astype(np.int64))
    C, P = dense_brute(A, B)
    res = oracle.spgemm(A, B, exact_int=True)
    D, Sm = csr_result_to_dense(res, m, n, np.int64)
    assert np.array_equal(Sm, P > 0), "structure must be every (i,j) reached by a product"
    assert np.array_equal(D, C)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_brute_force_f64_exact_rational(seed):
    m, k, n = 9, 11, 8
    A = random_csr(m, k, 0.5, seed, values="f64", dup_frac=0.2)
    B = random_csr(k, n, 0.5, seed + 1, values="f64", sort_cols=False)
    res = oracle.spgemm(A, B)
    exact = {}
    absum = {}
    for i in range(m):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            kk = A.col_idx[e]
            for f in range(B.row_ptr[kk], B.row_ptr[kk + 1]):
                j = B.col_idx[f]
                exact[(i, j)] = exact.get((i, j), Fraction(0)) + Fraction(A.val[e]) * Fraction(B.val[f])
                absum[(i, j)] = absum.get((i, j), 0.0) + abs(A.val[e]) * abs(B.val[f])
    got = {}
    for i in range(m):
        for t in range(res.row_ptr[i], res.row_ptr[i + 1]):
            got[(i, int(res.col_idx[t]))] = (res.val[t], res.abs[t])
    assert set(got) == set(exact)
    for key, (v, s) in got.items():
        ref = float(exact[key])          # correctly rounded exact sum
        assert abs(v - ref) <= np.spacing(abs(ref)) + 1e-30 * s
        assert s == pytest.approx(absum[key], rel=1e-14)


def test_identity_products():
    A = rmat(8, 8, GRAPH500_ABCD, seed=3, values="f64")
    I = identity(A.rows)
    for res in (oracle.spgemm(A, I), oracle.spgemm(I, A)):
        assert np.array_equal(res.row_ptr, A.row_ptr)
        assert np.array_equal(res.col_idx, A.col_idx)
        assert np.array_equal(res.val, A.val)


def test_permutation_products():
    B = rmat(8, 4, GRAPH500_ABCD, seed=4, values="f64")
    rng = np.random.default_rng(0)
    perm = rng.permutation(B.rows)
    res = oracle.spgemm(permutation(perm), B)
    for i in range(B.rows):
        src = perm[i]
        s, e = B.row_ptr[src], B.row_ptr[src + 1]
        assert np.array_equal(res.col_idx[res.row_ptr[i]:res.row_ptr[i + 1]], B.col_idx[s:e])
        assert np.array_equal(res.val[res.row_ptr[i]:res.row_ptr[i + 1]], B.val[s:e])
    # right multiplication moves columns: (B P)[i, perm[j]] = B[i, j]
    resr = oracle.spgemm(B, permutation(perm))
    for i in range(B.rows):
        s, e = B.row_ptr[i], B.row_ptr[i + 1]
        want_cols = perm[B.col_idx[s:e]]
        o = np.argsort(want_cols)
        assert np.array_equal(resr.col_idx[resr.row_ptr[i]:resr.row_ptr[i + 1]], want_cols[o])
        assert np.array_equal(resr.val[resr.row_ptr[i]:resr.row_ptr[i + 1]], B.val[s:e][o])


def test_diagonal_scaling_bit_exact():
    B = rmat(8, 8, GRAPH500_ABCD, seed=5, values="f64")
    d = np.linspace(-3.0, 3.0, B.rows) + 0.1
    res = oracle.spgemm(diagonal(d), B)
    assert np.array_equal(res.col_idx, B.col_idx)
    want = np.repeat(d, np.diff(B.row_ptr)) * B.val
    assert np.array_equal(res.val, want)
    # float32 inputs: one product per entry, exact in double
    B32 = B.astype(np.float32)
    d32 = d.astype(np.float32)
    res32 = oracle.spgemm(diagonal(d32), B32)
    want32 = np.repeat(d32.astype(np.float64), np.diff(B.row_ptr)) * B32.val.astype(np.float64)
    assert np.array_equal(res32.val, want32)


def test_closed_form_flops_and_bounds():
    A = rmat(9, 8, GRAPH500_ABCD, seed=6, values="f64")
    B = rmat(9, 6, (0.45, 0.15, 0.15, 0.25), seed=7, values="f64")
    flop = oracle.row_flops(A, B)
    colcount_a = np.bincount(A.col_idx, minlength=A.cols)
    rowlen_b = np.diff(B.row_ptr)
    assert flop.sum() == int(np.dot(colcount_a.astype(np.int64), rowlen_b))
    res = oracle.spgemm(A, B)
    nnz = np.diff(res.row_ptr)
    assert np.all(nnz <= np.minimum(flop, B.cols))
    assert np.all((nnz == 0) == (flop == 0))


def test_all_ones_blocks():
    k, nb = 6, 5
    n = k * nb
    r, c = [], []
    for b in range(nb):
        for i in range(k):
            for j in range(k):
                r.append(b * k + i)
                c.append(b * k + j)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    M = Csr(n, n, rp, np.asarray(c, dtype=np.int32), np.ones(len(r)))
    res = oracle.spgemm(M, M)
    assert res.col_idx.size == nb * k * k
    assert np.all(res.val == k)
    assert np.all(res.abs == k)


def test_one_nonzero_per_row_b():
    A = rmat(8, 8, GRAPH500_ABCD, seed=8, values="f64")
    rng = np.random.default_rng(1)
    bc = rng.integers(0, 37, size=A.cols).astype(np.int32)
    B = Csr(A.cols, 37, np.arange(A.cols + 1, dtype=np.int64), bc, np.ones(A.cols))
    res = oracle.spgemm(A, B)
    for i in range(A.rows):
        ks = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert res.row_ptr[i + 1] - res.row_ptr[i] == np.unique(bc[ks]).size


def test_empty_and_degenerate():
    E = Csr(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    B = random_csr(5, 4, 0.5, 1)
    res = oracle.spgemm(E, B)
    assert res.row_ptr.tolist() == [0] and res.col_idx.size == 0
    Z = Csr(4, 5, np.zeros(5, np.int64), np.zeros(0, np.int32), np.zeros(0))
    res = oracle.spgemm(Z, B)
    assert res.row_ptr.tolist() == [0] * 5
    with pytest.raises(ValueError):
        oracle.spgemm(B, B)


def test_selected_rows_match_full():
    A = rmat(9, 8, GRAPH500_ABCD, seed=9, values="f64")
    full = oracle.spgemm(A, A)
    rows = np.array([511, 0, 17, 17, 300])
    part = oracle.spgemm(A, A, rows=rows)
    for t, i in enumerate(rows):
        a, b = full.row_ptr[i], full.row_ptr[i + 1]
        c, d = part.row_ptr[t], part.row_ptr[t + 1]
        assert np.array_equal(full.col_idx[a:b], part.col_idx[c:d])
        assert np.array_equal(full.val[a:b], part.val[c:d])


def test_scipy_cross_check_rmat10():
    sp = pytest.importorskip("scipy.sparse")
    A = rmat(10, 8, GRAPH500_ABCD, seed=1, values="int4")
    M = sp.csr_matrix((A.val.astype(np.float64), A.col_idx, A.row_ptr), shape=(A.rows, A.cols))
    C = (M @ M).tocsr()
    C.sort_indices()
    res = oracle.spgemm(A, A)
    assert np.array_equal(res.row_ptr, C.indptr.astype(np.int64))
    assert np.array_equal(res.col_idx, C.indices)
    assert np.array_equal(res.val, C.data)
    ri = oracle.spgemm(A, A, exact_int=True)
    assert np.array_equal(ri.val.astype(np.float64), res.val)


def test_scipy_cross_check_float():
    sp = pytest.importorskip("scipy.sparse")
    A = rmat(11, 8, (0.45, 0.15, 0.15, 0.25), seed=2, values="f64")
    B = rmat(11, 4, GRAPH500_ABCD, seed=3, values="f64")
    MA = sp.csr_matrix((A.val, A.col_idx, A.row_ptr), shape=(A.rows, A.cols))
    MB = sp.csr_matrix((B.val, B.col_idx, B.row_ptr), shape=(B.rows, B.cols))
    C = (MA @ MB).tocsr()
    C.sort_indices()
    res = oracle.spgemm(A, B)
    assert np.array_equal(res.row_ptr, C.indptr.astype(np.int64))
    assert np.array_equal(res.col_idx, C.indices)
    assert np.all(np.abs(res.val - C.data) <= 1e-14 * res.abs)
