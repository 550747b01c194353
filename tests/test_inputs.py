"""The seeded input generators on the CPU: the counter-based generator against
the published SplitMix64 sequence, and the R-MAT recipe against the
distribution it defines (each level picks quadrant a, b, c or d)."""
import numpy as np

from paper_2105_14156_gb300 import rmat as R


def test_splitmix64_known_answers():
    # the first outputs of SplitMix64 started from state 0 (Steele, Lea and
    # Flood's generator; the widely published test vector)
    got = R.bits64(np.uint64(0), np.arange(3))
    assert [int(x) for x in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_mean():
    u = R.uniform(R.stream_key(5, 1), np.arange(200_000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * (1 / np.sqrt(12 * u.size))
    # counter-addressable: a slice of the stream is the same draws
    assert np.array_equal(R.uniform(R.stream_key(5, 1), np.arange(1000, 1010, dtype=np.uint64)), u[1000:1010])


def test_rmat_quadrant_distribution():
    abcd = (0.45, 0.15, 0.15, 0.25)
    scale, m = 2, 400_000
    r, c = R._rmat_edges(R.stream_key(3, 1), scale, abcd, 0, m)
    counts = np.zeros((4, 4))
    np.add.at(counts, (r, c), 1)
    # P(row, col) is the product over the two levels of the quadrant picked
    q = np.array([[abcd[0], abcd[1]], [abcd[2], abcd[3]]])
    p = np.zeros((4, 4))
    for i in range(4):
        for j in range(4):
            p[i, j] = q[i >> 1, j >> 1] * q[i & 1, j & 1]
    sigma = np.sqrt(m * p * (1 - p))
    assert np.all(np.abs(counts - m * p) < 5 * sigma), (counts / m, p)


def test_csr_from_coo_merges_and_sorts():
    rp, ci = R.csr_from_coo(3, 5, [2, 0, 2, 0, 2], [4, 3, 1, 3, 4])
    assert rp.tolist() == [0, 1, 1, 3]
    assert ci.tolist() == [3, 1, 4]
    rp, ci = R.csr_from_coo(3, 5, [2, 0, 2, 0, 2], [4, 3, 1, 3, 4], merge=False)
    assert rp.tolist() == [0, 2, 2, 5] and ci.tolist() == [3, 3, 1, 4, 4]


def test_rmat_is_seeded_and_well_formed():
    A = R.rmat(10, 8, seed=4, values="f32")
    B = R.rmat(10, 8, seed=4, values="f32")
    C = R.rmat(10, 8, seed=5, values="f32")
    assert A.rows == A.cols == 1024
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col_idx, B.col_idx)
    assert np.array_equal(A.val, B.val)
    assert not np.array_equal(A.col_idx, C.col_idx) or not np.array_equal(A.row_ptr, C.row_ptr)
    assert 0 < A.nnz <= 8 * 1024                                   # duplicates merged
    for i in range(A.rows):
        row = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(row) > 0)                            # sorted, unique
    assert A.val.dtype == np.float32 and np.all(A.val >= -1) and np.all(A.val < 1)
    ints = R.rmat(8, 8, seed=4, values="int4").val
    assert set(np.unique(ints).tolist()) <= {1.0, 2.0, 3.0, 4.0}


def test_paper_like_pair_is_two_independent_scale14_matrices():
    A, B = R.paper_like_pair()
    assert A.rows == A.cols == B.rows == B.cols == 1 << 14
    assert A.val.dtype == np.float64
    assert 0.9 * 16 * (1 << 14) < A.nnz <= 16 * (1 << 14)
    assert not np.array_equal(A.row_ptr, B.row_ptr)
