"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Structure (row_ptr, col_idx) must match bit-exactly; values must match exactly
for integer-valued float32 data and within |c - c*| <= tol * sum|a||b|
(tol 1e-5 float32, 1e-12 float64) otherwise. Every execution path of the
planner (shared-memory hash with one warp or a thread group per row, dense
accumulator, global-memory spill; warp-rank, bitmap and bitonic write-out;
three hash functions) is forced in turn on inputs that span many tables and
leave ragged tails."""
import numpy as np
import pytest

from paper_2105_14156_gb300.rmat import Csr, GRAPH500_ABCD, rmat, workload
from tests.gpu_util import assert_matches_oracle, gpu_spgemm
from tests.helpers import identity, random_csr

pytestmark = pytest.mark.gpu

DEFAULT = dict(hash_kind=1, max_load=0.5, sym_max_tbits=15, num_max_tbits=14, group_shift=4, dense_ratio=4,
               bitmap_ratio=4, spill_blocks_per_sm=1, sym_dense_ratio=64, dense_blocks=0,
               sym_dense_blocks=0, warp_rows=1, bulk_copy=0, group_rows=0, row_window=16, row_window_tbits=7, dense_owner=0)

# Parameter sets that force each path.
PATHS = {
    "default": {},
    "warp_only_small_tables": dict(sym_max_tbits=7, num_max_tbits=7, dense_ratio=0, sym_dense_ratio=0),
    "spill_everything": dict(sym_max_tbits=5, num_max_tbits=5, dense_ratio=0, sym_dense_ratio=0),
    "dense_everything": dict(dense_ratio=1 << 20, sym_dense_ratio=1 << 20),
    "dense_four_blocks_per_sm": dict(dense_ratio=1 << 20, dense_blocks=4, num_max_tbits=5),
    "no_symbolic_dense": dict(sym_dense_ratio=0),
    "dense_counted_in_numeric": dict(dense_ratio=1 << 20, sym_dense_ratio=0),
    "dense_two_blocks_per_sm": dict(dense_ratio=1 << 20, dense_blocks=2),
    "dense_one_block_per_sm": dict(dense_ratio=1 << 20, dense_blocks=1),
    "dense_owner_computes": dict(dense_ratio=1 << 20, dense_owner=1),
    "dense_owner_four_blocks_per_sm": dict(dense_ratio=1 << 20, dense_owner=1, dense_blocks=4, num_max_tbits=5),
    "symbolic_dense_one_block_per_sm": dict(sym_dense_ratio=1 << 20, sym_dense_blocks=1),
    "symbolic_dense_eight_blocks_per_sm": dict(sym_dense_ratio=1 << 20, sym_dense_blocks=8),
    "group_per_row": dict(group_shift=0),
    "warp_rows_staged": dict(warp_rows=0),
    "bulk_copy_out": dict(bulk_copy=1),
    "group_rows_listed": dict(group_rows=1),
    "warp_rows_wide": dict(group_shift=6),
    "no_row_windows": dict(row_window=0),
    "row_windows": dict(row_window=16),
    "row_windows_wide": dict(row_window=32, row_window_tbits=8),
    "row_windows_high_bits": dict(row_window=8, hash_kind=2),
    "bitonic_only": dict(bitmap_ratio=0),
    "bitmap_always": dict(bitmap_ratio=1 << 20),
    "hash_low_bits": dict(hash_kind=0),
    "hash_high_bits": dict(hash_kind=2),
    "load_0.9": dict(max_load=0.9),
    "load_0.1": dict(max_load=0.1),
}


@pytest.fixture(scope="module")
def handle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_14156_gb300 import build, smash
    build.build()
    h = smash.Handle(0)
    yield h
    h.close()


def run(handle, A, B, dtype=None, **over):
    p = dict(DEFAULT)
    p.update(over)
    return gpu_spgemm(handle, A, B, dtype=dtype, **p)


def test_rmat10_int_bit_exact(handle):
    """Config: R-MAT scale 10, edge factor 8, integer values {1..4} in float32."""
    A = workload("rmat10_int")
    C = run(handle, A, A)
    assert_matches_oracle(C, A, A, exact=True)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_paths_f64(handle, path):
    A = rmat(11, 16, GRAPH500_ABCD, seed=21, values="f64")
    C = run(handle, A, A, **PATHS[path])
    assert_matches_oracle(C, A, A)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_paths_f32_int_exact(handle, path):
    A = rmat(11, 8, (0.45, 0.15, 0.15, 0.25), seed=22, values="int4")
    C = run(handle, A, A, **PATHS[path])
    assert_matches_oracle(C, A, A, exact=True)


@pytest.mark.parametrize("path", ["default", "spill_everything", "dense_everything", "bitonic_only"])
def test_rectangular_f32(handle, path):
    A = random_csr(700, 333, 0.03, 31, values="f32")
    B = random_csr(333, 1500, 0.02, 32, values="f32")
    C = run(handle, A, B, **PATHS[path])
    assert_matches_oracle(C, A, B)


def test_unsorted_and_duplicate_columns(handle):
    A = random_csr(300, 300, 0.05, 41, values="f64", sort_cols=False, dup_frac=0.3)
    B = random_csr(300, 300, 0.05, 42, values="f64", sort_cols=False, dup_frac=0.3)
    for path in ("default", "spill_everything", "dense_everything"):
        C = run(handle, A, B, **PATHS[path])
        assert_matches_oracle(C, A, B)


def test_unsorted_and_duplicate_columns_many_windows(handle):
    """B's rows regrouped by column window when they are unsorted and hold
    duplicate columns."""
    A = random_csr(120, 200, 0.1, 43, values="f64", sort_cols=False, dup_frac=0.3)
    B = random_csr(200, 50000, 0.004, 44, values="f64", sort_cols=False, dup_frac=0.3)
    C = run(handle, A, B, dense_ratio=1 << 20, dense_blocks=4)
    assert_matches_oracle(C, A, B)


def test_empty_inputs(handle):
    from paper_2105_14156_gb300 import smash
    E = Csr(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    B = random_csr(5, 7, 0.5, 1)
    C = run(handle, E, B)
    assert C.rows == 0 and C.col_idx.size == 0
    Z = Csr(6, 5, np.zeros(7, np.int64), np.zeros(0, np.int32), np.zeros(0))
    C = run(handle, Z, B)
    assert C.row_ptr.tolist() == [0] * 7
    # all-empty rows of B
    A = random_csr(6, 5, 0.5, 2)
    BZ = Csr(5, 7, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0))
    C = run(handle, A, BZ)
    assert C.row_ptr.tolist() == [0] * 7


def test_single_column_b(handle):
    A = rmat(9, 8, GRAPH500_ABCD, seed=5, values="f64")
    B = random_csr(A.cols, 1, 0.5, 6, values="f64")
    C = run(handle, A, B)
    assert_matches_oracle(C, A, B)


def test_one_fully_dense_row(handle):
    """A row of A touching every row of B: the largest possible row of C."""
    n = 3000
    B = random_csr(n, n, 0.004, 8, values="f64")
    r = np.concatenate([np.zeros(n, np.int64), 1 + np.arange(200) % (n - 1)])
    c = np.concatenate([np.arange(n), (7 * np.arange(200)) % n])
    from paper_2105_14156_gb300.rmat import csr_from_coo
    rp, ci = csr_from_coo(n, n, r, c)
    A = Csr(n, n, rp, ci, np.linspace(-1, 1, ci.size))
    for path in ("default", "spill_everything", "bitonic_only", "warp_only_small_tables"):
        C = run(handle, A, B, **PATHS[path])
        assert_matches_oracle(C, A, B)


def test_congruent_columns_defeat_low_bits(handle):
    """Columns that agree modulo the table size collide under low-bit hashing."""
    n, cols = 64, 1 << 16
    rows, cs = [], []
    for i in range(n):
        for t in range(40):
            rows.append(i)
            cs.append((t * 1024 + i) % cols)
    from paper_2105_14156_gb300.rmat import csr_from_coo
    rp, ci = csr_from_coo(n, cols, np.array(rows), np.array(cs))
    B = Csr(n, cols, rp, ci, np.linspace(-2, 2, ci.size))
    A = random_csr(200, n, 0.2, 9, values="f64")
    for kind in (0, 1, 2):
        C = run(handle, A, B, hash_kind=kind, dense_ratio=0)
        assert_matches_oracle(C, A, B)


@pytest.mark.parametrize("ncols,dense_blocks", [(3000, 1), (20000, 1), (40000, 1), (110000, 1), (110000, 4),
                                                (40000, 2), (70001, 4)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("owner", [0, 1])
def test_dense_rows_windows(handle, ncols, dense_blocks, dtype, owner):
    """Dense rows split into one or many column windows (the last one ragged),
    at 1, 2 or 4 blocks per SM (wider or narrower windows), merged by atomic
    adds or by the warps that own the columns (many products per column: lanes
    of one step often hit the same column)."""
    A = random_csr(96, 64, 0.3, 51, values=dtype)
    B = random_csr(64, ncols, 800.0 / ncols, 52, values=dtype)
    C = run(handle, A, B, dense_ratio=1 << 20, dense_blocks=dense_blocks, dense_owner=owner)
    assert_matches_oracle(C, A, B)


@pytest.mark.parametrize("dense_blocks", [1, 2, 4])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_dense_owner_unsorted_duplicate_b(handle, dense_blocks, dtype):
    """Owner-computes windows over a B whose rows are unsorted and repeat
    columns (B regrouped by warp slice; equal columns of one row of B land in
    the same step), and small-integer values that must sum exactly."""
    A = random_csr(80, 64, 0.3, 151, values=dtype)
    B = random_csr(64, 30000, 0.03, 152, values=dtype, sort_cols=False, dup_frac=0.3)
    C = run(handle, A, B, dense_ratio=1 << 20, dense_blocks=dense_blocks, dense_owner=1)
    assert_matches_oracle(C, A, B)
    Ai = random_csr(80, 64, 0.3, 153, values="int")
    Bi = random_csr(64, 30000, 0.03, 154, values="int", sort_cols=False, dup_frac=0.3)
    Ci = run(handle, Ai, Bi, dense_ratio=1 << 20, dense_blocks=dense_blocks, dense_owner=1)
    assert_matches_oracle(Ci, Ai, Bi, exact=True)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("owner", [0, 1])
def test_dense_windows_zero_values_and_cancellations(handle, dtype, owner):
    """Window columns whose products are all zero (+0.0 or -0.0) or cancel
    exactly keep their entries: the structure comes from which columns were
    hit, never from the values."""
    A = random_csr(96, 64, 0.3, 55, values=dtype)
    B = random_csr(64, 20000, 0.04, 56, values=dtype)
    pick = np.array([1.0, -1.0, 0.0, -0.0])
    for M, seed in ((A, 57), (B, 58)):
        idx = np.random.default_rng(seed).integers(0, 4, M.val.size)
        M.val[:] = pick[idx].astype(M.val.dtype)
    C = run(handle, A, B, dense_ratio=1 << 20, dense_blocks=2, dense_owner=owner)
    assert_matches_oracle(C, A, B)
    # every C entry whose products are all zero is still present
    assert np.sum(C.val == 0) > 0


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("max_load", [0.5, 0.7])
def test_tiny_rows_thread_per_row(handle, dtype, max_load):
    """Rows of a few products (bins of at most 128 slots) merged one thread per
    row: unsorted rows of B with duplicate columns, empty rows, and rows whose
    many products collapse onto few columns (binned one bin up)."""
    # enough rows (more than one 128-thread block per SM) for the thread-per-row path
    A = random_csr(60000, 20000, 0.00015, 81, values=dtype)
    B = random_csr(20000, 50000, 0.00006, 82, values=dtype, sort_cols=False, dup_frac=0.2)
    C = run(handle, A, B, max_load=max_load)
    assert_matches_oracle(C, A, B)
    # few columns of B: every row's bound is at most 8 columns, its products many
    A2 = random_csr(400, 300, 0.2, 83, values=dtype)
    B2 = random_csr(300, 8, 0.5, 84, values=dtype)
    C2 = run(handle, A2, B2, max_load=max_load)
    assert_matches_oracle(C2, A2, B2)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("max_load", [0.5, 0.7])
@pytest.mark.parametrize("window", [2, 5, 16, 32])
def test_row_windows(handle, dtype, max_load, window):
    """Windows of short rows sharing one (row, column)-tagged table per warp:
    unsorted rows of B with duplicate columns (hashed windows), rows without
    repeated columns (staged windows), empty rows inside a window, a last
    window cut short (the row count is not a multiple of the window), and
    rows whose many products collapse onto few columns."""
    A = random_csr(30011, 20000, 0.00015, 181, values=dtype)
    B = random_csr(20000, 50000, 0.00006, 182, values=dtype, sort_cols=False, dup_frac=0.2)
    C = run(handle, A, B, max_load=max_load, row_window=window, row_window_tbits=8)
    assert_matches_oracle(C, A, B)
    Bs = random_csr(20000, 50000, 0.00006, 183, values=dtype)
    C = run(handle, A, Bs, max_load=max_load, row_window=window, row_window_tbits=7)
    assert_matches_oracle(C, A, Bs)
    A2 = random_csr(401, 300, 0.2, 184, values=dtype)
    B2 = random_csr(300, 8, 0.5, 185, values=dtype)
    C2 = run(handle, A2, B2, max_load=max_load, row_window=window, row_window_tbits=5)
    assert_matches_oracle(C2, A2, B2)


def test_row_windows_integer_values_exact(handle):
    """Small-integer float32 data through the row windows: sums are exact."""
    A = rmat(12, 2, GRAPH500_ABCD, seed=186, values="int4")
    C = run(handle, A, A, row_window=16, row_window_tbits=8)
    assert_matches_oracle(C, A, A, exact=True)


def disjoint_block_b(nrows, width, keep, seed, values):
    """B whose row k holds `keep` columns of [k*width, (k+1)*width): no two rows
    share a column, so every row of A*B repeats no column."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for k in range(nrows):
        c = np.sort(rng.choice(width, keep, replace=False)) + k * width
        rows.append(np.full(keep, k))
        cols.append(c)
    from paper_2105_14156_gb300.rmat import csr_from_coo
    rp, ci = csr_from_coo(nrows, nrows * width, np.concatenate(rows), np.concatenate(cols))
    v = rng.uniform(-1, 1, ci.size)
    return Csr(nrows, nrows * width, rp, ci, v.astype(np.float32) if values == "f32" else v)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("group_shift", [4, 2])
def test_thread_group_rows_without_repeats(handle, dtype, group_shift):
    """Rows of 500-1000 products that repeat no column (B's rows have disjoint
    columns): in exact mode, after the symbolic phase, their products skip the
    thread-group table and are sorted straight into C."""
    A = random_csr(3001, 300, 0.02, 191, values=dtype)
    B = disjoint_block_b(300, 200, 150, 192, dtype)
    C = run(handle, A, B, group_shift=group_shift)
    assert_matches_oracle(C, A, B)


def test_tiny_rows_integer_values_exact(handle):
    """Small-integer float32 data: the thread-per-row merge is exact."""
    A = rmat(12, 2, GRAPH500_ABCD, seed=85, values="int4")
    C = run(handle, A, A)
    assert_matches_oracle(C, A, A, exact=True)


def test_dense_rows_without_windows(handle):
    """Dense rows whose few products do not pay for slicing a tall B by column
    window take the global-memory hash instead."""
    A = random_csr(40, 100000, 5e-5, 71, values="f64")
    B = random_csr(100000, 200000, 5e-5, 72, values="f64")
    C = run(handle, A, B, dense_ratio=1 << 20)
    assert_matches_oracle(C, A, B)


def test_dense_counts_of_other_operands_not_reused(handle):
    """The numeric phase reuses the symbolic phase's dense-row counts only for
    the operands they were made for: symbolic(A1, B1), symbolic(A2, B2), then
    numeric(A1, B1) counts A1*B1's dense rows itself."""
    from paper_2105_14156_gb300 import smash
    handle.set_params(**dict(DEFAULT, dense_ratio=1 << 20))
    A1 = random_csr(80, 64, 0.3, 61, values="f64")
    B1 = random_csr(64, 9000, 0.05, 62, values="f64")
    A2 = random_csr(70, 64, 0.4, 63, values="f64")
    B2 = random_csr(64, 9000, 0.07, 64, values="f64")
    d = [smash.to_device(M) for M in (A1, B1, A2, B2)]
    c_rp1, nnz1 = handle.symbolic(d[0], d[1])
    handle.symbolic(d[2], d[3])
    C1 = handle.numeric(d[0], d[1], c_rp1, nnz1)
    handle.check()
    assert_matches_oracle(C1.to_host(), A1, B1)


def test_identity(handle):
    A = rmat(10, 8, GRAPH500_ABCD, seed=3, values="f64")
    C = run(handle, A, identity(A.rows))
    assert np.array_equal(C.row_ptr, A.row_ptr)
    assert np.array_equal(C.col_idx, A.col_idx)
    assert np.array_equal(C.val, A.val)


def test_bad_column_index_is_reported(handle):
    from paper_2105_14156_gb300 import smash
    A = random_csr(50, 40, 0.2, 11, values="f64")
    B = random_csr(40, 30, 0.2, 12, values="f64")
    B.col_idx = B.col_idx.copy()
    B.col_idx[3] = 30          # out of range
    with pytest.raises(smash.SmashError) as ei:
        run(handle, A, B)
    assert ei.value.status == 1
    # the handle stays usable
    B2 = random_csr(40, 30, 0.2, 12, values="f64")
    assert_matches_oracle(run(handle, A, B2), A, B2)


@pytest.mark.parametrize("dense", [0, 1 << 20])
def test_row_of_b_too_long_is_reported(handle, dense):
    """A row of B with 2^21 entries is outside the stated limits: the call
    reports SMASH_ERR_UNSUPPORTED (found by the kernels' checks, no access
    past the row), whether the rows that reach it are hashed or dense, and
    the handle stays usable."""
    from paper_2105_14156_gb300 import smash
    from paper_2105_14156_gb300.rmat import csr_from_coo
    n = 1 << 21
    # row 0 of B: 2^21 entries over 16 columns (repeats are separate terms)
    brows = np.concatenate([np.zeros(n, np.int64), np.ones(3, np.int64)])
    bcols = np.concatenate([np.arange(n, dtype=np.int64) % 16, np.array([0, 5, 9])])
    rp, ci = csr_from_coo(2, 16, brows, bcols, merge=False)
    B = Csr(2, 16, rp, ci, np.ones(ci.size))
    arp, aci = csr_from_coo(3, 2, np.array([0, 1, 2]), np.array([0, 1, 1]))
    A = Csr(3, 2, arp, aci, np.ones(aci.size))
    with pytest.raises(smash.SmashError) as ei:
        run(handle, A, B, dense_ratio=dense)
    assert ei.value.status == 3
    A2 = random_csr(50, 40, 0.2, 13, values="f64")
    B2 = random_csr(40, 30, 0.2, 14, values="f64")
    assert_matches_oracle(run(handle, A2, B2), A2, B2)


def test_shape_mismatch(handle):
    from paper_2105_14156_gb300 import smash
    A = random_csr(10, 9, 0.3, 1)
    B = random_csr(8, 7, 0.3, 2)
    with pytest.raises(smash.SmashError) as ei:
        run(handle, A, B)
    assert ei.value.status == 2


def test_repeatable_structure(handle):
    A = rmat(12, 16, GRAPH500_ABCD, seed=4, values="f64")
    C1 = run(handle, A, A)
    C2 = run(handle, A, A)
    assert np.array_equal(C1.row_ptr, C2.row_ptr)
    assert np.array_equal(C1.col_idx, C2.col_idx)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_output_arrays_not_16_byte_aligned(handle, dtype):
    """C's arrays starting off a 16-byte boundary: the rows are stored by the
    lanes instead of bulk copies; the result is the same."""
    import torch
    from paper_2105_14156_gb300 import smash
    handle.set_params(**dict(DEFAULT, bulk_copy=1))
    A = rmat(11, 8, (0.45, 0.15, 0.15, 0.25), seed=23, values=dtype)
    dA = smash.to_device(A)
    c_rp, nnz = handle.symbolic(dA, dA)
    ci = torch.empty(nnz + 1, dtype=torch.int32, device="cuda")[1:]
    val = torch.empty(nnz + 1, dtype=dA.val.dtype, device="cuda")[1:]
    assert ci.data_ptr() % 16 != 0 and val.data_ptr() % 16 != 0
    out = smash.DeviceCsr(A.rows, A.cols, c_rp, ci, val)
    C = handle.numeric(dA, dA, c_rp, nnz, out=out)
    handle.check()
    assert_matches_oracle(C.to_host(), A, A)
