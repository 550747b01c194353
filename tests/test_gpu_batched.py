"""Batched products on the GPU (one persistent launch) against the oracle,
product by product: the batched workload's shapes (R-MAT A_i, 256-column
sparse B_i), plus batches that force block-wide ("big") rows and rows left to
the regular path ("huge"), empty products, both value types, every table size
of the autotuner."""
import numpy as np
import pytest

from paper_2105_14156_gb300.rmat import Csr, GRAPH500_ABCD, batched_pair, rmat
from tests.gpu_util import assert_matches_oracle
from tests.helpers import random_csr

pytestmark = pytest.mark.gpu


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


def run_batch(handle, pairs, dtype=None):
    from paper_2105_14156_gb300 import smash
    dev = [(smash.to_device(A, dtype=dtype), smash.to_device(B, dtype=dtype)) for A, B in pairs]
    Cs, stats, owner = handle.spgemm_batched(dev)
    host = [C.to_host() for C in Cs]
    if owner:
        owner.free()
    return host, stats


def small_pairs(count, seed=5, n_hi=600):
    return [batched_pair(seed, i, n_hi=n_hi) for i in range(count)]


@pytest.mark.parametrize("bits", [8, 9, 10, 11])
def test_batched_workload_shapes(handle, bits):
    pairs = small_pairs(24, n_hi=1500)
    handle.batched_table_bits(bits)
    host, stats = run_batch(handle, pairs)
    assert stats["products"] == 24
    for (A, B), C in zip(pairs, host):
        assert_matches_oracle(C, A, B)
    handle.batched_table_bits(10)


def test_batched_f64(handle):
    pairs = small_pairs(10, seed=6)
    host, _ = run_batch(handle, pairs, dtype=np.float64)
    for (A, B), C in zip(pairs, host):
        assert_matches_oracle(C, A.astype(np.float64), B.astype(np.float64))


def test_batched_big_and_huge_rows(handle):
    """Wide B (no dense accumulator) with rows of every size: warp tables,
    block tables and rows beyond a block (regular path)."""
    pairs = [
        (rmat(10, 16, GRAPH500_ABCD, seed=81, values="f32"), rmat(10, 16, GRAPH500_ABCD, seed=82, values="f32")),
        (random_csr(300, 400, 0.05, 83, values="f32"), random_csr(400, 30000, 0.004, 84, values="f32")),
        (random_csr(50, 400, 0.6, 85, values="f32"), random_csr(400, 30000, 0.02, 86, values="f32")),
    ]
    host, stats = run_batch(handle, pairs)
    assert stats["big_rows"] > 0 and stats["huge_rows"] > 0
    for (A, B), C in zip(pairs, host):
        assert_matches_oracle(C, A, B)


def test_batched_empty_and_degenerate(handle):
    E = Csr(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    B5 = random_csr(5, 7, 0.5, 1, values="f32")
    Z = Csr(6, 5, np.zeros(7, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    A6 = random_csr(6, 5, 0.5, 2, values="f32")
    BZ = Csr(5, 7, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    pairs = [(E, B5), (Z, B5), (A6, BZ), (A6, B5)]
    host, _ = run_batch(handle, pairs)
    assert host[0].rows == 0 and host[0].col_idx.size == 0
    assert host[1].row_ptr.tolist() == [0] * 7
    assert host[2].row_ptr.tolist() == [0] * 7
    assert_matches_oracle(host[3], A6, B5)


def test_batched_repeat_and_autotune(handle):
    pairs = small_pairs(16, seed=9)
    from paper_2105_14156_gb300 import smash
    dev = [(smash.to_device(A), smash.to_device(B)) for A, B in pairs]
    bits, ms = handle.batched_autotune(dev)
    assert 8 <= bits <= 11 and ms > 0
    for _ in range(2):
        Cs, _, owner = handle.spgemm_batched(dev)
        host = [C.to_host() for C in Cs]
        owner.free()
        for (A, B), C in zip(pairs, host):
            assert_matches_oracle(C, A, B)


@pytest.mark.parametrize("cutoffs", [(0, 3), (1, 2), (3, 0), (2, 1)])
def test_batched_row_cutoffs(handle, cutoffs):
    """Rows moved between the warp, block and regular paths by the cutoffs:
    the products are the same."""
    pairs = [
        (rmat(10, 16, GRAPH500_ABCD, seed=91, values="f32"), rmat(10, 16, GRAPH500_ABCD, seed=92, values="f32")),
        (random_csr(300, 400, 0.05, 93, values="f32"), random_csr(400, 30000, 0.004, 94, values="f32")),
    ] + small_pairs(6, seed=13)
    handle.batched_table_bits(9)
    handle.batched_row_cutoffs(*cutoffs)
    try:
        host, stats = run_batch(handle, pairs)
    finally:
        handle.batched_row_cutoffs(0, 3)
        handle.batched_table_bits(10)
    for (A, B), C in zip(pairs, host):
        assert_matches_oracle(C, A, B)
