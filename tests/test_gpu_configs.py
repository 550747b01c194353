"""The evaluated configurations at their full sizes, through the C ABI, against
the oracle (Eq. row_wise): structure bit-exact, values within |c - c*| <=
tol * sum|a||b| (tol 1e-5 float32, 1e-12 float64).

  * R-MAT scale 16, edge factor 16, float64, plain two-pass path: every row.
  * R-MAT scale 20, edge factor 8, (.45,.15,.15,.25), float32, learned sizing
    with the autotuned planner parameters (and the plain path): every row.
  * R-MAT scale 18, edge factor 16, float32, learned sizing: the whole row
    pointer against the oracle's exact counts, columns and values on rows
    sampled from every power-of-two product range (the heaviest rows among them).
  * The 512-product batched workload in one persistent launch: every product.

The oracle runs in row chunks on all host cores (tests/oracle_par.py)."""
import numpy as np
import pytest

import oracle
from paper_2105_14156_gb300.rmat import batched_workload, workload
from tests import oracle_par
from tests.gpu_util import assert_matches_oracle, device_rows

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


@pytest.fixture(scope="module")
def model(handle):
    """A predictor trained on the device on R-MAT matrices of scales 12-16
    (the training recipe of the learned configuration, fewer matrices)."""
    from paper_2105_14156_gb300 import learned
    mats = learned.training_matrices(range(20), workers=8)
    m, loss, secs, n = learned.train(handle, mats, epochs=8, batch=4096)
    yield m
    m.close()


def test_rmat16_f64_plain_all_rows(handle):
    """R-MAT scale 16, edge factor 16, float64 U[-1,1], C = A*A: every row."""
    from paper_2105_14156_gb300 import smash
    A = workload("rmat16_f64")
    dA, dB = smash.to_device(A), smash.to_device(A)
    C = handle.spgemm(dA, dB, check=True).to_host()
    ref = oracle_par.spgemm_rows(A, A)
    assert_matches_oracle(C, A, A, ref=ref)


def test_rmat20_learned_autotuned_all_rows(handle, model):
    """R-MAT scale 20, edge factor 8, (.45,.15,.15,.25), float32 U[-1,1],
    C = A*A with learned sizing and the autotuned planner (heavy rows take
    the global-memory hash): every row; the plain path on the same handle too."""
    from paper_2105_14156_gb300 import autotune, smash
    A = workload("rmat20_f32")
    dA, dB = smash.to_device(A), smash.to_device(A)
    saved = handle.params.as_dict()
    try:
        autotune.tune(handle, dA, dB, "rmat20_f32", cache_path=None)
        C, stats, owner = handle.spgemm_learned(dA, dB, model, margin=0.15)
        handle.check()
        Ch = C.to_host()
        owner.free()
        del C
        Cp = handle.spgemm(dA, dB, check=True).to_host()
    finally:
        handle.set_params(**saved)
    ref = oracle_par.spgemm_rows(A, A)
    assert_matches_oracle(Ch, A, A, ref=ref)
    assert stats["c_nnz"] == Ch.col_idx.size
    assert_matches_oracle(Cp, A, A, ref=ref)


def _stratified_rows(flop, per_range=24, seed=0):
    """Up to per_range random rows from every range [2^b, 2^(b+1)) of products,
    the 16 heaviest rows and a few rows without products."""
    rng = np.random.default_rng(seed)
    picks = [np.argsort(flop)[-16:]]
    nz = flop > 0
    b = np.zeros_like(flop)
    b[nz] = np.floor(np.log2(flop[nz])).astype(flop.dtype)
    for r in range(0, int(b.max()) + 1):
        idx = np.flatnonzero(nz & (b == r))
        if idx.size:
            picks.append(rng.choice(idx, min(per_range, idx.size), replace=False))
    picks.append(np.flatnonzero(~nz)[:8])
    return np.unique(np.concatenate(picks))


def test_rmat18_learned_row_ptr_and_sampled_rows(handle, model):
    """R-MAT scale 18, edge factor 16, float32 U[-1,1], C = A*A with learned
    sizing: nnz(C_i) of every row against the oracle's exact count; columns and
    values of rows sampled from every product range."""
    from paper_2105_14156_gb300 import smash
    A = workload("rmat18_f32")
    dA, dB = smash.to_device(A), smash.to_device(A)
    C, stats, owner = handle.spgemm_learned(dA, dB, model, margin=0.15)
    handle.check()
    try:
        ref_nnz = oracle_par.row_nnz(A, A)
        got_nnz = np.diff(C.row_ptr.cpu().numpy())
        assert np.array_equal(got_nnz, ref_nnz), "row lengths differ on %d rows" % np.count_nonzero(
            got_nnz != ref_nnz)
        assert stats["c_nnz"] == int(ref_nnz.sum())
        rows = _stratified_rows(oracle.row_flops(A, A))
        sub = device_rows(C, rows)
    finally:
        owner.free()
    ref = oracle_par.spgemm_rows(A, A, rows=rows)
    assert_matches_oracle(sub, A, A, ref=ref)


def test_batched_512_all_products(handle):
    """The batched workload: 512 pairs (R-MAT A_i with n_i log-uniform in
    [64, 8192], degree U[4, 32]; B_i n_i x 256 at 5 % density; float32) in one
    persistent launch with the autotuned table size: every product."""
    import concurrent.futures as cf
    from paper_2105_14156_gb300 import smash
    pairs = batched_workload(512, seed=7)
    dev = smash.BatchedInputs([(smash.to_device(a), smash.to_device(b)) for a, b in pairs])
    handle.batched_autotune(dev)
    Cs, stats, owner = handle.spgemm_batched(dev)
    handle.check()
    host = [c.to_host() for c in Cs]
    owner.free()
    assert stats["products"] == 512
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        refs = list(ex.map(lambda p: oracle.spgemm(p[0], p[1]), pairs))
    for (A, B), C, ref in zip(pairs, host, refs):
        assert_matches_oracle(C, A, B, ref=ref)
