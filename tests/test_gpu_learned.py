"""Learned sizing on the GPU: the MLP kernels against the float64 oracle, and
C = A*B through spgemm_learned against the SpGEMM oracle (structure exact,
values within tolerance), including forced under-prediction where every
overflowing row goes through the exact fallback."""
import numpy as np
import pytest

import oracle
from oracle import mlp as mlp_oracle
from paper_2105_14156_gb300.rmat import GRAPH500_ABCD, rmat
from tests.gpu_util import assert_matches_oracle

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


@pytest.fixture(scope="module")
def trained(handle):
    from paper_2105_14156_gb300 import learned
    from paper_2105_14156_gb300.rmat import training_matrix
    mats = [training_matrix(s) for s in (0, 5, 10, 1, 6)]   # scales 12 and 13
    model, loss, secs, n = learned.train(handle, mats, epochs=40, batch=512)
    return model, loss, n


def bf16_round(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def test_gradient_matches_oracle(handle):
    import torch
    from paper_2105_14156_gb300 import smash
    rng = np.random.default_rng(3)
    model = smash.Model(handle, seed=7)
    p = rng.normal(0, 0.2, smash.MLP_PARAMS).astype(np.float32)
    norm = np.concatenate([rng.normal(0, 1, 6), rng.uniform(0.5, 2, 6)]).astype(np.float32)
    model.set(p, norm)
    feats = rng.normal(0, 2, (1000, 6)).astype(np.float32)
    targets = rng.normal(0, 1, 1000).astype(np.float32)
    g, loss = handle.mlp_gradient(model, torch.from_numpy(feats).cuda(), torch.from_numpy(targets).cuda())
    x = mlp_oracle.normalise(feats, norm[:6].astype(np.float64), norm[6:].astype(np.float64))
    ref_loss, ref_g = mlp_oracle.loss_and_grad(p.astype(np.float64), x, targets.astype(np.float64))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - ref_loss) <= 1e-4 * max(1.0, ref_loss)
    scale = np.max(np.abs(ref_g))
    assert np.max(np.abs(g - ref_g)) <= 2e-4 * scale, np.max(np.abs(g - ref_g)) / scale
    model.close()


def test_predict_matches_oracle_with_bf16_weights(handle):
    import torch
    from paper_2105_14156_gb300 import smash
    rng = np.random.default_rng(4)
    model = smash.Model(handle, seed=9)
    p = rng.normal(0, 0.2, smash.MLP_PARAMS).astype(np.float32)
    norm = np.concatenate([rng.normal(0, 1, 6), rng.uniform(0.5, 2, 6)]).astype(np.float32)
    model.set(p, norm)
    feats = rng.normal(0, 2, (500, 6)).astype(np.float32)
    y = handle.mlp_predict(model, torch.from_numpy(feats).cuda()).cpu().numpy()
    x = mlp_oracle.normalise(feats, norm[:6].astype(np.float64), norm[6:].astype(np.float64))
    ref, _ = mlp_oracle.forward(bf16_round(p).astype(np.float64), x)
    assert np.max(np.abs(y - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
    model.close()


def test_tensor_core_predict_within_bf16_activation_bound(handle):
    """The forward pass of the learned path (layer 2 on the tensor cores, the
    layer-1 activations rounded to bf16, fp32 accumulation) against the float64
    oracle with the same bf16 weights. Rounding h1 to bf16 changes each h1_v by
    at most 2^-9 |h1_v|, so per row |y - y*| <= 2^-9 sum_u |w3_u| sum_v
    |W2_uv| |h1_v| (relu is 1-Lipschitz), plus fp32 accumulation error."""
    import torch
    from oracle.mlp import unpack
    from paper_2105_14156_gb300 import smash
    rng = np.random.default_rng(5)
    model = smash.Model(handle, seed=10)
    p = rng.normal(0, 0.2, smash.MLP_PARAMS).astype(np.float32)
    norm = np.concatenate([rng.normal(0, 1, 6), rng.uniform(0.5, 2, 6)]).astype(np.float32)
    model.set(p, norm)
    n = 1000   # 31 full warps of 32 rows and a ragged one
    feats = rng.normal(0, 2, (n, 6)).astype(np.float32)
    y = handle.mlp_predict(model, torch.from_numpy(feats).cuda(), tensor_cores=True).cpu().numpy()
    pb = bf16_round(p).astype(np.float64)
    x = mlp_oracle.normalise(feats, norm[:6].astype(np.float64), norm[6:].astype(np.float64))
    ref, (_, _, h1, _, _) = mlp_oracle.forward(pb, x)
    w = unpack(pb)
    bound = 2.0 ** -9 * (np.abs(h1) @ np.abs(w["W2"]).T) @ np.abs(w["w3"])
    err = np.abs(y - ref)
    assert np.all(err <= 1.01 * bound + 1e-4 * np.maximum(1.0, np.abs(ref))), np.max(err - bound)
    # and the bound is not vacuous: the two forward passes differ
    assert np.max(err) > 0
    model.close()


def test_save_load_roundtrip(handle, tmp_path):
    from paper_2105_14156_gb300 import smash
    m1 = smash.Model(handle, seed=11)
    p, n = m1.get()
    path = str(tmp_path / "m.bin")
    m1.save(path)
    m2 = smash.Model(handle, seed=12)
    m2.load(path)
    p2, n2 = m2.get()
    assert np.array_equal(p, p2) and np.array_equal(n, n2)
    m1.close()
    m2.close()


def test_training_reduces_loss(handle, trained):
    model, loss, n = trained
    assert n > 10000
    assert loss < 0.2, loss     # mean squared error of log1p(nnz)


@pytest.mark.parametrize("values", ["f64", "f32"])
def test_learned_matches_oracle(handle, trained, values):
    from paper_2105_14156_gb300 import smash
    model, _, _ = trained
    A = rmat(12, 16, GRAPH500_ABCD, seed=33, values=values)
    dA = smash.to_device(A)
    C, stats, owner = handle.spgemm_learned(dA, dA, model, margin=0.15)
    Ch = C.to_host()
    owner.free()
    assert_matches_oracle(Ch, A, A)
    assert stats["c_nnz"] == Ch.col_idx.size
    assert stats["overflow_rows"] < 0.2 * A.rows


def test_forced_underprediction_falls_back(handle, trained):
    from paper_2105_14156_gb300 import smash
    model, _, _ = trained
    A = rmat(11, 16, GRAPH500_ABCD, seed=34, values="int4")
    dA = smash.to_device(A)
    C, stats, owner = handle.spgemm_learned(dA, dA, model, margin=-0.9)
    Ch = C.to_host()
    owner.free()
    assert stats["overflow_rows"] > 0.5 * np.count_nonzero(np.diff(Ch.row_ptr))
    assert_matches_oracle(Ch, A, A, exact=True)


def test_learned_rectangular_and_empty_rows(handle, trained):
    from paper_2105_14156_gb300 import smash
    from tests.helpers import random_csr
    model, _, _ = trained
    A = random_csr(500, 300, 0.02, 61, values="f64")
    B = random_csr(300, 900, 0.03, 62, values="f64")
    for margin in (0.15, -0.5, 3.0):
        C, stats, owner = handle.spgemm_learned(smash.to_device(A), smash.to_device(B), model, margin=margin)
        Ch = C.to_host()
        owner.free()
        assert_matches_oracle(Ch, A, B)


@pytest.mark.parametrize("margin", [0.15, -0.6, 3.0])
@pytest.mark.parametrize("values", ["f32", "f64"])
def test_learned_many_tiny_rows(handle, trained, margin, values):
    """Enough rows of a few products for the thread-per-row bins in capacity
    mode: rows that fit their predicted room are written there, the others
    (forced by the negative margin) overflow to the exact fallback."""
    from paper_2105_14156_gb300 import smash
    from tests.helpers import random_csr
    model, _, _ = trained
    A = random_csr(60000, 20000, 0.00015, 91, values=values)
    B = random_csr(20000, 50000, 0.00006, 92, values=values, sort_cols=False, dup_frac=0.2)
    C, stats, owner = handle.spgemm_learned(smash.to_device(A), smash.to_device(B), model, margin=margin)
    Ch = C.to_host()
    owner.free()
    assert_matches_oracle(Ch, A, B)
    assert stats["c_nnz"] == Ch.col_idx.size


@pytest.mark.parametrize("margin", [0.15, -0.6, 3.0])
@pytest.mark.parametrize("values", ["f32", "f64"])
def test_learned_row_windows(handle, trained, margin, values):
    """Row windows in capacity mode: windows whose rows fit their predicted
    room are staged and merged, the others hashed; rows over their room
    (forced by the negative margin) are marked and redone by the exact
    fallback, the other rows of their window are kept."""
    from paper_2105_14156_gb300 import smash
    from tests.helpers import random_csr
    model, _, _ = trained
    A = random_csr(30011, 20000, 0.00015, 191, values=values)
    B = random_csr(20000, 50000, 0.00006, 192, values=values, sort_cols=False, dup_frac=0.2)
    defaults = handle.params.as_dict()
    handle.set_params(row_window=16, row_window_tbits=8)
    try:
        C, stats, owner = handle.spgemm_learned(smash.to_device(A), smash.to_device(B), model, margin=margin)
        handle.check()
        Ch = C.to_host()
        owner.free()
        R = rmat(12, 8, GRAPH500_ABCD, seed=193, values=values)
        dR = smash.to_device(R)
        C2, stats2, owner2 = handle.spgemm_learned(dR, dR, model, margin=margin)
        handle.check()
        C2h = C2.to_host()
        owner2.free()
    finally:
        handle.set_params(**defaults)
    assert_matches_oracle(Ch, A, B)
    assert stats["c_nnz"] == Ch.col_idx.size
    assert_matches_oracle(C2h, R, R)
    if margin < 0:
        assert stats["overflow_rows"] > 0


@pytest.mark.parametrize("margin", [0.15, -0.9, 3.0])
@pytest.mark.parametrize("dense_blocks", [2, 4])
@pytest.mark.parametrize("owner", [0, 1])
def test_learned_dense_rows_in_arena(handle, trained, margin, dense_blocks, owner):
    """Dense rows of the learned path: column-window items write into the arena
    (several windows per row); an arena too small for them (margin -0.9) sends
    the rows to the exact fallback."""
    from paper_2105_14156_gb300 import smash
    from tests.helpers import random_csr
    model, _, _ = trained
    A = random_csr(300, 200, 0.1, 81, values="f64")
    B = random_csr(200, 30000, 0.01, 82, values="f64")
    defaults = handle.params.as_dict()
    handle.set_params(dense_ratio=1 << 20, dense_blocks=dense_blocks, dense_owner=owner)
    try:
        C, stats, owner = handle.spgemm_learned(smash.to_device(A), smash.to_device(B), model, margin=margin)
        Ch = C.to_host()
        owner.free()
    finally:
        handle.set_params(**defaults)
    assert_matches_oracle(Ch, A, B)
    if margin < 0:
        assert stats["overflow_rows"] > 0


@pytest.mark.parametrize("margin", [0.15, -0.9, 3.0])
@pytest.mark.parametrize("values", ["f32", "f64"])
def test_learned_global_hash_rows(handle, trained, margin, values):
    """Capacity mode of the global-memory hash: shared-memory tables capped at
    32 slots and no dense rows, so every row with a predicted capacity above
    16 hashes in global memory. Rows that fit their predicted room are written
    there; rows whose table or room proves too small (forced by margin -0.9)
    take the exact fallback."""
    from paper_2105_14156_gb300 import smash
    model, _, _ = trained
    A = rmat(11, 16, GRAPH500_ABCD, seed=35, values=values)
    defaults = handle.params.as_dict()
    handle.set_params(num_max_tbits=5, sym_max_tbits=5, dense_ratio=0, sym_dense_ratio=0)
    try:
        dA = smash.to_device(A)
        C, stats, owner = handle.spgemm_learned(dA, dA, model, margin=margin)
        handle.check()
        Ch = C.to_host()
        owner.free()
    finally:
        handle.set_params(**defaults)
    assert_matches_oracle(Ch, A, A)
    assert stats["c_nnz"] == Ch.col_idx.size
    if margin < 0:
        assert stats["overflow_rows"] > 0


@pytest.mark.parametrize("margin", [0.15, -0.9])
def test_learned_dense_rows_without_windows(handle, trained, margin):
    """Dense rows whose few products do not pay for slicing a tall B by column
    window: in the learned path they hash in global memory in capacity mode
    (no arena), fitting or (margin -0.9) overflowing to the exact fallback."""
    from paper_2105_14156_gb300 import smash
    from tests.helpers import random_csr
    model, _, _ = trained
    A = random_csr(40, 100000, 5e-5, 71, values="f64")
    B = random_csr(100000, 200000, 5e-5, 72, values="f64")
    defaults = handle.params.as_dict()
    handle.set_params(dense_ratio=1 << 20)
    try:
        C, stats, owner = handle.spgemm_learned(smash.to_device(A), smash.to_device(B), model, margin=margin)
        handle.check()
        Ch = C.to_host()
        owner.free()
    finally:
        handle.set_params(**defaults)
    assert_matches_oracle(Ch, A, B)
    assert stats["c_nnz"] == Ch.col_idx.size


def test_training_rows_targets_from_exact_counts(handle):
    """Training samples made by the library: one per row with products, in row
    order; the target is log1p of the oracle's exact row count and feature 1
    is log1p of the row's product count."""
    import oracle
    from paper_2105_14156_gb300 import smash
    A = rmat(11, 16, GRAPH500_ABCD, seed=37, values="f32")
    dA = smash.to_device(A)
    f, t = handle.training_rows(dA, dA)
    flop = oracle.row_flops(A, A)
    keep = np.flatnonzero(flop > 0)
    assert f.shape == (keep.size, 6) and t.shape == (keep.size,)
    nnz = oracle.row_nnz(A, A)[keep]
    t = t.cpu().numpy()
    assert np.allclose(t, np.log1p(nnz.astype(np.float64)), rtol=1e-6, atol=0)
    f1 = f[:, 1].cpu().numpy()
    assert np.allclose(f1, np.log1p(flop[keep].astype(np.float64)), rtol=1e-6, atol=0)


@pytest.mark.parametrize("values", ["f32", "f64"])
def test_bound_sized_one_pass_matches_oracle(handle, values):
    """The one-pass pipeline without the network (every row sized by its bound
    min(flop_i, cols)): exact C, no row overflows."""
    from paper_2105_14156_gb300 import smash
    A = rmat(12, 16, GRAPH500_ABCD, seed=38, values=values)
    dA = smash.to_device(A)
    C, stats, owner = handle.spgemm_learned(dA, dA, None)
    handle.check()
    Ch = C.to_host()
    owner.free()
    assert_matches_oracle(Ch, A, A)
    assert stats["overflow_rows"] == 0
    assert stats["c_nnz"] == Ch.col_idx.size

@pytest.mark.parametrize("values", ["f32", "f64"])
@pytest.mark.parametrize("group_shift", [4, 2])
def test_bound_sized_thread_group_merge(handle, values, group_shift):
    """Capacity mode in the thread-group rows: every row's ~1200 products fit
    its room (the bound min(flop_i, cols)), so they are staged, sorted and
    merged (about a fifth of them repeat a column) instead of hashed."""
    from paper_2105_14156_gb300 import smash
    from tests.helpers import random_csr
    A = random_csr(3001, 300, 0.02, 195, values=values)
    B = random_csr(300, 3000, 0.067, 196, values=values)
    defaults = handle.params.as_dict()
    handle.set_params(group_shift=group_shift)
    try:
        dA, dB = smash.to_device(A), smash.to_device(B)
        C, stats, owner = handle.spgemm_learned(dA, dB, None)
        handle.check()
        Ch = C.to_host()
        owner.free()
    finally:
        handle.set_params(**defaults)
    assert_matches_oracle(Ch, A, B)
    assert stats["overflow_rows"] == 0


def _vstack(*mats):
    from paper_2105_14156_gb300.rmat import Csr
    rp = [np.zeros(1, np.int64)]
    base = 0
    for m in mats:
        rp.append(m.row_ptr[1:] + base)
        base += m.nnz
    return Csr(sum(m.rows for m in mats), mats[0].cols, np.concatenate(rp),
               np.concatenate([m.col_idx for m in mats]), np.concatenate([m.val for m in mats]))


@pytest.mark.parametrize("margin", [0.15, -0.6, 3.0, None])
@pytest.mark.parametrize("values", ["f32", "f64"])
def test_learned_compaction_mixed_row_lengths(handle, trained, margin, values):
    """The copy of staged rows into C over stretches of rows of a few entries
    (a stretch of output spans more rows than a block lists, so its warps walk
    the rows), rows of a few hundred entries (rows listed in shared memory),
    rows of ~16,000 entries (stretches inside one row, skipped whole when the
    row is written elsewhere), empty rows between, and overflowing rows the
    copy skips (negative margin); None sizes every row by its bound."""
    from paper_2105_14156_gb300 import smash
    from tests.helpers import random_csr
    model, _, _ = trained
    A = _vstack(random_csr(20000, 2000, 0.00025, 401, values=values),
                random_csr(1500, 2000, 0.015, 402, values=values),
                random_csr(4, 2000, 3.0, 406, values=values),
                random_csr(20000, 2000, 0.00025, 403, values=values),
                random_csr(700, 2000, 0.015, 404, values=values))
    B = random_csr(2000, 80000, 0.000125, 405, values=values)
    C, stats, owner = handle.spgemm_learned(smash.to_device(A), smash.to_device(B),
                                            None if margin is None else model,
                                            **({} if margin is None else {"margin": margin}))
    handle.check()
    Ch = C.to_host()
    owner.free()
    assert_matches_oracle(Ch, A, B)
    assert stats["c_nnz"] == Ch.col_idx.size
    if margin is not None and margin < 0:
        assert stats["overflow_rows"] > 0
