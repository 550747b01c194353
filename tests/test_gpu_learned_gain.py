"""What the trained row-size network gains over the same one-pass pipeline
without it (every row sized by its bound min(flop_i, cols)), on an R-MAT
product whose rows repeat columns (products / nnz(C) above 2): both give the
exact C; the network's capacities stage far fewer entries than the bound's,
few rows overflow to the exact fallback, and the staged bytes are what the
one-pass pipeline moves twice (write, then compaction into C)."""
import numpy as np
import pytest

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


def test_network_stages_less_than_the_bound(handle):
    import time
    import torch
    import oracle
    from paper_2105_14156_gb300 import learned, smash
    from paper_2105_14156_gb300.rmat import training_matrix
    mats = [training_matrix(s) for s in range(10)]          # scales 12-16, seeds 0-9
    model, loss, _, _ = learned.train(handle, mats, epochs=8, batch=4096)
    A = rmat(14, 16, GRAPH500_ABCD, seed=41, values="f32")   # not in the training set
    dA = smash.to_device(A)
    flop = oracle.row_flops(A, A)
    res = {}
    for name, m in (("network", model), ("bound", None)):
        C, st, owner = handle.spgemm_learned(dA, dA, m, margin=0.3)
        handle.check()
        Ch = C.to_host()
        owner.free()
        assert_matches_oracle(Ch, A, A)
        # the time of a second call (warm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C2, st2, o2 = handle.spgemm_learned(dA, dA, m, margin=0.3)
        torch.cuda.synchronize()
        res[name] = dict(st, ms=1e3 * (time.perf_counter() - t0))
        o2.free()
    cnnz = res["network"]["c_nnz"]
    assert flop.sum() > 2 * cnnz                             # columns repeat: cf > 2
    s_net = res["network"]["staged_nnz"] / cnnz
    s_bound = res["bound"]["staged_nnz"] / cnnz
    print("staged / nnz(C): network %.2f, bound %.2f; overflow rows %d of %d; ms network %.2f bound %.2f"
          % (s_net, s_bound, res["network"]["overflow_rows"], A.rows, res["network"]["ms"], res["bound"]["ms"]))
    assert res["bound"]["overflow_rows"] == 0
    assert res["network"]["overflow_rows"] <= 0.05 * A.rows
    assert s_net < 0.8 * s_bound
    model.close()
