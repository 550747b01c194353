"""The symbolic entry point that allocates nothing, against spgemm_symbolic.

spgemm_symbolic_noalloc serves callers that cannot allocate device memory:
all of its scratch lives in a fixed array inside the library. It must give
the same row pointer and nnz(C) as the regular symbolic phase (integer
counts: exact), on consecutive calls that reuse the shared array, and refuse
inputs wider than its limit. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2105_14156_gb300.rmat import GRAPH500_ABCD, rmat
from tests.helpers import random_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_and_handle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_14156_gb300 import build, smash
    build.build()
    torch.cuda.set_device(0)
    h = smash.Handle(0)
    yield smash.load_library(), h
    h.close()


def noalloc_symbolic(lib, A, B):
    import torch
    from paper_2105_14156_gb300 import smash
    c_rp = torch.full((A.rows + 1,), -7, dtype=torch.int64, device="cuda")
    nnz = ctypes.c_int64(-1)
    sa, sb = A.struct(), B.struct()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.spgemm_symbolic_noalloc(ctypes.byref(sa), ctypes.byref(sb), c_rp.data_ptr(), ctypes.byref(nnz), stream)
    return st, c_rp, int(nnz.value)


def test_noalloc_matches_symbolic_twice(lib_and_handle):
    from paper_2105_14156_gb300 import smash
    lib, h = lib_and_handle
    cases = [
        (rmat(12, 16, GRAPH500_ABCD, seed=71, values="f32"), None),
        (random_csr(900, 700, 0.02, 72, values="f32", sort_cols=False, dup_frac=0.2),
         random_csr(700, 60000, 0.01, 73, values="f32")),
    ]
    for A, B in cases:
        B = A if B is None else B
        dA, dB = smash.to_device(A), smash.to_device(B)
        ref_rp, ref_nnz = h.symbolic(dA, dB)
        for _ in range(2):
            st, c_rp, nnz = noalloc_symbolic(lib, dA, dB)
            assert st == 0, smash.STATUS.get(st)
            assert nnz == ref_nnz
            assert np.array_equal(c_rp.cpu().numpy(), ref_rp.cpu().numpy())


def test_noalloc_rejects_wide_b(lib_and_handle):
    from paper_2105_14156_gb300 import smash
    lib, _ = lib_and_handle
    A = random_csr(20, 30, 0.2, 74, values="f32")
    B = random_csr(30, 70000, 0.001, 75, values="f32")
    st, _, _ = noalloc_symbolic(lib, smash.to_device(A), smash.to_device(B))
    assert st == 3   # SMASH_ERR_UNSUPPORTED
