"""Failure detection without a GPU fault: a bounded in-kernel wait that runs
out (the batched kernel's grid barrier waiting for an arrival that never
comes) ends the call with SMASH_ERR_TIMEOUT and leaves the handle usable; an
allocator that returns NULL on its k-th call makes the call fail with
SMASH_ERR_ALLOC, nothing allocated through it stays allocated, and the handle
works again afterwards."""
import numpy as np
import pytest

from paper_2105_14156_gb300.rmat import GRAPH500_ABCD, batched_pair, rmat
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


def test_batched_barrier_wait_runs_out(handle):
    from paper_2105_14156_gb300 import smash
    pairs = [batched_pair(11, i, n_hi=600) for i in range(6)]
    dev = [(smash.to_device(a), smash.to_device(b)) for a, b in pairs]
    handle.batched_set_wait(4000, 1)      # about 1 ms, one arrival that never comes
    try:
        with pytest.raises(smash.SmashError) as ei:
            handle.spgemm_batched(dev)
        assert ei.value.status == 6       # SMASH_ERR_TIMEOUT
    finally:
        handle.batched_set_wait(0, 0)
    Cs, stats, owner = handle.spgemm_batched(dev)
    handle.check()
    host = [c.to_host() for c in Cs]
    owner.free()
    for (A, B), C in zip(pairs, host):
        assert_matches_oracle(C, A, B)


class CountingAllocator:
    """Device allocations through torch's caching allocator; the k-th request
    (counted from arm()) returns NULL. live: the blocks not yet freed."""

    def __init__(self, fail_at):
        self.fail_at = fail_at
        self.calls = 0
        self.armed = False
        self.live = {}

    def arm(self):
        self.armed = True
        self.calls = 0

    def alloc(self, nbytes):
        import torch
        if self.armed:
            self.calls += 1
            if self.calls == self.fail_at:
                return 0
        p = torch.cuda.caching_allocator_alloc(nbytes, 0, torch.cuda.current_stream())
        self.live[p] = nbytes
        return p

    def free(self, p):
        import torch
        torch.cuda.caching_allocator_delete(p)
        self.live.pop(p, None)


@pytest.mark.parametrize("path", ["plain", "learned", "bound", "batched"])
def test_allocation_failure_leaves_nothing_behind(handle, path):
    from paper_2105_14156_gb300 import smash
    A = rmat(11, 16, GRAPH500_ABCD, seed=71, values="f32")
    dA = smash.to_device(A)
    pairs = [batched_pair(12, i, n_hi=500) for i in range(4)]
    dpairs = [(smash.to_device(a), smash.to_device(b)) for a, b in pairs]
    model = smash.Model(handle, seed=3) if path == "learned" else None

    def run():
        if path == "plain":
            return None, handle.spgemm(dA, dA, check=True)
        if path in ("learned", "bound"):
            C, st, owner = handle.spgemm_learned(dA, dA, model if path == "learned" else None, margin=0.15)
            handle.check()
            return owner, C
        Cs, st, owner = handle.spgemm_batched(dpairs)
        handle.check()
        return owner, Cs

    failures = 0
    for k in range(1, 25):
        al = CountingAllocator(k)
        handle.set_allocator(al.alloc, al.free)
        al.arm()
        try:
            owner, _ = run()
            if owner is not None:
                owner.free()
        except smash.SmashError as e:
            assert e.status == 4, e      # SMASH_ERR_ALLOC, nothing else
            failures += 1
        # back to cudaMalloc: the handle's scratch goes back through al.free
        handle.set_allocator(None)
        assert not al.live, "%d blocks left allocated after failing at request %d" % (len(al.live), k)
        if al.calls < k:
            break                         # the call needed fewer than k allocations
    assert failures > 0
    # the handle works after the failures
    if path == "batched":
        owner, Cs = run()
        for (a, b), C in zip(pairs, [c.to_host() for c in Cs]):
            assert_matches_oracle(C, a, b)
        owner.free()
    else:
        owner, C = run()
        assert_matches_oracle(C.to_host(), A, A)
        if owner is not None:
            owner.free()
    if model is not None:
        model.close()
