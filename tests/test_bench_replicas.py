"""The N > 1 path of bench.py on the CPU: two gloo ranks, each an independent
replica with its own time (the rows of C are independent, so ranks exchange
nothing but the timing). The job's time is the slowest rank's, and its value
counts every rank's products."""
import os
import socket

import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), SMASH_BENCH_BACKEND="gloo")
    import bench
    r, w, local, dist = bench.dist_setup()
    assert (r, w, local) == (rank, world, rank)
    t = bench.replica_max(1.0 + rank, dist, "cpu")       # rank r took 1 + r seconds
    v = bench.replica_gflops(w, 10 ** 9, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_replicas_gloo():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert [r for r, _, _ in out] == [0, 1]
    for _, t, v in out:
        assert t == 2.0                     # the slowest replica's time
        assert abs(v - 2.0) < 1e-12         # 2 ranks x 2 flops x 1e9 products / 2 s = 2 GFLOP/s


def test_single_rank_is_identity():
    import bench
    assert bench.replica_max(1.25, None, "cpu") == 1.25
    assert abs(bench.replica_gflops(1, 5 * 10 ** 8, 0.5) - 2.0) < 1e-12
