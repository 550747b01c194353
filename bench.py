"""Benchmark of the SMASH row-wise hash SpGEMM on GB300, through the C ABI.

Main line (value): R-MAT scale 20 (1,048,576 x 1,048,576), edge factor 8,
(a,b,c,d) = (.45,.15,.15,.25), float32 U[-1,1], C = A*A with learned sizing
(the row-size network trained on the device on 200 seeded R-MAT matrices of
scales 12-16, outside the timed region) and the planner parameters chosen by
the autotuner; heavy rows take the global-memory hash. One step = the whole
spgemm_learned call with A and B resident in HBM: per-row counts, the network
and the bins, one hashing pass into a capacity-sized staging buffer, the
exact fallback for rows that did not fit, C's row pointer, C's allocation and
assembly. L2 (129 MB) is flushed between timed steps by writing a 256 MiB
buffer outside the timed region. value = useful GFLOP/s = 2 * products / step
time (CUDA events on the launching stream).

Variants (same JSON line, "variants", each timed over --variant-steps steps):
the plain two-pass path and the one-pass path sized by the bound min(flop_i,
cols) (the pipeline without the network) on the same workload; R-MAT scale 18
(learned / bound / plain); 512 batched products in one persistent launch
against 512 separate plain calls and against one plain call on their
block-diagonal concatenation; R-MAT scale 16 float64 (plain); the paper-like
product of two independent R-MAT scale-14 matrices (float64, plain).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl smash|reference]
                       [--variants all|none] [--workload NAME] [--path learned|plain|bound]
With torchrun (N > 1) every rank runs an independent replica (the rows of C
are independent; no exchange step): value = all ranks' products / max time.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpGEMM useful GFLOP/s and HBM GB/s: learned/batched vs plain hash, same GB300"
WORKLOADS = {
    "rmat20_f32": "R-MAT scale 20 (1048576 x 1048576), edge factor 8, (a,b,c,d)=(0.45,0.15,0.15,0.25), "
                  "float32 U[-1,1], C = A*A (A and B separate copies)",
    "rmat16_f64": "R-MAT scale 16 (65536 x 65536), edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
                  "float64 values U[-1,1], C = A*A (A and B separate copies)",
    "rmat10_int": "R-MAT scale 10, edge factor 8, (0.57,0.19,0.19,0.05), float32 integer values {1..4}, C = A*A",
    "rmat17_f32": "R-MAT scale 17, edge factor 16, (0.57,0.19,0.19,0.05), float32 U[-1,1], C = A*A "
                  "(a smaller case of the scale-18 workload, for captures)",
    "rmat18_f32": "R-MAT scale 18, edge factor 16, (0.57,0.19,0.19,0.05), float32 U[-1,1], C = A*A",
}
PATHS = {"learned": "learned sizing (row-size network) + autotuned planner",
         "bound": "one pass sized by min(flop_i, cols) + autotuned planner",
         "plain": "plain two-pass (symbolic, then numeric) + autotuned planner"}
TRAIN_SEEDS = list(range(200))


def row_products(A, B) -> np.ndarray:
    """flop_i = sum over A_i of |B_k| (host bookkeeping for the metric)."""
    blen = np.diff(B.row_ptr)
    per = blen[A.col_idx].astype(np.int64)
    out = np.zeros(A.rows, dtype=np.int64)
    nz = np.diff(A.row_ptr) > 0
    if per.size:
        out[nz] = np.add.reduceat(per, A.row_ptr[:-1][nz])
    return out


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def source_hash() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2105_14156_gb300", "csrc", "*"))):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def smem_atomic_peak(vb: int):
    """Measured shared-memory atomic add rate (Gop/s, random slots, whole GPU)
    for the value type, from the committed probe summary."""
    path = os.path.join(ROOT, "profiles", "smem_atomics_gb300.md")
    key = "| f64 add, local, spread |" if vb == 8 else "| f32 add, local, spread |"
    try:
        for line in open(path):
            if line.startswith(key):
                return float(line.split("|")[2])
    except OSError:
        pass
    return None


def chunked_copies(pairs, streams, main, chunk_bytes=64 << 20):
    """dst.copy_(src) for each (dst, src) pair between pinned host memory and the
    device, cut into chunks dealt round-robin to `streams` (several copy engines
    at once); the copy streams start after the work queued on `main`, and `main`
    waits for them."""
    import torch
    for cs in streams:
        cs.wait_stream(main)
    q = 0
    for dst, src in pairs:
        n = src.numel()
        step = max(1, chunk_bytes // max(1, src.element_size()))
        for a in range(0, n, step):
            cs = streams[q % len(streams)]
            q += 1
            with torch.cuda.stream(cs):
                dst[a:a + step].copy_(src[a:a + step], non_blocking=True)
    for cs in streams:
        main.wait_stream(cs)


E2E_BLOCKS = 4


def end_to_end(h, args, A, B, flop, model, margin, stream, dev, blocks):
    """Median seconds of the product through the public API with host buffers:
    every step copies A and B from pinned host memory and C back to pinned host
    memory inside the timed region. blocks > 1: A is cut into that many row
    blocks of about equal products, each multiplied by its own call; a block's
    C goes back to the host on a copy stream while the next block computes
    (C's row pointer shifted by the entries of the blocks before it)."""
    import torch
    from paper_2105_14156_gb300 import smash
    cum = np.concatenate([[0], np.cumsum(flop)])
    cuts = [0] + [int(np.searchsorted(cum, cum[-1] * q / blocks)) for q in range(1, blocks)] + [A.rows]
    cuts = sorted(set(min(max(c, 0), A.rows) for c in cuts))
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    # inputs: B whole; A's columns and values whole, its row pointer per block (rebased to 0)
    h_in = [pin(B.row_ptr), pin(B.col_idx), pin(B.val), pin(A.col_idx), pin(A.val)]
    h_rp = [pin(A.row_ptr[r0:r1 + 1] - A.row_ptr[r0]) for r0, r1 in zip(cuts[:-1], cuts[1:])]
    h2d = sum(t.numel() * t.element_size() for t in h_in + h_rp)
    copy_streams = [torch.cuda.Stream(dev) for _ in range(4)]
    times, out_host, d2h = [], None, 0
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_in = [torch.empty(t.shape, dtype=t.dtype, device=dev) for t in h_in]
        d_rp = [torch.empty(t.shape, dtype=t.dtype, device=dev) for t in h_rp]
        chunked_copies(list(zip(d_in + d_rp, h_in + h_rp)), copy_streams, stream)
        dB = smash.DeviceCsr(B.rows, B.cols, d_in[0], d_in[1], d_in[2])
        keep, off = [], 0
        for q, (r0, r1) in enumerate(zip(cuts[:-1], cuts[1:])):
            a0, a1 = int(A.row_ptr[r0]), int(A.row_ptr[r1])
            dA = smash.DeviceCsr(r1 - r0, A.cols, d_rp[q], d_in[3][a0:a1], d_in[4][a0:a1])
            owner = None
            if args.path == "plain":
                C = h.spgemm(dA, dB, stream)
            else:
                C, _, owner = h.spgemm_learned(dA, dB, model if args.path == "learned" else None, margin=margin,
                                               stream=stream)
            if out_host is None:
                # sized on the untimed first step (the product's nnz is fixed)
                out_host = [torch.zeros(A.rows + 1, dtype=torch.int64).pin_memory(),
                            torch.empty(int(1.2 * sum(flop)) + 1, dtype=torch.int32).pin_memory(),
                            torch.empty(int(1.2 * sum(flop)) + 1, dtype=C.val.dtype).pin_memory()]
            n = C.nnz
            rp = C.row_ptr[1:] + off if off else C.row_ptr[1:]
            cs = copy_streams[q % len(copy_streams)]
            cs.wait_stream(stream)
            with torch.cuda.stream(cs):
                out_host[0][r0 + 1:r1 + 1].copy_(rp, non_blocking=True)
                out_host[1][off:off + n].copy_(C.col_idx, non_blocking=True)
                out_host[2][off:off + n].copy_(C.val, non_blocking=True)
            keep.append((C, rp, owner))
            off += n
        for cs in copy_streams:
            stream.wait_stream(cs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        d2h = 8 * (A.rows + 1) + (4 + out_host[2].element_size()) * off
        if k > 0:
            times.append(dt)
        for C, rp, owner in keep:
            if owner is not None:
                owner.free()
        del keep, d_in, d_rp, dB
    # (untimed) the assembled row pointer ends at the entries copied
    assert int(out_host[0][A.rows]) == off
    return {"seconds": statistics.median(times), "h2d": h2d, "d2h": d2h, "blocks": len(cuts) - 1,
            "c": (out_host[0], out_host[1][:off], out_host[2][:off])}


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = source_hash()
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("workload") == workload and f.get("src") == cur:
            return float(f["dram_bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        win = [s for (t, s) in self.samples if t0 - 0.15 <= t <= t1 + 0.15]
        if not win and self.samples:
            win = [min(self.samples, key=lambda x: abs(x[0] - (t0 + t1) / 2))[1]]
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(s[1]) for s in win if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in win if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in win for k in range(4) if len(s) > 5 + k and s[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(win)}


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(os.environ.get("SMASH_BENCH_BACKEND", "nccl"))
    return rank, world, local, dist


def replica_max(local: float, dist, device) -> float:
    """Max over ranks of a per-rank time: the job of N replicas ends with its
    slowest one (identity on a single rank)."""
    if not dist:
        return local
    import torch
    t = torch.tensor([local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_gflops(world: int, products: int, seconds: float) -> float:
    """Whole-job useful GFLOP/s of N replicas: every rank multiplied the same
    operands (2 flops per product), all in the max-over-ranks time."""
    from paper_2105_14156_gb300 import metrics
    return world * metrics.useful_gflops(products, seconds)


def oracle_rows(A, B, rows, threads: int):
    """The oracle, as it stands, on the given rows: in one call (threads = 1)
    or in contiguous row chunks on `threads` host threads (its C calls release
    the interpreter lock)."""
    import oracle
    if threads <= 1:
        oracle.spgemm(A, B, rows=rows)
        return
    chunks = np.array_split(rows, 4 * threads)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda c: oracle.spgemm(A, B, rows=c), [c for c in chunks if c.size]))


def sample_rows(A, flop, budget_products: float, seed: int):
    rng = np.random.default_rng(seed)
    order = rng.permutation(A.rows)
    cum = np.cumsum(flop[order])
    k = int(np.searchsorted(cum, budget_products)) + 1
    return np.sort(order[:min(k, A.rows)])


def cpu_baseline(A, B, flop, budget_products: float, seed: int = 0):
    """The oracle as it stands on a seeded random sample of rows, single-threaded
    and on all host cores (the main figure)."""
    import oracle
    oracle.build()
    rows = sample_rows(A, flop, budget_products, seed)
    prods = int(flop[rows].sum())
    cores = os.cpu_count() or 1
    out = {}
    for threads in (1, cores):
        t0 = time.perf_counter()
        oracle_rows(A, B, rows, threads)
        dt = time.perf_counter() - t0
        out[threads] = (2.0 * prods / dt / 1e9, dt)
    cpu = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                cpu = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    sample = "%d of %d rows drawn at random (seed %d), %d of %d products" % (rows.size, A.rows, seed, prods,
                                                                            int(flop.sum()))
    return {"value": out[cores][0], "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": sample + ", %.1f s on %d threads" % (out[cores][1], cores),
            "host_cpu": cpu,
            "single_thread": {"value": out[1][0], "unit": "GFLOP/s", "cores": 1,
                              "sample": sample + ", %.1f s on 1 thread" % out[1][1]}}


def run_reference(args, A, B, flop, rank):
    """Reference arm: the CPU oracle as it stands, on all host cores, on bounded
    samples of the workload."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    per_step = float(os.environ.get("SMASH_REF_STEP_PRODUCTS", "1e8"))
    vals = []
    for k in range(args.warmup + args.steps):
        rows = sample_rows(A, flop, per_step, seed=k)
        prods = int(flop[rows].sum())
        t0 = time.perf_counter()
        oracle_rows(A, B, rows, cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            vals.append(2.0 * prods / dt / 1e9)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 2.0 * per_step / (value * 1e9) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if A.val.dtype == np.float64 else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload]},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": "each step: rows drawn at random until about %.0e products, %d threads"
                                       % (per_step, cores)},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed(fn, steps, flush, stream):
    """Per-step CUDA-event times (ms), L2 flushed before every step."""
    import torch
    out = []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
        del r
    return out


def kernel_bytes(t, vb, nnz_b, total_products):
    """Algorithmic bytes of one timed launch group: A, B and C each moved once,
    B's bytes shared out over the launch groups by their products."""
    rows, a_nnz, prods, c_nnz = t["rows"], t["a_nnz"], t["products"], t["c_nnz"]
    share = prods / total_products if total_products else 0.0
    if t["name"] in ("sym_hash", "sym_warp", "sym_rowwin", "sym_tiny", "sym_dense", "sym_spill", "num_dense_count"):
        return 12 * rows + 4 * a_nnz + 4 * nnz_b * share
    if t["name"] in ("num_hash", "num_warp", "num_rowwin", "num_group", "num_tiny", "num_spill", "num_dense_window"):
        return 16 * rows + (4 + vb) * (a_nnz + c_nnz) + (4 + vb) * nnz_b * share
    return None


def step_fn(h, path, dA, dB, model, stream, stats=None, margin=0.15):
    """One product on the chosen path; returns a callable for timed()."""
    if path == "plain":
        return lambda: h.spgemm(dA, dB, stream)

    def f():
        C, st, owner = h.spgemm_learned(dA, dB, model if path == "learned" else None, margin=margin, stream=stream)
        if stats is not None:
            stats.update(st)
        owner.free()
    return f


def tune_margin(h, dA, dB, model, stream, flush, candidates=(0.05, 0.15, 0.3, 0.6)):
    """The learned path's capacity margin with the shortest product (median of
    3 timed runs each), the learned-sizing counterpart of the planner's tuner."""
    best, best_ms = 0.15, float("inf")
    for m in candidates:
        f = step_fn(h, "learned", dA, dB, model, stream, margin=m)
        f()
        t = statistics.median(timed(f, 3, flush, stream))
        if t < best_ms:
            best, best_ms = m, t
    return best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="smash", choices=["smash", "reference"])
    ap.add_argument("--workload", default="rmat20_f32", choices=sorted(WORKLOADS))
    ap.add_argument("--path", default="learned", choices=sorted(PATHS))
    ap.add_argument("--cpu-products", type=float, default=1e8)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-blocks", type=int, default=E2E_BLOCKS,
                    help="row blocks of A in the end-to-end measurement (1: one call)")
    ap.add_argument("--variants", default="all", choices=["all", "none"])
    ap.add_argument("--variant-steps", type=int, default=10)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--params", default=None,
                    help='planner parameters as JSON, e.g. \'{"hash_kind": 2}\' (implies --no-autotune)')
    ap.add_argument("--save-model", default=None, help="write the trained row-size model to this file")
    ap.add_argument("--load-model", default=None, help="use this trained model instead of training one")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.e2e_steps = max(args.e2e_steps, 1)

    from paper_2105_14156_gb300 import metrics
    from paper_2105_14156_gb300.rmat import workload

    rank, world, local, dist = dist_setup()
    A = workload(args.workload)
    B = A
    flop = row_products(A, B)
    products = int(flop.sum())

    if args.impl == "reference":
        rc = run_reference(args, A, B, flop, rank)
        if dist:
            dist.barrier()
        return rc

    do_var = args.variants == "all" and world == 1
    need_model = args.path == "learned" or do_var
    train_mats, gen_train_s = None, 0.0
    if need_model and not args.load_model:
        # CPU work first: the spawn pool starts before the first CUDA call
        from paper_2105_14156_gb300 import learned
        t0 = time.perf_counter()
        train_mats = learned.training_matrices(TRAIN_SEEDS, workers=min(16, os.cpu_count() or 1))
        gen_train_s = time.perf_counter() - t0

    import torch
    from paper_2105_14156_gb300 import autotune, build, learned, smash

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    h = smash.Handle(local)
    h.use_torch_allocator()
    dA = smash.to_device(A, dev)
    dB = smash.to_device(B, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    model, training = None, None
    if need_model and args.load_model:
        model = smash.Model(h)
        model.load(args.load_model)
        training = {"loaded": args.load_model}
    elif need_model:
        model, loss, train_s, nsamp = learned.train(h, train_mats, epochs=8, batch=4096)
        training = {"matrices": len(train_mats), "samples": nsamp, "final_mse": loss, "device_train_s": train_s,
                    "cpu_generation_s": gen_train_s, "epochs": 8, "batch": 4096}
        del train_mats
    if model is not None and args.save_model:
        model.save(args.save_model)
    tuned = None
    margin = 0.15
    if args.params:
        h.set_params(**json.loads(args.params))
        tuned = dict(json.loads(args.params), given=True)
        args.no_autotune = True
    if not args.no_autotune:
        tuned, _ = autotune.tune(h, dA, dB, args.workload, cache_path=None)
        if args.path == "learned":
            margin = tune_margin(h, dA, dB, model, stream, flush)
            tuned = dict(tuned, margin=margin)

    stats = {}
    step = step_fn(h, args.path, dA, dB, model, stream, stats, margin)
    for _ in range(args.warmup):
        C = step()
        del C
    h.check(stream)
    vb = A.val.dtype.itemsize

    sampler = ClockSampler(local)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    h.set_timing(True)
    t_wall0 = time.time()
    times = timed(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    kt = h.timings()
    h.set_timing(False)
    if dist:
        dist.barrier()
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)
    h.check(stream)
    if args.path == "plain":
        c_nnz = h.stats().c_nnz
    else:
        c_nnz = stats["c_nnz"]

    ms = replica_max(sum(times) / len(times), dist, dev)

    # dominant kernel: the launch group that moves the most algorithmic bytes,
    # roofline from its live per-launch event timing. The bins of a phase run
    # side by side on four streams, most products first, so this group starts
    # on an idle GPU and its event window is its own duration (the windows of
    # groups launched after it also count the time spent waiting for SMs).
    peaks, peak_src = load_peaks()
    launches = int(sum(t["kernels"] for t in kt))
    dom = max((t for t in kt if kernel_bytes(t, vb, B.nnz, products) is not None),
              key=lambda t: kernel_bytes(t, vb, B.nnz, products))
    per_launch_ms = dom["ms"] / dom["launches"]
    per_launch_bytes = kernel_bytes(dom, vb, B.nnz, products) / dom["launches"]
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
    traffic = recorded_traffic(dom["name"] + "_b%d" % dom["bin"], args.workload)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": "%s (bin %d)" % (dom["name"], dom["bin"]),
                "share_of_step": dom["ms"] / args.steps / ms,
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src}
    apeak = smem_atomic_peak(vb)
    if apeak:
        arate = dom["products"] / (dom["ms"] / 1e3) / 1e9
        roofline["smem_atomic"] = {"achieved": arate, "peak": apeak, "unit": "Gop/s", "frac": arate / apeak,
                                   "peak_source": "measured (profiles/smem_atomics_gb300.md, random slots)"}

    # end to end through the public API with host buffers: one call on the
    # whole of A, and the same product cut into row blocks of A whose results
    # go back to the host while the next block computes
    single = end_to_end(h, args, A, B, flop, model, margin, stream, dev, blocks=1)
    piped = end_to_end(h, args, A, B, flop, model, margin, stream, dev, blocks=max(1, args.e2e_blocks))
    # the blocked product equals the single call's: structure exactly, values up to
    # the order of the atomic adds
    (rp1, ci1, v1), (rp2, ci2, v2) = single["c"], piped["c"]
    assert torch.equal(rp1, rp2) and torch.equal(ci1, ci2), "row-blocked product differs from the single call"
    assert torch.allclose(v1.double(), v2.double(), rtol=1e-5, atol=1e-6), "row-blocked values differ"
    del single["c"], piped["c"]
    e2e_s = replica_max(piped["seconds"], dist, dev)
    e2e_single_s = replica_max(single["seconds"], dist, dev)
    h2d, d2h = piped["h2d"], piped["d2h"]

    step_bytes = metrics.spgemm_bytes(A.rows, A.nnz, B.rows, B.nnz, A.rows, c_nnz, vb)
    achieved_step = step_bytes / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": replica_gflops(world, products, ms / 1e3), "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if vb == 8 else "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "path": PATHS[args.path],
                   "products": products, "nnz_a": A.nnz, "nnz_c": c_nnz,
                   "l2": "flushed between timed steps (256 MiB write outside the timed region)",
                   "parallelism": "replicas" if world > 1 else "single", "autotuned": tuned},
        "hbm_gbs_per_gpu": achieved_step,
        "step_roofline": {"bound": "hbm", "achieved": achieved_step, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                          "frac": achieved_step / peaks["hbm_gbs"], "per_gpu": True,
                          "note": "bytes(A)+bytes(B)+bytes(C) per step over the step time, one GPU"},
        "roofline": roofline,
        "kernels": [{k: t[k] for k in ("name", "bin", "launches", "rows", "products", "ms")} for t in
                    sorted(kt, key=lambda t: -t["ms"])[:10]],
        "e2e": {"value": replica_gflops(world, products, e2e_s), "unit": "GFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "method": "%d row blocks of A, one public call each; each block's C is copied to pinned host "
                          "memory while the next block computes" % piped["blocks"],
                "single_call": {"value": replica_gflops(world, products, e2e_single_s), "unit": "GFLOP/s",
                                "h2d_bytes_per_step": single["h2d"], "d2h_bytes_per_step": single["d2h"]}},
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if args.path != "plain":
        line["learned_stats"] = {k: stats.get(k) for k in ("rows", "overflow_rows", "staged_nnz", "c_nnz")}
    if training:
        line["training"] = training

    if do_var:
        line["variants"] = run_variants(h, dev, flush, stream, args, model, peaks, dA, dB, products, ms, margin)

    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(A, B, flop, args.cpu_products)
    if model is not None:
        model.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_variants(h, dev, flush, stream, args, model, peaks, dA, dB, products, main_ms, margin):
    import torch
    from paper_2105_14156_gb300 import autotune, metrics, smash
    from paper_2105_14156_gb300.rmat import batched_workload, block_diagonal, paper_like_pair, workload
    K = max(10, args.variant_steps)
    out = {}

    def gf(prods, ms_):
        return metrics.useful_gflops(prods, ms_ / 1e3)

    def median_ms(fn, steps=K):
        fn()
        return statistics.median(timed(fn, steps, flush, stream))

    # the other paths on the main workload, same tuned parameters
    vb = dA.val.element_size()
    for path in ("plain", "bound", "learned"):
        if path == args.path:
            continue
        st = {}
        t = median_ms(step_fn(h, path, dA, dB, model, stream, st, margin))
        out["main_" + path] = {"ms": t, "gflops": gf(products, t), "main_over_this": t / main_ms,
                               "overflow_rows": st.get("overflow_rows"), "staged_nnz": st.get("staged_nnz")}

    # R-MAT scale 18, float32: learned / bound / plain (default parameters)
    saved = h.params.as_dict()
    h.set_params(**smash.default_params().as_dict())
    A18 = workload("rmat18_f32")
    p18 = int(row_products(A18, A18).sum())
    d18a, d18b = smash.to_device(A18, dev), smash.to_device(A18, dev)
    res18 = {}
    for path in ("plain", "bound", "learned"):
        st = {}
        t = median_ms(step_fn(h, path, d18a, d18b, model, stream, st))
        res18[path] = {"ms": t, "gflops": gf(p18, t), "overflow_rows": st.get("overflow_rows"),
                       "staged_over_cnnz": (st["staged_nnz"] / st["c_nnz"]) if st.get("c_nnz") else None}
    res18["products"] = p18
    res18["learned_over_plain"] = res18["plain"]["ms"] / res18["learned"]["ms"]
    res18["learned_over_bound"] = res18["bound"]["ms"] / res18["learned"]["ms"]
    out["rmat18_f32"] = res18
    del d18a, d18b, A18
    torch.cuda.empty_cache()

    # batched: 512 products in one persistent launch; 512 separate plain calls;
    # one plain call on the block-diagonal concatenation (the same products,
    # no per-call host round trips)
    pairs = batched_workload(512, seed=7)
    dev_pairs = [(smash.to_device(a, dev), smash.to_device(b, dev)) for a, b in pairs]
    pb = int(sum(row_products(a, b).sum() for a, b in pairs))
    binp = smash.BatchedInputs(dev_pairs)
    bits, _ = h.batched_autotune(binp, stream)
    cut = h.batched_row_cutoffs()
    bstats = {}

    def bstep():
        Cs, st, owner = h.spgemm_batched(binp, stream)
        bstats.update(st)
        owner.free()

    t_batch = median_ms(bstep)

    def sstep():
        for a, b in dev_pairs:
            h.spgemm(a, b, stream)

    t_sep = median_ms(sstep, max(3, K // 3))
    Abd, Bbd = block_diagonal(pairs)
    dAbd, dBbd = smash.to_device(Abd, dev), smash.to_device(Bbd, dev)
    t_bd = median_ms(lambda: h.spgemm(dAbd, dBbd, stream))
    out["batched_512"] = {"products_flop": pb, "c_nnz": bstats.get("c_nnz"), "batched_ms": t_batch,
                          "separate_ms": t_sep, "block_diagonal_ms": t_bd,
                          "batched_gflops": gf(pb, t_batch), "separate_gflops": gf(pb, t_sep),
                          "block_diagonal_gflops": gf(pb, t_bd),
                          "speedup_vs_separate": t_sep / t_batch, "speedup_vs_block_diagonal": t_bd / t_batch,
                          "table_bits": bits, "row_cutoffs": {"warp_less": cut[0], "block_more": cut[1]},
                          "big_rows": bstats.get("big_rows"), "huge_rows": bstats.get("huge_rows")}
    del dev_pairs, pairs, binp, dAbd, dBbd
    torch.cuda.empty_cache()

    # R-MAT scale 16, float64, plain two-pass (default parameters)
    A16 = workload("rmat16_f64")
    p16 = int(row_products(A16, A16).sum())
    d16a, d16b = smash.to_device(A16, dev), smash.to_device(A16, dev)
    t16 = median_ms(lambda: h.spgemm(d16a, d16b, stream))
    c16 = h.stats().c_nnz
    b16 = metrics.spgemm_bytes(A16.rows, A16.nnz, A16.rows, A16.nnz, A16.rows, c16, 8)
    out["rmat16_f64"] = {"products": p16, "c_nnz": c16, "plain_ms": t16, "plain_gflops": gf(p16, t16),
                         "hbm_roofline_frac": b16 / (t16 / 1e3) / 1e9 / peaks["hbm_gbs"]}
    del d16a, d16b, A16

    # the paper-like product: two independent R-MAT scale-14 matrices, float64
    Ap, Bp = paper_like_pair()
    pp = int(row_products(Ap, Bp).sum())
    dap, dbp = smash.to_device(Ap, dev), smash.to_device(Bp, dev)
    tp = median_ms(lambda: h.spgemm(dap, dbp, stream))
    cp_ = h.stats().c_nnz
    out["paper_like_ab_f64"] = {
        "workload": "two independent R-MAT scale 14, edge factor 16, (.45,.15,.15,.25), float64, C = A*B, plain",
        "nnz_a": Ap.nnz, "nnz_b": Bp.nnz, "products": pp, "c_nnz": cp_, "cf": pp / cp_ if cp_ else None,
        "plain_ms": tp, "plain_gflops": gf(pp, tp),
        "paper_context": "105.4 ms for the paper's 16K x 16K R-MAT pair (Version 3, simulated PIUMA block; "
                         "other hardware and matrices: context only)"}
    h.set_params(**saved)
    return out


if __name__ == "__main__":
    sys.exit(main())
