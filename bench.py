"""Benchmark: C = A*A on R-MAT through the SMASH C ABI on GB300.

One step = the whole plain two-pass path on one input: per-row product
counts and binning, the symbolic hash pass, the row-pointer scan, allocation
of C, the numeric hash pass with write-back (shared-memory tables, dense
rows, global-memory spill, per-row sort). Inputs are resident in HBM when the
timed region starts; L2 (129 MB) is flushed between timed steps by writing a
256 MiB buffer outside the timed region.

Prints one JSON line (rank 0). Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl smash|reference]
Multi-GPU (torchrun): every rank runs an independent replica of the workload
(the rows of C are independent; there is no exchange step), value = products
of all ranks / max time over ranks, "scaling": "weak".
"""
from __future__ import annotations

import argparse
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
    "rmat16_f64": "R-MAT scale 16 (65536 x 65536), edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
                  "float64 values U[-1,1], C = A*A (A and B separate copies), plain two-pass hash",
    "rmat10_int": "R-MAT scale 10, edge factor 8, (0.57,0.19,0.19,0.05), float32 integer values {1..4}, C = A*A",
    "rmat18_f32": "R-MAT scale 18, edge factor 16, (0.57,0.19,0.19,0.05), float32 U[-1,1], C = A*A",
    "rmat20_f32": "R-MAT scale 20, edge factor 8, (0.45,0.15,0.15,0.25), float32 U[-1,1], C = A*A",
}


def row_products(A, B) -> np.ndarray:
    """flop_i = sum over A_i of |B_k| (host bookkeeping for the metric)."""
    blen = np.diff(B.row_ptr)
    per = blen[A.col_idx].astype(np.int64)
    out = np.zeros(A.rows, dtype=np.int64)
    nz = np.diff(A.row_ptr) > 0
    out[nz] = np.add.reduceat(per, A.row_ptr[:-1][nz]) if per.size else 0
    return out


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


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
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
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


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("SMASH_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def cpu_baseline(A, B, flop, budget_products: float, seed: int = 0):
    """The oracle on a seeded random sample of rows (about budget_products products)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    order = rng.permutation(A.rows)
    cum = np.cumsum(flop[order])
    k = int(np.searchsorted(cum, budget_products)) + 1
    rows = np.sort(order[:min(k, A.rows)])
    t0 = time.perf_counter()
    oracle.spgemm(A, B, rows=rows)
    dt = time.perf_counter() - t0
    prods = int(flop[rows].sum())
    return {"value": 2.0 * prods / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": "%d of %d rows drawn at random (seed %d), %d of %d products, %.1f s single-threaded"
                      % (rows.size, A.rows, seed, prods, int(flop.sum()), dt)}


def run_reference(args, A, B, flop, rank, world):
    """Reference arm: the CPU oracle as it stands, on bounded samples of the workload."""
    if rank != 0:
        return 0
    vals = []
    per_step = float(os.environ.get("SMASH_REF_STEP_PRODUCTS", "2e7"))
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(A, B, flop, per_step, seed=k)
        if k >= args.warmup:
            vals.append(cb["value"])
    value = statistics.median(vals)
    t_step = 2.0 * per_step / (value * 1e9)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload]},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: rows drawn at random until about %.0e products" % per_step},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="smash", choices=["smash", "reference"])
    ap.add_argument("--workload", default="rmat16_f64", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-products", type=float, default=2e8)
    ap.add_argument("--e2e-steps", type=int, default=3)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.e2e_steps = max(args.e2e_steps, 1)

    from paper_2105_14156_gb300 import metrics
    from paper_2105_14156_gb300.rmat import workload

    rank, world, local, dist = dist_setup(args.gpus)
    A = workload(args.workload)
    B = A
    flop = row_products(A, B)
    products = int(flop.sum())

    if args.impl == "reference":
        rc = run_reference(args, A, B, flop, rank, world)
        if dist:
            dist.barrier()
        return rc

    import torch
    from paper_2105_14156_gb300 import build, smash

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    h = smash.Handle(local)
    dA = smash.to_device(A, dev)
    dB = smash.to_device(B, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        return h.spgemm(dA, dB, stream)

    for _ in range(args.warmup):
        C = step()
    h.check(stream)
    torch.cuda.synchronize()
    c_nnz = C.nnz
    vb = A.val.dtype.itemsize

    sampler = ClockSampler(local)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    times = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        C = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall1 = time.time()
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)
    h.check(stream)

    ms = sum(times) / len(times)
    if dist:
        t = torch.tensor([ms], dtype=torch.float64, device=dev if dist.get_backend() == "nccl" else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the public API with host buffers
    pinned = {}
    for name, M in (("A", A), ("B", B)):
        pinned[name] = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
                        for x in (M.row_ptr, M.col_idx, M.val)]
    e2e_times = []
    h2d = sum(t.numel() * t.element_size() for lst in pinned.values() for t in lst)
    d2h = 0
    out_host = None
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dAe = smash.DeviceCsr(A.rows, A.cols, *[t.to(dev, non_blocking=True) for t in pinned["A"]])
        dBe = smash.DeviceCsr(B.rows, B.cols, *[t.to(dev, non_blocking=True) for t in pinned["B"]])
        Ce = h.spgemm(dAe, dBe, stream)
        if out_host is None or out_host[1].numel() != Ce.nnz:
            out_host = [torch.empty(Ce.rows + 1, dtype=torch.int64).pin_memory(),
                        torch.empty(Ce.nnz, dtype=torch.int32).pin_memory(),
                        torch.empty(Ce.nnz, dtype=Ce.val.dtype).pin_memory()]
        out_host[0].copy_(Ce.row_ptr, non_blocking=True)
        out_host[1].copy_(Ce.col_idx, non_blocking=True)
        out_host[2].copy_(Ce.val, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        d2h = sum(t.numel() * t.element_size() for t in out_host)
        if k > 0:
            e2e_times.append(dt)
        del dAe, dBe, Ce
    e2e_s = statistics.median(e2e_times)
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev if dist.get_backend() == "nccl" else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    peaks, peak_src = load_peaks()
    step_bytes = metrics.spgemm_bytes(A.rows, A.nnz, B.rows, B.nnz, A.rows, c_nnz, vb)
    gflops = world * metrics.useful_gflops(products, ms / 1e3)
    achieved_gbs = step_bytes / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": gflops, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if vb == 8 else "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                   "products": products, "nnz_a": A.nnz, "nnz_c": c_nnz,
                   "l2": "flushed between timed steps (256 MiB write outside the timed region)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "hbm_gbs": achieved_gbs,
        "step_roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                          "frac": achieved_gbs / peaks["hbm_gbs"], "traffic": None,
                          "note": "bytes(A)+bytes(B)+bytes(C) per step over the step time; peak %s" % peak_src},
        "e2e": {"value": world * metrics.useful_gflops(products, e2e_s), "unit": "GFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
        "gpu_launches": None,
    }
    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(A, B, flop, args.cpu_products)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
