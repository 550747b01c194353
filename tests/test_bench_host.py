"""Host-side measurement plumbing of bench.py on the CPU: the useful-flop count
behind every GFLOP/s figure, the CPU baseline's row sample, the gate that keeps
an ncu DRAM figure only while the kernel sources it was taken on are unchanged,
and the readers of the measured peaks."""
import os

import numpy as np

import oracle
from tests.helpers import random_csr


def test_row_products_match_the_oracle_flop_count():
    import bench
    A = random_csr(700, 300, 0.03, 501, values="f32")
    B = random_csr(300, 900, 0.02, 502, values="f32")
    A.row_ptr[100:200] = A.row_ptr[100]          # rows 100-198 empty, row 199 takes their entries
    got = bench.row_products(A, B)
    assert got.dtype == np.int64
    assert np.array_equal(got, oracle.row_flops(A, B))
    assert np.all(got[100:199] == 0)


class _Rows:
    rows = 1000


def test_cpu_sample_reaches_its_budget_and_is_seeded():
    import bench
    flop = np.arange(1, 1001, dtype=np.int64)
    rows = bench.sample_rows(_Rows(), flop, 5000.0, seed=3)
    again = bench.sample_rows(_Rows(), flop, 5000.0, seed=3)
    assert np.array_equal(rows, again)
    assert np.all(np.diff(rows) > 0)             # sorted, no repeats
    assert flop[rows].sum() >= 5000              # the budget is reached, and without the last
    assert flop[rows].sum() - flop[rows].max() < 5000   # row drawn (at most the largest) it is not
    other = bench.sample_rows(_Rows(), flop, 5000.0, seed=4)
    assert not np.array_equal(rows, other)
    everything = bench.sample_rows(_Rows(), flop, 1e12, seed=3)
    assert np.array_equal(everything, np.arange(1000))


def _fake_tree(root, text):
    csrc = os.path.join(root, "paper_2105_14156_gb300", "csrc")
    os.makedirs(csrc, exist_ok=True)
    with open(os.path.join(csrc, "k.cu"), "w") as f:
        f.write(text)
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)


def test_recorded_traffic_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    import bench
    root = str(tmp_path)
    _fake_tree(root, "kernel v1")
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.recorded_traffic("num_hash_b6", "rmat20_f32") is None   # no summary at all
    src = bench.source_hash()
    with open(os.path.join(root, "profiles", "dram_traffic.txt"), "w") as f:
        f.write("# comment line\n")
        f.write("kernel=num_hash_b6 workload=rmat20_f32 src=%s dram_bytes_per_launch=123456\n" % src)
        f.write("kernel=num_warp_b4 workload=rmat20_f32 src=%s dram_bytes_per_launch=999\n" % src)
    assert bench.recorded_traffic("num_hash_b6", "rmat20_f32") == 123456.0
    assert bench.recorded_traffic("num_hash_b6", "rmat18_f32") is None   # other workload
    assert bench.recorded_traffic("num_hash_b7", "rmat20_f32") is None   # other kernel
    _fake_tree(root, "kernel v2")                                         # sources changed
    assert bench.source_hash() != src
    assert bench.recorded_traffic("num_hash_b6", "rmat20_f32") is None


def test_committed_traffic_record_is_well_formed():
    import bench
    path = os.path.join(bench.ROOT, "profiles", "dram_traffic.txt")
    recs = [dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            for line in open(path) if not line.startswith("#") and line.strip()]
    assert recs
    for r in recs:
        assert set(r) == {"kernel", "workload", "src", "dram_bytes_per_launch"}
        assert len(r["src"]) == 16
        assert float(r["dram_bytes_per_launch"]) > 0


def test_peak_readers(tmp_path, monkeypatch):
    import bench
    peaks, src = bench.load_peaks()
    assert peaks["hbm_gbs"] > 0
    assert src in ("measured", "fallback")
    assert bench.smem_atomic_peak(4) > 0 and bench.smem_atomic_peak(8) > 0
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == ({"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback")
    assert bench.smem_atomic_peak(4) is None
