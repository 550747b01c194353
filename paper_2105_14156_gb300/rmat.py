"""Seeded synthetic inputs: R-MAT sparse matrices and batched feature matrices.

This module only draws inputs. It holds none of the SpGEMM arithmetic, and both
the CUDA path's tests and the CPU oracle's tests take their matrices from here.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
draw of a stream is the SplitMix64 finaliser applied to ``key + (i+1)*GAMMA``.
Every draw is therefore addressable by (stream key, counter), independent of
the order in which arrays are built.

R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004) is the workload the paper
evaluates on (Results chapter, "Experimental Methodology"): every edge descends
``scale`` levels of the adjacency matrix and at each level picks one quadrant
with probabilities (a, b, c, d), one uniform draw per level. No noise is added,
edges are directed, self-loops are kept and duplicate edges are merged into one
nonzero. Values are drawn per unique nonzero, in CSR order, from a second stream.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)
_S11 = np.uint64(11)

GRAPH500_ABCD = (0.57, 0.19, 0.19, 0.05)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = (z ^ (z >> _S30)) * _M1
    z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of an independent stream derived from (seed, stream id)."""
    with np.errstate(over="ignore"):
        z = np.array([(seed * 0x2545F4914F6CDD1D + stream * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019)
                      & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix(z)[0]


def bits64(key: np.uint64, ctr: np.ndarray) -> np.ndarray:
    """The ctr-th 64-bit draw of stream ``key`` (ctr: uint64-compatible array)."""
    c = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + (c + np.uint64(1)) * GAMMA)


def uniform(key: np.uint64, ctr: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (bits64(key, ctr) >> _S11).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Csr:
    """Host CSR matrix: int64 row_ptr[rows+1], int32 col_idx[nnz], values[nnz]."""
    rows: int
    cols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.rows > 0 else 0

    def astype(self, dtype) -> "Csr":
        return Csr(self.rows, self.cols, self.row_ptr, self.col_idx, self.val.astype(dtype))


def csr_from_coo(rows: int, cols: int, r: np.ndarray, c: np.ndarray, merge: bool = True) -> tuple:
    """Sort (r, c) pairs row-major, optionally merge duplicates; return (row_ptr, col_idx)."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    key = r * np.int64(max(cols, 1)) + c
    key = np.unique(key) if merge else np.sort(key)
    rr = key // max(cols, 1)
    cc = (key % max(cols, 1)).astype(np.int32)
    row_ptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(np.bincount(rr, minlength=rows), out=row_ptr[1:])
    return row_ptr, cc


def _rmat_edges(key: np.uint64, scale: int, abcd, first: int, count: int):
    """Row/col of R-MAT edges first..first+count-1 (one uniform per level)."""
    a, b, c, _ = abcd
    t_ab, t_abc = a + b, a + b + c
    e = np.arange(first, first + count, dtype=np.uint64)
    row = np.zeros(count, dtype=np.int64)
    col = np.zeros(count, dtype=np.int64)
    s = np.uint64(scale)
    for lvl in range(scale):
        u = uniform(key, e * s + np.uint64(lvl))
        bit = np.int64(1) << np.int64(scale - 1 - lvl)
        down = u >= t_ab                      # quadrants c and d: lower half
        right = ((u >= a) & (u < t_ab)) | (u >= t_abc)   # quadrants b and d
        row += np.where(down, bit, 0)
        col += np.where(right, bit, 0)
    return row, col


def draw_values(key: np.uint64, nnz: int, kind: str) -> np.ndarray:
    """Values for nnz nonzeros in CSR order.

    kind: "f64" / "f32" uniform in [-1, 1); "int4" uniform integers {1..4} stored
    as float32 (exactly representable)."""
    u = uniform(key, np.arange(nnz, dtype=np.uint64))
    if kind == "f64":
        return 2.0 * u - 1.0
    if kind == "f32":
        return (2.0 * u - 1.0).astype(np.float32)
    if kind == "int4":
        return (1.0 + np.floor(4.0 * u)).astype(np.float32)
    raise ValueError(kind)


def rmat(scale: int, edge_factor: int, abcd=GRAPH500_ABCD, seed: int = 1, values: str = "f64") -> Csr:
    """Square 2^scale R-MAT matrix with edge_factor * 2^scale drawn edges, merged."""
    n = 1 << scale
    m = edge_factor * n
    kE = stream_key(seed, 1)
    kV = stream_key(seed, 2)
    r, c = _rmat_edges(kE, scale, abcd, 0, m)
    row_ptr, col_idx = csr_from_coo(n, n, r, c)
    val = draw_values(kV, int(row_ptr[-1]), values)
    return Csr(n, n, row_ptr, col_idx, val)


def batched_pair(seed: int, index: int, n_lo: int = 64, n_hi: int = 8192, deg_lo: float = 4.0,
                 deg_hi: float = 32.0, b_cols: int = 256, b_density: float = 0.05,
                 abcd=GRAPH500_ABCD):
    """One (A_i, B_i) pair of the batched workload.

    n_i = round(exp(U[ln n_lo, ln n_hi])), average degree U[deg_lo, deg_hi];
    A_i: R-MAT at scale ceil(log2 n_i), edges with an endpoint >= n_i redrawn
    until round(deg*n_i) edges are kept, then duplicates merged.
    B_i: n_i x b_cols with round(b_density * n_i * b_cols) distinct uniform
    positions. Values uniform in [-1, 1) (float32)."""
    kP = stream_key(seed, 1000 + 4 * index)
    kA = stream_key(seed, 1001 + 4 * index)
    kB = stream_key(seed, 1002 + 4 * index)
    kV = stream_key(seed, 1003 + 4 * index)
    u = uniform(kP, np.arange(2, dtype=np.uint64))
    n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
    deg = deg_lo + u[1] * (deg_hi - deg_lo)
    m = int(round(deg * n))
    scale = max(1, int(math.ceil(math.log2(n))))
    rows, cols = [], []
    kept, first = 0, 0
    while kept < m:
        want = max(1024, 2 * (m - kept))
        r, c = _rmat_edges(kA, scale, abcd, first, want)
        first += want
        ok = (r < n) & (c < n)
        r, c = r[ok], c[ok]
        take = min(m - kept, r.size)
        rows.append(r[:take])
        cols.append(c[:take])
        kept += take
    a_rp, a_ci = csr_from_coo(n, n, np.concatenate(rows), np.concatenate(cols))
    target = int(round(b_density * n * b_cols))
    total = n * b_cols
    chosen = np.empty(0, dtype=np.int64)
    ctr = 0
    while chosen.size < target:
        want = 2 * (target - chosen.size) + 64
        p = np.floor(uniform(kB, np.arange(ctr, ctr + want, dtype=np.uint64)) * total).astype(np.int64)
        ctr += want
        allp = np.concatenate([chosen, p])
        _, first_idx = np.unique(allp, return_index=True)
        chosen = allp[np.sort(first_idx)]
    chosen = chosen[:target]
    b_rp, b_ci = csr_from_coo(n, b_cols, chosen // b_cols, chosen % b_cols)
    va = draw_values(kV, int(a_rp[-1]) + int(b_rp[-1]), "f32")
    A = Csr(n, n, a_rp, a_ci, va[: int(a_rp[-1])].copy())
    B = Csr(n, b_cols, b_rp, b_ci, va[int(a_rp[-1]):].copy())
    return A, B


def batched_workload(count: int = 512, seed: int = 7, **kw):
    """The batched workload: ``count`` independent pairs (A_i, B_i)."""
    return [batched_pair(seed, i, **kw) for i in range(count)]


def block_diagonal(pairs):
    """(diag(A_1, ..., A_m), diag(B_1, ..., B_m)): the products of a batch laid
    out as one product whose rows and columns are the batch's, block by block."""
    def diag(mats):
        rows = sum(M.rows for M in mats)
        cols = sum(M.cols for M in mats)
        rp = np.zeros(rows + 1, dtype=np.int64)
        ci, val = [], []
        r0 = c0 = e0 = 0
        for M in mats:
            rp[r0 + 1:r0 + M.rows + 1] = M.row_ptr[1:] + e0
            ci.append(M.col_idx.astype(np.int64) + c0)
            val.append(M.val)
            r0 += M.rows
            c0 += M.cols
            e0 += M.nnz
        return Csr(rows, cols, rp, np.concatenate(ci).astype(np.int32), np.concatenate(val))
    return diag([a for a, _ in pairs]), diag([b for _, b in pairs])


def paper_like_pair():
    """Two independently drawn R-MAT matrices of scale 14 (16K x 16K), edge
    factor 16, (a,b,c,d) = (.45,.15,.15,.25), float64 values: the closest seeded
    stand-in for the pair of 16K x 16K R-MAT matrices multiplied in the paper's
    evaluation (whose R-MAT parameters are not given)."""
    abcd = (0.45, 0.15, 0.15, 0.25)
    return rmat(14, 16, abcd, seed=1, values="f64"), rmat(14, 16, abcd, seed=2, values="f64")


def training_matrix(seed: int, edge_factor: int = 16) -> Csr:
    """Training set member ``seed``: R-MAT scale 12 + (seed mod 5), float32 U[-1,1]."""
    return rmat(12 + (seed % 5), edge_factor, GRAPH500_ABCD, seed=10_000 + seed, values="f32")


# Named workloads (sizes and value distributions of the evaluated configurations).
def workload(name: str):
    if name == "rmat10_int":
        return rmat(10, 8, GRAPH500_ABCD, seed=1, values="int4")
    if name == "rmat16_f64":
        return rmat(16, 16, GRAPH500_ABCD, seed=1, values="f64")
    if name == "rmat17_f32":
        return rmat(17, 16, GRAPH500_ABCD, seed=1, values="f32")
    if name == "rmat18_f32":
        return rmat(18, 16, GRAPH500_ABCD, seed=1, values="f32")
    if name == "rmat20_f32":
        return rmat(20, 8, (0.45, 0.15, 0.15, 0.25), seed=1, values="f32")
    if name == "rmat14_pair_f64":
        return paper_like_pair()
    raise KeyError(name)
