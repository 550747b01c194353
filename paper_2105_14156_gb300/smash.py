"""Python binding of the SMASH SpGEMM C ABI (include/smash.h).

Argument marshalling only: torch tensors provide device memory and streams,
every step of the computation runs in the CUDA library. There is no CPU
fallback: if the compiled library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsmash.so")

OK = 0
STATUS = {0: "SMASH_OK", 1: "SMASH_ERR_INVALID_ARG", 2: "SMASH_ERR_SHAPE_MISMATCH", 3: "SMASH_ERR_UNSUPPORTED",
          4: "SMASH_ERR_ALLOC", 5: "SMASH_ERR_CUDA", 6: "SMASH_ERR_TIMEOUT", 7: "SMASH_ERR_INTERNAL"}
F32, F64 = 0, 1

# Every symbol declared in include/smash.h (checked by the tests).
EXPORTS = [
    "smash_default_params", "smash_create", "smash_destroy", "smash_set_params", "smash_get_params",
    "smash_set_allocator", "spgemm_symbolic", "spgemm_numeric", "smash_check", "smash_get_stats",
    "smash_status_string", "smash_set_timing", "smash_get_timings",
]


class SmashError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__("%s: %s" % (where, STATUS.get(status, "status %d" % status)))
        self.status = status


class CsrStruct(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("hash_kind", ctypes.c_int32), ("max_load", ctypes.c_float), ("sym_max_tbits", ctypes.c_int32),
                ("num_max_tbits", ctypes.c_int32), ("group_shift", ctypes.c_int32),
                ("dense_ratio", ctypes.c_int32), ("bitmap_ratio", ctypes.c_int32),
                ("spill_blocks_per_sm", ctypes.c_int32), ("sym_dense_ratio", ctypes.c_int32),
                ("cluster_max", ctypes.c_int32), ("hot_cols", ctypes.c_int32), ("hot_factor", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Stats(ctypes.Structure):
    _fields_ = [("rows_per_bin", ctypes.c_int64 * 16), ("products", ctypes.c_int64),
                ("max_row_products", ctypes.c_int64), ("c_nnz", ctypes.c_int64),
                ("a_nnz_per_bin", ctypes.c_int64 * 16), ("products_per_bin", ctypes.c_int64 * 16),
                ("c_nnz_per_bin", ctypes.c_int64 * 16)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("bin", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("launches", ctypes.c_int64), ("rows", ctypes.c_int64), ("a_nnz", ctypes.c_int64),
                ("products", ctypes.c_int64), ("c_nnz", ctypes.c_int64), ("ms", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["name"] = self.name.decode()
        return d


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsmash.so (built by paper_2105_14156_gb300.build). Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libsmash.so not built (%s): run paper_2105_14156_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.smash_default_params.argtypes = [ctypes.POINTER(Params)]
        lib.smash_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(Params)]
        lib.smash_destroy.argtypes = [P]
        lib.smash_set_params.argtypes = [P, ctypes.POINTER(Params)]
        lib.smash_get_params.argtypes = [P, ctypes.POINTER(Params)]
        lib.smash_set_allocator.argtypes = [P, P, P, P]
        lib.spgemm_symbolic.argtypes = [P, ctypes.POINTER(CsrStruct), ctypes.POINTER(CsrStruct), P,
                                        ctypes.POINTER(ctypes.c_int64), P]
        lib.spgemm_numeric.argtypes = [P, ctypes.POINTER(CsrStruct), ctypes.POINTER(CsrStruct), ctypes.c_int,
                                       ctypes.POINTER(CsrStruct), P]
        lib.smash_check.argtypes = [P, P]
        lib.smash_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
        lib.smash_set_timing.argtypes = [P, ctypes.c_int]
        lib.smash_get_timings.argtypes = [P, ctypes.POINTER(KernelTime), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]
        lib.smash_status_string.argtypes = [ctypes.c_int]
        lib.smash_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            f = getattr(lib, name)
            if f.restype is None or f.restype is ctypes.c_int:
                if name != "smash_status_string":
                    f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != OK:
        raise SmashError(status, where)


def default_params() -> Params:
    p = Params()
    _check(load_library().smash_default_params(ctypes.byref(p)), "smash_default_params")
    return p


@dataclasses.dataclass
class DeviceCsr:
    """CSR matrix in device memory: torch tensors int64 row_ptr, int32 col_idx, val."""
    rows: int
    cols: int
    row_ptr: "object"
    col_idx: "object"
    val: "object"

    @property
    def nnz(self) -> int:
        return int(self.col_idx.numel())

    def struct(self) -> CsrStruct:
        return CsrStruct(self.rows, self.cols, self.nnz, self.row_ptr.data_ptr(),
                         self.col_idx.data_ptr() if self.col_idx.numel() else None,
                         self.val.data_ptr() if self.val is not None and self.val.numel() else None)

    def to_host(self):
        from .rmat import Csr
        return Csr(self.rows, self.cols, self.row_ptr.cpu().numpy(), self.col_idx.cpu().numpy(),
                   self.val.cpu().numpy() if self.val is not None else None)

    def nbytes(self) -> int:
        vb = self.val.element_size() if self.val is not None else 0
        return 8 * (self.rows + 1) + (4 + vb) * self.nnz


def to_device(M, device="cuda", dtype=None, non_blocking=False) -> DeviceCsr:
    """Copy a host Csr (rmat.Csr) to the device."""
    import torch
    val = np.ascontiguousarray(M.val if dtype is None else M.val.astype(dtype))
    return DeviceCsr(M.rows, M.cols,
                     torch.from_numpy(np.ascontiguousarray(M.row_ptr, dtype=np.int64)).to(device, non_blocking=non_blocking),
                     torch.from_numpy(np.ascontiguousarray(M.col_idx, dtype=np.int32)).to(device, non_blocking=non_blocking),
                     torch.from_numpy(val).to(device, non_blocking=non_blocking))


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError("values must be float32 or float64, got %s" % t.dtype)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Handle:
    """A library handle bound to one CUDA device."""

    def __init__(self, device: int = 0, params: Params | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the SMASH library has no CPU path")
        self.lib = load_library()
        self.device = device
        h = ctypes.c_void_p()
        _check(self.lib.smash_create(ctypes.byref(h), device, ctypes.byref(params) if params else None),
               "smash_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.smash_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # parameters and statistics
    @property
    def params(self) -> Params:
        p = Params()
        _check(self.lib.smash_get_params(self.h, ctypes.byref(p)), "smash_get_params")
        return p

    @params.setter
    def params(self, p: Params):
        _check(self.lib.smash_set_params(self.h, ctypes.byref(p)), "smash_set_params")

    def set_params(self, **kw):
        p = self.params
        for k, v in kw.items():
            setattr(p, k, v)
        self.params = p

    def stats(self) -> Stats:
        s = Stats()
        _check(self.lib.smash_get_stats(self.h, ctypes.byref(s)), "smash_get_stats")
        return s

    def set_timing(self, enable: bool):
        _check(self.lib.smash_set_timing(self.h, 1 if enable else 0), "smash_set_timing")

    def timings(self):
        """Per-(kernel, bin) event-timed totals since timing was enabled."""
        n = ctypes.c_int(0)
        _check(self.lib.smash_get_timings(self.h, None, 0, ctypes.byref(n)), "smash_get_timings")
        arr = (KernelTime * max(n.value, 1))()
        _check(self.lib.smash_get_timings(self.h, arr, n.value, ctypes.byref(n)), "smash_get_timings")
        return [arr[k].as_dict() for k in range(n.value)]

    def check(self, stream=None):
        _check(self.lib.smash_check(self.h, _stream_ptr(stream)), "smash_check")

    # the two phases
    def symbolic(self, A: DeviceCsr, B: DeviceCsr, stream=None):
        """C's row pointer (device int64[A.rows+1]) and nnz(C)."""
        import torch
        c_rp = torch.empty(A.rows + 1, dtype=torch.int64, device=A.row_ptr.device)
        nnz = ctypes.c_int64(0)
        sa, sb = A.struct(), B.struct()
        _check(self.lib.spgemm_symbolic(self.h, ctypes.byref(sa), ctypes.byref(sb), c_rp.data_ptr(),
                                        ctypes.byref(nnz), _stream_ptr(stream)), "spgemm_symbolic")
        return c_rp, int(nnz.value)

    def numeric(self, A: DeviceCsr, B: DeviceCsr, c_rp, c_nnz: int, stream=None, out: DeviceCsr | None = None):
        """Fill C's columns and values (device), given the symbolic row pointer."""
        import torch
        dt = _dtype_code(A.val)
        if B.val.dtype != A.val.dtype:
            raise TypeError("A and B values must have the same dtype")
        if out is None:
            out = DeviceCsr(A.rows, B.cols, c_rp,
                            torch.empty(c_nnz, dtype=torch.int32, device=A.row_ptr.device),
                            torch.empty(c_nnz, dtype=A.val.dtype, device=A.row_ptr.device))
        sa, sb, sc = A.struct(), B.struct(), out.struct()
        _check(self.lib.spgemm_numeric(self.h, ctypes.byref(sa), ctypes.byref(sb), dt, ctypes.byref(sc),
                                       _stream_ptr(stream)), "spgemm_numeric")
        return out

    def spgemm(self, A: DeviceCsr, B: DeviceCsr, stream=None, check: bool = False) -> DeviceCsr:
        """C = A*B: symbolic phase, allocation of C, numeric phase."""
        c_rp, c_nnz = self.symbolic(A, B, stream)
        C = self.numeric(A, B, c_rp, c_nnz, stream)
        if check:
            self.check(stream)
        return C
