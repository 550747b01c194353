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
    "smash_train_cfg_default", "smash_model_create", "smash_model_destroy", "smash_model_get", "smash_model_set",
    "smash_model_save", "smash_model_load", "smash_row_features", "smash_mlp_train", "smash_mlp_gradient",
    "smash_mlp_predict", "smash_mlp_predict_tc", "spgemm_learned", "smash_free_csr", "spgemm_symbolic_noalloc",
    "spgemm_batched", "smash_batched_set_table_bits", "smash_batched_get_table_bits", "smash_batched_autotune",
    "smash_training_rows", "smash_batched_set_wait", "smash_batched_set_row_cutoffs",
    "smash_batched_get_row_cutoffs",
]


class BatchedStats(ctypes.Structure):
    _fields_ = [("products", ctypes.c_int64), ("rows", ctypes.c_int64), ("big_rows", ctypes.c_int64),
                ("huge_rows", ctypes.c_int64), ("flop", ctypes.c_int64), ("c_nnz", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}
MLP_PARAMS = 4673


class TrainCfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("weight_decay", ctypes.c_float), ("seed", ctypes.c_uint64), ("reserved", ctypes.c_int32 * 4)]


class LearnedStats(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("overflow_rows", ctypes.c_int64), ("staged_nnz", ctypes.c_int64),
                ("c_nnz", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class _DeviceArray:
    """Zero-copy view of library-allocated device memory (CUDA array interface)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


def _view(ptr, n, dtype):
    import torch
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device="cuda")
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.float32: "<f4", torch.float64: "<f8"}[dtype]
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda")


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
                ("dense_blocks", ctypes.c_int32), ("sym_dense_blocks", ctypes.c_int32),
                ("warp_rows", ctypes.c_int32), ("bulk_copy", ctypes.c_int32), ("group_rows", ctypes.c_int32),
                ("row_window", ctypes.c_int32), ("row_window_tbits", ctypes.c_int32),
                ("dense_owner", ctypes.c_int32)]

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
                ("products", ctypes.c_int64), ("c_nnz", ctypes.c_int64), ("ms", ctypes.c_double),
                ("kernels", ctypes.c_int64)]

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
        lib.smash_train_cfg_default.argtypes = [ctypes.POINTER(TrainCfg)]
        lib.smash_model_create.argtypes = [P, ctypes.POINTER(P), ctypes.c_uint64]
        lib.smash_model_destroy.argtypes = [P]
        lib.smash_model_get.argtypes = [P, P, P]
        lib.smash_model_set.argtypes = [P, P, P]
        lib.smash_model_save.argtypes = [P, ctypes.c_char_p]
        lib.smash_model_load.argtypes = [P, ctypes.c_char_p]
        lib.smash_row_features.argtypes = [P, ctypes.POINTER(CsrStruct), ctypes.POINTER(CsrStruct), P, P]
        lib.smash_training_rows.argtypes = [P, ctypes.POINTER(CsrStruct), ctypes.POINTER(CsrStruct), P, P,
                                            ctypes.POINTER(ctypes.c_int64), P]
        lib.smash_mlp_train.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.POINTER(TrainCfg),
                                        ctypes.POINTER(ctypes.c_float), P]
        lib.smash_mlp_gradient.argtypes = [P, P, P, P, ctypes.c_int64, P, ctypes.POINTER(ctypes.c_float), P]
        lib.smash_mlp_predict.argtypes = [P, P, P, ctypes.c_int64, P, P]
        lib.smash_mlp_predict_tc.argtypes = [P, P, P, ctypes.c_int64, P, P]
        lib.spgemm_learned.argtypes = [P, ctypes.POINTER(CsrStruct), ctypes.POINTER(CsrStruct), ctypes.c_int, P,
                                       ctypes.c_float, ctypes.POINTER(CsrStruct), ctypes.POINTER(LearnedStats), P]
        lib.smash_free_csr.argtypes = [P, ctypes.POINTER(CsrStruct)]
        lib.spgemm_symbolic_noalloc.argtypes = [ctypes.POINTER(CsrStruct), ctypes.POINTER(CsrStruct), P,
                                                ctypes.POINTER(ctypes.c_int64), P]
        lib.spgemm_batched.argtypes = [P, ctypes.c_int, ctypes.POINTER(CsrStruct), ctypes.POINTER(CsrStruct),
                                       ctypes.c_int, ctypes.POINTER(CsrStruct), ctypes.POINTER(BatchedStats), P]
        lib.smash_batched_set_table_bits.argtypes = [P, ctypes.c_int]
        lib.smash_batched_get_table_bits.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
        lib.smash_batched_set_wait.argtypes = [P, ctypes.c_int64, ctypes.c_int]
        lib.smash_batched_set_row_cutoffs.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.smash_batched_get_row_cutoffs.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        lib.smash_batched_autotune.argtypes = [P, ctypes.c_int, ctypes.POINTER(CsrStruct),
                                               ctypes.POINTER(CsrStruct), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_float), P]
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

    def use_torch_allocator(self):
        """Route the handle's device allocations (scratch, and the C arrays of the
        learned and batched calls) through torch's caching allocator."""
        import torch
        ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
        FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
        dev = self.device

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch.cuda.current_stream(dev))
            except Exception:
                return None

        def _free(ptr, ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC(_alloc)   # keep the callbacks alive
        self._free_cb = FREE(_free)
        _check(self.lib.smash_set_allocator(self.h, ctypes.cast(self._alloc_cb, ctypes.c_void_p),
                                            ctypes.cast(self._free_cb, ctypes.c_void_p), None),
               "smash_set_allocator")

    def set_allocator(self, alloc=None, free=None):
        """Route the handle's device allocations through Python callables:
        alloc(nbytes) -> device pointer (int, 0 on failure), free(ptr). None
        restores cudaMalloc / cudaFree."""
        ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
        FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
        if alloc is None:
            _check(self.lib.smash_set_allocator(self.h, None, None, None), "smash_set_allocator")
            self._alloc_cb = self._free_cb = None
            return
        self._alloc_cb = ALLOC(lambda nbytes, ctx: alloc(int(nbytes)) or None)
        self._free_cb = FREE(lambda ptr, ctx: free(ptr))
        _check(self.lib.smash_set_allocator(self.h, ctypes.cast(self._alloc_cb, ctypes.c_void_p),
                                            ctypes.cast(self._free_cb, ctypes.c_void_p), None),
               "smash_set_allocator")

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

    # learned sizing
    def features(self, A: DeviceCsr, B: DeviceCsr, stream=None):
        import torch
        f = torch.empty((A.rows, 6), dtype=torch.float32, device=A.row_ptr.device)
        sa, sb = A.struct(), B.struct()
        _check(self.lib.smash_row_features(self.h, ctypes.byref(sa), ctypes.byref(sb), f.data_ptr(),
                                           _stream_ptr(stream)), "smash_row_features")
        return f

    def training_rows(self, A: DeviceCsr, B: DeviceCsr, stream=None):
        """Training samples of C = A*B made by the library: (features [n, 6],
        targets log1p(nnz(C_i)) [n]) of the rows with at least one product."""
        import torch
        f = torch.empty((A.rows, 6), dtype=torch.float32, device=A.row_ptr.device)
        t = torch.empty(A.rows, dtype=torch.float32, device=A.row_ptr.device)
        n = ctypes.c_int64(0)
        sa, sb = A.struct(), B.struct()
        _check(self.lib.smash_training_rows(self.h, ctypes.byref(sa), ctypes.byref(sb), f.data_ptr(), t.data_ptr(),
                                            ctypes.byref(n), _stream_ptr(stream)), "smash_training_rows")
        return f[: n.value], t[: n.value]

    def mlp_train(self, model: "Model", feats, targets, stream=None, **cfg) -> float:
        c = TrainCfg()
        _check(self.lib.smash_train_cfg_default(ctypes.byref(c)), "smash_train_cfg_default")
        for k, v in cfg.items():
            setattr(c, k, v)
        loss = ctypes.c_float(0)
        feats = feats.contiguous()
        targets = targets.contiguous()
        _check(self.lib.smash_mlp_train(self.h, model.m, feats.data_ptr(), targets.data_ptr(), feats.shape[0],
                                        ctypes.byref(c), ctypes.byref(loss), _stream_ptr(stream)), "smash_mlp_train")
        return float(loss.value)

    def mlp_gradient(self, model: "Model", feats, targets, stream=None):
        import torch
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=feats.device)
        loss = ctypes.c_float(0)
        _check(self.lib.smash_mlp_gradient(self.h, model.m, feats.contiguous().data_ptr(),
                                           targets.contiguous().data_ptr(), feats.shape[0], g.data_ptr(),
                                           ctypes.byref(loss), _stream_ptr(stream)), "smash_mlp_gradient")
        return g, float(loss.value)

    def mlp_predict(self, model: "Model", feats, stream=None, tensor_cores: bool = False):
        """Predictions of the model for raw features (device float32 [n, 6]);
        tensor_cores: the forward pass spgemm_learned uses (bf16 layer 2)."""
        import torch
        y = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
        fn = self.lib.smash_mlp_predict_tc if tensor_cores else self.lib.smash_mlp_predict
        _check(fn(self.h, model.m, feats.contiguous().data_ptr(), feats.shape[0], y.data_ptr(),
                  _stream_ptr(stream)), "smash_mlp_predict")
        return y

    def spgemm_learned(self, A: DeviceCsr, B: DeviceCsr, model: "Model | None", margin: float = 0.15, stream=None):
        """C = A*B sized by the model (model None: every row sized by its bound
        min(flop_i, cols), the same one-pass pipeline without the network).
        Returns (C as zero-copy views, stats, owner); call owner.free() (or let
        it be collected) to release C's arrays."""
        import torch
        dt = _dtype_code(A.val)
        sa, sb = A.struct(), B.struct()
        sc = CsrStruct()
        st = LearnedStats()
        _check(self.lib.spgemm_learned(self.h, ctypes.byref(sa), ctypes.byref(sb), dt,
                                       model.m if model is not None else None, margin,
                                       ctypes.byref(sc), ctypes.byref(st), _stream_ptr(stream)), "spgemm_learned")
        owner = LibraryCsr(self, sc)
        vdt = A.val.dtype
        C = DeviceCsr(int(sc.rows), int(sc.cols), _view(sc.row_ptr, int(sc.rows) + 1, torch.int64),
                      _view(sc.col_idx, int(sc.nnz), torch.int32), _view(sc.val, int(sc.nnz), vdt))
        return C, st.as_dict(), owner


def _pair_structs(pairs):
    n = len(pairs)
    SA = (CsrStruct * max(n, 1))()
    SB = (CsrStruct * max(n, 1))()
    for m, (A, B) in enumerate(pairs):
        SA[m] = A.struct()
        SB[m] = B.struct()
    return SA, SB


class BatchedInputs:
    """The descriptors of a list of (A, B) device pairs, built once and reused
    by every batched call on them (the arrays must stay alive and unchanged)."""

    def __init__(self, pairs):
        self.pairs = list(pairs)
        self.n = len(self.pairs)
        self.SA, self.SB = _pair_structs(self.pairs)
        self.dt = _dtype_code(self.pairs[0][0].val) if self.n else 0
        self.vdt = self.pairs[0][0].val.dtype if self.n else None


class BatchedResult:
    """The products of a batched call, C_m as zero-copy views made on access."""

    def __init__(self, structs, vdt):
        self.SC = structs
        self.vdt = vdt

    def __len__(self):
        return len(self.SC)

    def __getitem__(self, m):
        import torch
        if m < 0:
            m += len(self.SC)
        c = self.SC[m]
        return DeviceCsr(int(c.rows), int(c.cols), _view(c.row_ptr, int(c.rows) + 1, torch.int64),
                         _view(c.col_idx, int(c.nnz), torch.int32), _view(c.val, int(c.nnz), self.vdt))

    def __iter__(self):
        for m in range(len(self.SC)):
            yield self[m]


def _batched(self, pairs, stream=None):
    """C_m = A_m * B_m for all pairs (a list of (A, B), or BatchedInputs) in
    one persistent launch. Returns (the products, stats, owner): the products
    index as C_m views; owner.free() releases their memory."""
    inp = pairs if isinstance(pairs, BatchedInputs) else BatchedInputs(pairs)
    n = inp.n
    if n == 0:
        return BatchedResult([], None), BatchedStats().as_dict(), None
    SC = (CsrStruct * n)()
    st = BatchedStats()
    _check(self.lib.spgemm_batched(self.h, n, inp.SA, inp.SB, inp.dt, SC, ctypes.byref(st), _stream_ptr(stream)),
           "spgemm_batched")
    return BatchedResult(SC, inp.vdt), st.as_dict(), LibraryCsr(self, SC[0])


def _batched_autotune(self, pairs, stream=None):
    inp = pairs if isinstance(pairs, BatchedInputs) else BatchedInputs(pairs)
    bits = ctypes.c_int(0)
    ms = ctypes.c_float(0)
    _check(self.lib.smash_batched_autotune(self.h, inp.n, inp.SA, inp.SB, inp.dt, ctypes.byref(bits),
                                           ctypes.byref(ms), _stream_ptr(stream)), "smash_batched_autotune")
    return int(bits.value), float(ms.value)


def _batched_table_bits(self, bits=None):
    if bits is not None:
        _check(self.lib.smash_batched_set_table_bits(self.h, int(bits)), "smash_batched_set_table_bits")
    b = ctypes.c_int(0)
    _check(self.lib.smash_batched_get_table_bits(self.h, ctypes.byref(b)), "smash_batched_get_table_bits")
    return int(b.value)


def _batched_set_wait(self, wait_spins: int = 0, missing_arrivals: int = 0):
    _check(self.lib.smash_batched_set_wait(self.h, int(wait_spins), int(missing_arrivals)), "smash_batched_set_wait")


def _batched_row_cutoffs(self, warp_less=None, block_more=None):
    """Set (when given) and return (warp_less, block_more) of the batched kernel."""
    if warp_less is not None:
        _check(self.lib.smash_batched_set_row_cutoffs(self.h, int(warp_less), int(block_more)),
               "smash_batched_set_row_cutoffs")
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(self.lib.smash_batched_get_row_cutoffs(self.h, ctypes.byref(a), ctypes.byref(b)),
           "smash_batched_get_row_cutoffs")
    return int(a.value), int(b.value)


Handle.spgemm_batched = _batched
Handle.batched_row_cutoffs = _batched_row_cutoffs
Handle.batched_set_wait = _batched_set_wait
Handle.batched_autotune = _batched_autotune
Handle.batched_table_bits = _batched_table_bits


class LibraryCsr:
    """Owner of a CSR whose arrays the library allocated (learned / batched calls)."""

    def __init__(self, handle: Handle, s: CsrStruct):
        self.handle = handle
        self.s = s

    def free(self):
        if self.s is not None and self.handle.h:
            self.handle.lib.smash_free_csr(self.handle.h, ctypes.byref(self.s))
        self.s = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Model:
    """Row-size predictor (weights on the device)."""

    def __init__(self, handle: Handle, seed: int = 1):
        self.handle = handle
        self.lib = handle.lib
        m = ctypes.c_void_p()
        _check(self.lib.smash_model_create(handle.h, ctypes.byref(m), seed), "smash_model_create")
        self.m = m

    def close(self):
        if getattr(self, "m", None):
            self.lib.smash_model_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        n = np.zeros(12, dtype=np.float32)
        _check(self.lib.smash_model_get(self.m, p.ctypes.data, n.ctypes.data), "smash_model_get")
        return p, n

    def set(self, params=None, norm=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        n = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        _check(self.lib.smash_model_set(self.m, p.ctypes.data if p is not None else None,
                                        n.ctypes.data if n is not None else None), "smash_model_set")

    def save(self, path: str):
        _check(self.lib.smash_model_save(self.m, path.encode()), "smash_model_save")

    def load(self, path: str):
        _check(self.lib.smash_model_load(self.m, path.encode()), "smash_model_load")
