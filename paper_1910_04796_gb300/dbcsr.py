"""Thin ctypes binding of ``libdbcsr_gb.so`` (C ABI in ``include/dbcsr_gb.h``).

Argument marshalling only: every step of the multiply runs in the library's
CUDA kernels. PyTorch supplies the CUDA stream (and, optionally, the device
allocator). The binding refuses to run without the compiled library -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERR_ARG, ERR_DIM, ERR_ALLOC, ERR_OVERFLOW, ERR_TIMEOUT, ERR_CUDA, ERR_STATE = -1, -2, -3, -4, -5, -6, -7
PATH_AUTO, PATH_STACKS, PATH_DENSE, PATH_HYBRID = 0, 1, 2, 3
PREC_FP64, PREC_OZAKI, PREC_TF32, PREC_FP32 = 0, 1, 2, 3
_PREC = {"fp64": PREC_FP64, "ozaki": PREC_OZAKI, "tf32": PREC_TF32, "fp32": PREC_FP32}
_PATH = {"auto": PATH_AUTO, "stacks": PATH_STACKS, "dense": PATH_DENSE, "hybrid": PATH_HYBRID}


class DbcsrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dbcsr error {code}: {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("path", C.c_int), ("precision", C.c_int), ("ozaki_slices", C.c_int),
                ("kernel", C.c_int), ("timing", C.c_int), ("reuse_plan", C.c_int), ("hybrid_panel", C.c_int),
                ("hybrid_fill_pct", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_products", C.c_int64), ("n_stacks", C.c_int64), ("n_shapes", C.c_int64),
                ("c_blocks", C.c_int64), ("useful_flops", C.c_double), ("path", C.c_int),
                ("precision", C.c_int), ("kernel_launches", C.c_int), ("dense_panels", C.c_int),
                ("ms_setup", C.c_float), ("ms_main", C.c_float), ("ms_finish", C.c_float),
                ("ms_total", C.c_float), ("main_flops", C.c_double), ("main_bytes", C.c_double),
                ("ms_kernel", C.c_float), ("reserved_f", C.c_float)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None
_keep = []

# C-ABI entry points declared in include/dbcsr_gb.h: (name, restype, argtypes)
_P = C.c_void_p
_IP = C.POINTER(C.c_int)
_LP = C.POINTER(C.c_int64)
_DP = C.POINTER(C.c_double)
SIGNATURES = [
    ("dbcsr_init", C.c_int, [_P]),
    ("dbcsr_set_allocator", C.c_int, [ALLOC_FN, FREE_FN, _P]),
    ("dbcsr_create", C.c_int, [C.POINTER(_P), C.c_int, C.c_int, _IP, _IP, C.c_int64, _IP, _IP, _P, C.c_int]),
    ("dbcsr_release", C.c_int, [C.POINTER(_P)]),
    ("dbcsr_get_info", C.c_int, [_P, _IP, _IP, _LP, _LP]),
    ("dbcsr_get_index", C.c_int, [_P, _IP, _IP, _LP]),
    ("dbcsr_get_data", C.c_int, [_P, _P, C.c_int]),
    ("dbcsr_set_data", C.c_int, [_P, _P, C.c_int]),
    ("dbcsr_data_ptr", C.c_int, [_P, C.POINTER(_P)]),
    ("dbcsr_get_block", C.c_int, [_P, C.c_int, C.c_int, _DP, _IP]),
    ("dbcsr_multiply", C.c_int, [C.c_char, C.c_char, C.c_double, _P, _P, C.c_double, _P, C.POINTER(Opts)]),
    ("dbcsr_get_stats", C.c_int, [C.POINTER(Stats)]),
    ("dbcsr_set_tuning", C.c_int, [_IP, _IP, _IP, C.c_int]),
    ("dbcsr_set_tuning_mnk", C.c_int, [_IP, _IP, _IP, _IP, C.c_int]),
    ("dbcsr_get_stacks", C.c_int, [C.c_char, C.c_char, _P, _P, C.c_int, _IP, C.c_int64, _LP]),
    ("dbcsr_dgemm_emulated_noalloc", C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_double, _P, C.c_int64, _P,
                                               C.c_int64, C.c_double, _P, C.c_int64, C.c_int, _P]),
    ("dbcsr_set_wait_limit", C.c_int, [C.c_int64]),
    ("dbcsr_sync", C.c_int, []),
    ("dbcsr_last_error", C.c_char_p, []),
    ("dbcsr_version", C.c_char_p, []),
]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load the compiled library (building it first if asked). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or (build_if_missing and not _build.up_to_date()):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is not built")
        _build.build()
    L = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        raise DbcsrError(rc, load().dbcsr_last_error().decode())


def init(stream=None):
    """Bind the library to a CUDA stream (default: torch's current stream)."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("dbcsr: no CUDA device -- the library has no CPU path")
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    _check(load().dbcsr_init(C.c_void_p(handle)))


def set_allocator(alloc=None, free=None):
    """Route device allocations through Python callables (dbcsr_set_allocator).

    ``alloc(nbytes, stream)`` returns a device address (int), or None to refuse;
    ``free(ptr, nbytes, stream)`` takes back what ``alloc`` gave. Both None
    restores the library's own stream-ordered pool. The library returns every
    block to the hook that made it, even after a switch, so the callables are
    kept alive for the life of the process.
    """
    L = load()
    if alloc is None and free is None:
        _check(L.dbcsr_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return
    if alloc is None or free is None:
        raise ValueError("set_allocator: give both alloc and free, or neither")
    def _alloc(nbytes, stream, ctx):
        try:
            return alloc(int(nbytes), stream or 0)
        except Exception:  # an exception must not cross into C: report a refusal
            return None

    fa = ALLOC_FN(_alloc)
    ff = FREE_FN(lambda ptr, nbytes, stream, ctx: free(ptr, int(nbytes), stream or 0))
    _keep.extend([fa, ff])
    _check(L.dbcsr_set_allocator(fa, ff, None))


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch
    L = load()
    if not enable:
        _check(L.dbcsr_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:  # allocation failure is reported to the library as NULL
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    _keep.extend([fa, ff])
    _check(L.dbcsr_set_allocator(fa, ff, None))


def _ip(a):
    return a.ctypes.data_as(_IP)


class Matrix:
    """Handle of a library-owned block-sparse matrix."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)

    @classmethod
    def create(cls, row_sizes, col_sizes, blk_row, blk_col, data=None):
        """Create from host arrays; ``data`` is numpy (host) or a CUDA torch tensor (device)."""
        L = load()
        rs = np.ascontiguousarray(row_sizes, np.int32)
        cs = np.ascontiguousarray(col_sizes, np.int32)
        br = np.ascontiguousarray(blk_row, np.int32)
        bc = np.ascontiguousarray(blk_col, np.int32)
        h = C.c_void_p()
        on_dev = 0
        ptr = None
        keep = None
        if data is not None:
            if hasattr(data, "is_cuda") and data.is_cuda:
                import torch
                assert data.dtype == torch.float64 and data.is_contiguous()
                ptr, on_dev = C.c_void_p(data.data_ptr()), 1
            else:
                keep = np.ascontiguousarray(data, np.float64)
                ptr = keep.ctypes.data_as(C.c_void_p)
        _check(L.dbcsr_create(C.byref(h), len(rs), len(cs), _ip(rs), _ip(cs), len(br), _ip(br), _ip(bc),
                              ptr, on_dev))
        return cls(h.value)

    @classmethod
    def from_blocks(cls, M, device_data=None):
        """Create from any object with row_sizes/col_sizes/blk_row/blk_col/data."""
        return cls.create(M.row_sizes, M.col_sizes, M.blk_row, M.blk_col,
                          device_data if device_data is not None else M.data)

    @property
    def handle(self):
        return self._h

    def release(self):
        if self._h and self._h.value:
            _check(load().dbcsr_release(C.byref(self._h)))

    def __del__(self):
        try:
            if _lib is not None and self._h and self._h.value:
                _lib.dbcsr_release(C.byref(self._h))
        except Exception:
            pass

    def info(self):
        a, b = C.c_int(), C.c_int()
        n, e = C.c_int64(), C.c_int64()
        _check(load().dbcsr_get_info(self._h, C.byref(a), C.byref(b), C.byref(n), C.byref(e)))
        return a.value, b.value, n.value, e.value

    def index(self):
        nbr, nbc, n, e = self.info()
        br = np.zeros(max(n, 1), np.int32)
        bc = np.zeros(max(n, 1), np.int32)
        off = np.zeros(max(n, 1), np.int64)
        _check(load().dbcsr_get_index(self._h, _ip(br), _ip(bc), off.ctypes.data_as(_LP)))
        return br[:n], bc[:n], off[:n]

    def data(self, out: np.ndarray | None = None) -> np.ndarray:
        """The stored values (CSR block order) on the host; ``out``: a float64
        host array of at least nelems entries to fill (e.g. pinned memory)."""
        nbr, nbc, n, e = self.info()
        if out is None:
            out = np.zeros(max(e, 1), np.float64)
        elif out.dtype != np.float64 or out.size < e or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out: contiguous float64 array with at least nelems entries")
        _check(load().dbcsr_get_data(self._h, out.ctypes.data_as(C.c_void_p), 0))
        return out[:e]

    def data_device(self):
        """A CUDA torch tensor copy of the stored values (device to device)."""
        import torch
        nbr, nbc, n, e = self.info()
        out = torch.empty(max(e, 1), dtype=torch.float64, device="cuda")
        _check(load().dbcsr_get_data(self._h, C.c_void_p(out.data_ptr()), 1))
        return out[:e]

    def set_data(self, data):
        """Overwrite the stored values (numpy host array or CUDA float64 tensor, storage order)."""
        if hasattr(data, "is_cuda") and data.is_cuda:
            _check(load().dbcsr_set_data(self._h, C.c_void_p(data.data_ptr()), 1))
        else:
            d = np.ascontiguousarray(data, np.float64)
            _check(load().dbcsr_set_data(self._h, d.ctypes.data_as(C.c_void_p), 0))

    def data_ptr(self) -> int:
        p = C.c_void_p()
        _check(load().dbcsr_data_ptr(self._h, C.byref(p)))
        return p.value or 0

    def get_block(self, row, col, m, n):
        out = np.zeros(m * n, np.float64)
        found = C.c_int()
        _check(load().dbcsr_get_block(self._h, row, col, out.ctypes.data_as(_DP), C.byref(found)))
        return out.reshape((m, n), order="F") if found.value else None


def opts(path="auto", precision="fp64", ozaki_slices=0, kernel=0, timing=False, reuse_plan=False,
         hybrid_panel=0, hybrid_fill_pct=0) -> Opts:
    o = Opts()
    o.hybrid_panel = int(hybrid_panel)
    o.hybrid_fill_pct = int(hybrid_fill_pct)
    o.timing = 1 if timing else 0
    o.reuse_plan = 1 if reuse_plan else 0
    o.path = _PATH[path] if isinstance(path, str) else int(path)
    o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    o.ozaki_slices = ozaki_slices
    o.kernel = kernel
    return o


def multiply(transa, transb, alpha, A: Matrix, B: Matrix, beta, Cm: Matrix, path="auto", precision="fp64",
             ozaki_slices=0, kernel=0, timing=False, reuse_plan=False, hybrid_panel=0, hybrid_fill_pct=0):
    """C = alpha*op(A)*op(B) + beta*C on the GPU (see dbcsr_multiply)."""
    o = opts(path, precision, ozaki_slices, kernel, timing, reuse_plan, hybrid_panel, hybrid_fill_pct)
    _check(load().dbcsr_multiply(transa.encode(), transb.encode(), float(alpha), A.handle, B.handle,
                                 float(beta), Cm.handle, C.byref(o)))


def set_tuning(entries):
    """FP64 stack-kernel variant per C-block shape: iterable of (m, n, variant)."""
    e = np.asarray(list(entries), np.int32).reshape(-1, 3)
    m, n, v = (np.ascontiguousarray(e[:, q]) for q in range(3))
    _check(load().dbcsr_set_tuning(_ip(m), _ip(n), _ip(v), len(e)))


def set_tuning_mnk(entries):
    """FP64 stack-kernel variant per (m, n, k): iterable of (m, n, k, variant), all
    sizes 1..32; k is the inner size of a C block's first product. An empty
    iterable clears the table."""
    e = np.asarray(list(entries), np.int32).reshape(-1, 4)
    m, n, k, v = (np.ascontiguousarray(e[:, q]) for q in range(4))
    _check(load().dbcsr_set_tuning_mnk(_ip(m), _ip(n), _ip(k), _ip(v), len(e)))


def stats() -> dict:
    s = Stats()
    _check(load().dbcsr_get_stats(C.byref(s)))
    return {f: getattr(s, f) for f, _ in Stats._fields_ if f != "reserved"}


def get_stacks(transa, transb, A: Matrix, B: Matrix, stack_cap=30000) -> np.ndarray:
    """Canonical stack list as the GPU builds it: int32 (P, 7) = (stack, m, n, k, i, j, kblk)."""
    L = load()
    n = C.c_int64()
    _check(L.dbcsr_get_stacks(transa.encode(), transb.encode(), A.handle, B.handle, stack_cap, None, 0,
                              C.byref(n)))
    out = np.zeros((max(n.value, 1), 7), np.int32)
    _check(L.dbcsr_get_stacks(transa.encode(), transb.encode(), A.handle, B.handle, stack_cap, _ip(out),
                              n.value, C.byref(n)))
    return out[:n.value]


def sync():
    _check(load().dbcsr_sync())


def set_wait_limit(ns: int = 0):
    """Limit of each bounded wait in the tensor-core pipelines (dbcsr_set_wait_limit); 0 = default 4 s."""
    _check(load().dbcsr_set_wait_limit(int(ns)))


def version() -> str:
    return load().dbcsr_version().decode()


def has_precision(name: str) -> bool:
    """Whether the library implements the given precision (fp64, ozaki, tf32, fp32)."""
    return name in _AVAILABLE


_AVAILABLE = {"fp64", "ozaki", "tf32", "fp32"}


def dgemm_emulated_noalloc(alpha, A, B, beta, Cmat, slices=0, stream=None):
    """C = alpha*A*B + beta*C (emulated FP64) with no device allocation.

    A (M x K), B (K x N), C (M x N) are CUDA float64 tensors holding the
    matrices column-major, i.e. passed as their transposes in torch's
    row-major terms: A is a (K, M) contiguous tensor, etc. See
    dbcsr_dgemm_emulated_noalloc for who needs this and its size limit.
    """
    import torch
    K, M = A.shape
    N, K2 = B.shape
    assert K2 == K and tuple(Cmat.shape) == (N, M)
    for t in (A, B, Cmat):
        assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().dbcsr_dgemm_emulated_noalloc(M, N, K, float(alpha), C.c_void_p(A.data_ptr()), M,
                                               C.c_void_p(B.data_ptr()), K, float(beta),
                                               C.c_void_p(Cmat.data_ptr()), M, slices,
                                               C.c_void_p(stream.cuda_stream)))
