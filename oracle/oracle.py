"""ctypes wrapper around the C oracle -- test infrastructure only.

Every function here states one piece of what the GPU library computes, in the
plainest form, on the CPU, in FP64:

* ``multiply``      -- the local block-sparse product of the paper's Sec. II,
                       C = alpha*op(A)*op(B) + beta*C, on the blocked CSR layout;
                       optionally on a subset of C block rows, optionally in
                       double-double (Dot2) accumulation.
* ``stack_list``    -- the Traversal/Generation output of Sec. II (block-product
                       entries grouped into stacks of at most 30'000 per shape),
                       in one canonical order.
* ``densify`` /
  ``undensify``     -- Sec. III: coalescing all blocks into one dense matrix and
                       splitting it back following the original block sizes.
* ``dense_gemm``    -- the densified product of Sec. III (batch size 1), as a
                       plain triple loop.
* ``ozaki_*``       -- the INT8-slice emulation of an FP64 product (Ozaki,
                       Ogita, Oishi & Rump 2012, integer form), step by step.

Matrices are passed as any object with the attributes ``row_sizes``,
``col_sizes``, ``blk_row``, ``blk_col`` (int32 arrays) and ``data`` (float64:
the blocks concatenated in index order, each column-major).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


class _ObMat(C.Structure):
    _fields_ = [
        ("nbr", C.c_int), ("nbc", C.c_int),
        ("rs", C.POINTER(C.c_int)), ("cs", C.POINTER(C.c_int)),
        ("nblks", C.c_int64),
        ("br", C.POINTER(C.c_int)), ("bc", C.POINTER(C.c_int)),
        ("data", C.POINTER(C.c_double)),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.oracle_multiply.restype = C.c_int
        L.oracle_multiply.argtypes = [
            C.c_char, C.c_char, C.c_double, C.POINTER(_ObMat), C.POINTER(_ObMat),
            C.c_double, C.POINTER(_ObMat), C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int,
            C.POINTER(C.c_int64), C.POINTER(C.c_int64),
            C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        L.oracle_stack_list.restype = C.c_int64
        L.oracle_stack_list.argtypes = [C.c_char, C.c_char, C.POINTER(_ObMat), C.POINTER(_ObMat),
                                        C.c_int, C.POINTER(C.c_int), C.c_int64]
        L.oracle_dense_gemm.restype = None
        L.oracle_dense_gemm.argtypes = [C.c_char, C.c_char, C.c_int64, C.c_int64, C.c_int64,
                                        C.c_double, C.POINTER(C.c_double), C.c_int64,
                                        C.POINTER(C.c_double), C.c_int64, C.c_double,
                                        C.POINTER(C.c_double), C.c_int64, C.c_int]
        L.oracle_num_threads.restype = C.c_int
        _lib = L
    return _lib


@dataclass
class Blocks:
    """Result container: block index in CSR order and concatenated data."""
    row_sizes: np.ndarray
    col_sizes: np.ndarray
    blk_row: np.ndarray
    blk_col: np.ndarray
    data: np.ndarray
    blk_off: np.ndarray | None = None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _mk(M, keep):
    rs = np.ascontiguousarray(M.row_sizes, dtype=np.int32)
    cs = np.ascontiguousarray(M.col_sizes, dtype=np.int32)
    br = np.ascontiguousarray(M.blk_row, dtype=np.int32)
    bc = np.ascontiguousarray(M.blk_col, dtype=np.int32)
    d = np.ascontiguousarray(M.data, dtype=np.float64)
    if d.size == 0:
        d = np.zeros(1)
    keep.extend([rs, cs, br, bc, d])
    s = _ObMat(len(rs), len(cs), _ip(rs), _ip(cs), len(br), _ip(br), _ip(bc), _dp(d))
    return s


def threads() -> int:
    return lib().oracle_num_threads()


def multiply(transa, transb, alpha, A, B, beta, Cm=None, rows=None, mode=0, nthreads=0) -> Blocks:
    """C = alpha*op(A)*op(B) + beta*C (Sec. II). ``rows``: C block rows to compute.

    ``mode`` 0 = plain FP64 (k ascending, inner index ascending, no FMA
    contraction); 1 = double-double accumulation (Dot2); 2 = FP32 (inputs
    rounded to FP32, products and sums in FP32, alpha/beta in FP64).
    """
    keep = []
    a = _mk(A, keep)
    b = _mk(B, keep)
    c = _mk(Cm, keep) if Cm is not None else None
    rp = None
    nr = 0
    if rows is not None:
        r = np.ascontiguousarray(np.unique(np.asarray(rows, dtype=np.int32)))
        keep.append(r)
        rp, nr = _ip(r), len(r)
    nb, ne = C.c_int64(0), C.c_int64(0)
    L = lib()
    ta = transa.encode() if isinstance(transa, str) else transa
    tb = transb.encode() if isinstance(transb, str) else transb
    cref = C.byref(c) if c is not None else None
    rc = L.oracle_multiply(ta, tb, alpha, C.byref(a), C.byref(b), beta, cref, rp, nr, mode,
                           nthreads, C.byref(nb), C.byref(ne), None, None, None, None)
    if rc != 0:
        raise ValueError(f"oracle_multiply failed rc={rc}")
    obr = np.zeros(max(nb.value, 1), np.int32)
    obc = np.zeros(max(nb.value, 1), np.int32)
    ooff = np.zeros(max(nb.value, 1), np.int64)
    od = np.zeros(max(ne.value, 1), np.float64)
    rc = L.oracle_multiply(ta, tb, alpha, C.byref(a), C.byref(b), beta, cref, rp, nr, mode,
                           nthreads, C.byref(nb), C.byref(ne), _ip(obr), _ip(obc),
                           ooff.ctypes.data_as(C.POINTER(C.c_int64)), _dp(od))
    if rc != 0:
        raise ValueError(f"oracle_multiply failed rc={rc}")
    tr_a = transa in ("T", "t", "C", "c", b"T", b"C")
    tr_b = transb in ("T", "t", "C", "c", b"T", b"C")
    rs = np.asarray(A.col_sizes if tr_a else A.row_sizes, np.int32)
    cs = np.asarray(B.row_sizes if tr_b else B.col_sizes, np.int32)
    n = nb.value
    return Blocks(rs, cs, obr[:n], obc[:n], od[:ne.value], ooff[:n])


def stack_list(transa, transb, A, B, stack_cap=30000) -> np.ndarray:
    """Canonical stack list: int32 array (P, 7) of (stack, m, n, k, i, j, kblk)."""
    keep = []
    a = _mk(A, keep)
    b = _mk(B, keep)
    L = lib()
    ta = transa.encode() if isinstance(transa, str) else transa
    tb = transb.encode() if isinstance(transb, str) else transb
    n = L.oracle_stack_list(ta, tb, C.byref(a), C.byref(b), stack_cap, None, 0)
    if n < 0:
        raise ValueError(f"oracle_stack_list failed rc={n}")
    out = np.zeros((max(n, 1), 7), np.int32)
    n2 = L.oracle_stack_list(ta, tb, C.byref(a), C.byref(b), stack_cap, _ip(out), n)
    if n2 != n:
        raise ValueError("oracle_stack_list inconsistent count")
    return out[:n]


def dense_gemm(transa, transb, alpha, A, B, beta, Cd, nthreads=0):
    """Plain triple-loop GEMM on column-major (Fortran-ordered) 2-D arrays; updates Cd."""
    A = np.asfortranarray(A, dtype=np.float64)
    B = np.asfortranarray(B, dtype=np.float64)
    assert Cd.flags.f_contiguous and Cd.dtype == np.float64
    M, N = Cd.shape
    K = A.shape[0] if transa in ("T", "C") else A.shape[1]
    lib().oracle_dense_gemm(transa.encode(), transb.encode(), M, N, K, alpha, _dp(A), A.shape[0],
                            _dp(B), B.shape[0], beta, _dp(Cd), M, nthreads)
    return Cd


# --------------------------------------------------------------------------
# Densification (Sec. III): all blocks coalesced into one dense matrix, and
# the inverse split following the original block sizes.
# --------------------------------------------------------------------------
def densify(M) -> np.ndarray:
    """Dense (sum row sizes) x (sum col sizes) matrix; absent blocks are zero."""
    rs = np.asarray(M.row_sizes, np.int64)
    cs = np.asarray(M.col_sizes, np.int64)
    ro = np.concatenate([[0], np.cumsum(rs)])
    co = np.concatenate([[0], np.cumsum(cs)])
    D = np.zeros((int(ro[-1]), int(co[-1])), order="F")
    pos = 0
    for i, j in zip(np.asarray(M.blk_row), np.asarray(M.blk_col)):
        m, n = int(rs[i]), int(cs[j])
        D[ro[i]:ro[i] + m, co[j]:co[j] + n] = np.asarray(M.data[pos:pos + m * n]).reshape((m, n), order="F")
        pos += m * n
    return D


def undensify(D, row_sizes, col_sizes, blk_row, blk_col) -> np.ndarray:
    """Concatenated column-major blocks of D at the given block coordinates."""
    rs = np.asarray(row_sizes, np.int64)
    cs = np.asarray(col_sizes, np.int64)
    ro = np.concatenate([[0], np.cumsum(rs)])
    co = np.concatenate([[0], np.cumsum(cs)])
    out = []
    for i, j in zip(np.asarray(blk_row), np.asarray(blk_col)):
        out.append(np.asarray(D[ro[i]:ro[i] + rs[i], co[j]:co[j] + cs[j]]).reshape(-1, order="F"))
    return np.concatenate(out) if out else np.zeros(0)


def normwise_error(Cd, Cref, Ad, Bd) -> float:
    """||C - C_ref||_F / (||A||_F * ||B||_F), the accuracy measure used throughout."""
    den = np.linalg.norm(Ad) * np.linalg.norm(Bd)
    return float(np.linalg.norm(np.asarray(Cd) - np.asarray(Cref)) / (den if den > 0 else 1.0))


# --------------------------------------------------------------------------
# Emulated FP64 with 7-bit integer slices (Ozaki et al. 2012, integer form):
# row/column power-of-two scaling, truncated slices, exact integer level sums
# G_d (d = t + u <= s + 1), FP64 recombination from the smallest level up.
# --------------------------------------------------------------------------
def _ozaki_sigs():
    L = lib()
    if getattr(L, "_oz_ready", False):
        return L
    L.oracle_round_scaled_parts.restype = C.c_double
    L.oracle_round_scaled_parts.argtypes = [C.c_int64, C.c_uint64, C.c_int]
    L.oracle_ozaki_split.restype = None
    L.oracle_ozaki_split.argtypes = [C.c_double, C.c_int, C.POINTER(C.c_int)]
    L.oracle_ozaki_exponents.restype = None
    L.oracle_ozaki_exponents.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_double), C.c_int64,
                                         C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int),
                                         C.POINTER(C.c_int)]
    L.oracle_ozaki_gemm.restype = C.c_int
    L.oracle_ozaki_gemm.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_double, C.POINTER(C.c_double), C.c_int64,
                                    C.POINTER(C.c_double), C.c_int64, C.c_double, C.POINTER(C.c_double),
                                    C.c_int64, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int,
                                    C.POINTER(C.c_int64)]
    L._oz_ready = True
    return L


# exponent marker of a row of A / column of B that holds a NaN or an infinity:
# every C element of that row / column is NaN
OZ_NONFINITE = 1 << 20


def round_scaled(S: int, k: int) -> float:
    """The integer S (|S| < 2^127) times 2^k, rounded once to the nearest double."""
    S = int(S)
    assert -(1 << 127) < S < (1 << 127)
    u = S & ((1 << 128) - 1)
    hi, lo = u >> 64, u & ((1 << 64) - 1)
    if hi >= 1 << 63:
        hi -= 1 << 64
    return _ozaki_sigs().oracle_round_scaled_parts(hi, lo, int(k))


def ozaki_split(x: float, s: int):
    """Slices sigma_1..sigma_s of one pre-scaled value |x| < 1."""
    out = (C.c_int * s)()
    _ozaki_sigs().oracle_ozaki_split(float(x), s, out)
    return list(out)


def ozaki_exponents(Ad, Bd):
    Ad = np.asfortranarray(Ad, np.float64)
    Bd = np.asfortranarray(Bd, np.float64)
    M, K = Ad.shape
    N = Bd.shape[1]
    e = np.zeros(max(M, 1), np.int32)
    f = np.zeros(max(N, 1), np.int32)
    _ozaki_sigs().oracle_ozaki_exponents(M, N, K, _dp(Ad), max(M, 1), _dp(Bd), max(K, 1), _ip(e), _ip(f))
    return e[:M], f[:N]


def ozaki_gemm(alpha, Ad, Bd, beta, Cd, s=7, rows=None, nthreads=0, want_levels=False):
    """Emulated C = alpha*A*B + beta*C on dense column-major arrays (updates Cd).

    rows: only these rows of C are computed (the others are left as they are).
    Returns (Cd, levels) with levels[d-2][q][j] = G_d for the selected rows.
    """
    Ad = np.asfortranarray(Ad, np.float64)
    Bd = np.asfortranarray(Bd, np.float64)
    assert Cd.flags.f_contiguous and Cd.dtype == np.float64
    M, K = Ad.shape
    N = Bd.shape[1]
    rp, nr = None, 0
    keep = []
    if rows is not None:
        r = np.ascontiguousarray(np.unique(np.asarray(rows, np.int32)))
        keep.append(r)
        rp, nr = _ip(r), len(r)
    nsel = nr if rows is not None else M
    lv = np.zeros((s, max(nsel, 1), max(N, 1)), np.int64) if want_levels else None
    rc = _ozaki_sigs().oracle_ozaki_gemm(M, N, K, alpha, _dp(Ad), max(M, 1), _dp(Bd), max(K, 1), beta, _dp(Cd),
                                         max(M, 1), s, rp, nr, nthreads,
                                         lv.ctypes.data_as(C.POINTER(C.c_int64)) if lv is not None else None)
    if rc != 0:
        raise ValueError("oracle_ozaki_gemm failed")
    return Cd, lv


# --------------------------------------------------------------------------
# TF32 variant: inputs rounded FP64 -> FP32 (nearest even) -> TF32 (10-bit
# mantissa, nearest with ties away from zero); products and sums in FP32.
# --------------------------------------------------------------------------
def round_tf32(x) -> np.ndarray:
    """FP64 values rounded to TF32 (returned as FP64, exactly representable)."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).copy()
    mag = b & np.uint32(0x7FFFFFFF)
    finite = mag < np.uint32(0x7F800000)
    r = (mag + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    b = np.where(finite, (b & np.uint32(0x80000000)) | r, b)
    return b.view(np.float32).astype(np.float64)
