"""Helpers shared by the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr
from paper_1910_04796_gb300.synth import BlockSparse

_ready = False


def setup():
    global _ready
    if not _ready:
        dbcsr.init()
        _ready = True


def to_gpu(M):
    return dbcsr.Matrix.from_blocks(M)


def empty_like_c(row_sizes, col_sizes):
    return dbcsr.Matrix.create(row_sizes, col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))


def from_gpu(Mg, row_sizes, col_sizes):
    br, bc, off = Mg.index()
    return BlockSparse(np.asarray(row_sizes, np.int32), np.asarray(col_sizes, np.int32), br, bc, Mg.data())


def op_sizes(A, B, ta, tb):
    rs = A.col_sizes if ta in "TC" else A.row_sizes
    cs = B.row_sizes if tb in "TC" else B.col_sizes
    return np.asarray(rs, np.int32), np.asarray(cs, np.int32)


def gpu_multiply(ta, tb, alpha, A, B, beta, Cm=None, **kw):
    """Run the CUDA path; returns the result as BlockSparse (CSR order) and stats."""
    setup()
    rs, cs = op_sizes(A, B, ta, tb)
    Ag, Bg = to_gpu(A), to_gpu(B)
    Cg = to_gpu(Cm) if Cm is not None else empty_like_c(rs, cs)
    dbcsr.multiply(ta, tb, alpha, Ag, Bg, beta, Cg, **kw)
    st = dbcsr.stats()
    res = from_gpu(Cg, rs, cs)
    for m in (Ag, Bg, Cg):
        m.release()
    return res, st


def assert_same_pattern(got, ref):
    assert np.array_equal(np.asarray(got.blk_row), np.asarray(ref.blk_row)), "block rows differ"
    assert np.array_equal(np.asarray(got.blk_col), np.asarray(ref.blk_col)), "block cols differ"


def normwise(got, ref, A, B, ta="N", tb="N"):
    Ad = O.densify(A)
    Bd = O.densify(B)
    return O.normwise_error(O.densify(got), O.densify(ref), Ad, Bd)
