"""Uploads of host values on the transfer stream (GPU).

Values handed to dbcsr_create / dbcsr_set_data from page-locked memory are
copied on the library's transfer stream while the call returns (Sec. II:
host-to-device transfers overlapped with the computation through CUDA
streams); every later use of the matrix waits for its copy. The emulated dense
path waits for each operand where it first reads it, and for C only before the
recombination. A multiply issued right after the creates must give the same
bits as the same multiply from pageable inputs, whose copies complete inside
the call: a use that ran ahead of its copy would read stale or uninitialised
values and differ. (The pageable inputs' results are checked against the
oracle by the other parity tests.)
"""
import numpy as np
import pytest

from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import assert_same_pattern, from_gpu, setup

pytestmark = pytest.mark.gpu


def pinned(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory()
    return t, t.numpy()


def make(M, data):
    return dbcsr.Matrix.create(M.row_sizes, M.col_sizes, M.blk_row, M.blk_col, data)


def run(A, B, Cm, beta, keep, **kw):
    """Create A, B, C from the given host arrays and multiply at once."""
    Ag, Bg, Cg = make(A, keep[0]), make(B, keep[1]), make(Cm, keep[2])
    dbcsr.multiply("N", "N", 1.0, Ag, Bg, beta, Cg, **kw)
    got = from_gpu(Cg, Cm.row_sizes, B.col_sizes)
    for M in (Ag, Bg, Cg):
        M.release()
    return got


@pytest.mark.parametrize("precision,path,nb,bs", [("ozaki", "dense", 64, 22), ("ozaki", "dense", 12, 32),
                                                  ("fp64", "stacks", 48, 22), ("fp64", "dense", 24, 22)])
def test_pinned_creates_match_pageable(precision, path, nb, bs):
    # 64 x 64 blocks of 22: 16 MB per operand, so the copies take a while;
    # the 12 x 12 case has N < 256 (128-wide tiles, densified operands)
    setup()
    rng = np.random.default_rng(1100 + nb)
    A = synth.dense_matrix(rng, nb, nb, bs, bs)
    B = synth.dense_matrix(rng, nb, nb, bs, bs)
    Cm = synth.dense_matrix(rng, nb, nb, bs, bs)
    want = run(A, B, Cm, 1.0, (A.data, B.data, Cm.data), precision=precision, path=path)
    tA, hA = pinned(A.data)
    tB, hB = pinned(B.data)
    tC, hC = pinned(Cm.data)
    for _ in range(2):
        got = run(A, B, Cm, 1.0, (hA, hB, hC), precision=precision, path=path)
        assert_same_pattern(got, want)
        assert np.array_equal(got.data, want.data)


def test_pinned_set_data_then_multiply():
    # new values from pinned memory replace the old ones before the next multiply reads them
    setup()
    rng = np.random.default_rng(1110)
    A = synth.dense_matrix(rng, 40, 40, 22, 22)
    B = synth.dense_matrix(rng, 40, 40, 22, 22)
    A2 = synth.dense_matrix(rng, 40, 40, 22, 22)
    Ag, Bg = make(A, A.data), make(B, B.data)
    Cg = dbcsr.Matrix.create(A.row_sizes, B.col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))
    ref2 = make(A2, A2.data)
    Cref = dbcsr.Matrix.create(A.row_sizes, B.col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))
    dbcsr.multiply("N", "N", 1.0, ref2, Bg, 0.0, Cref, precision="ozaki", path="dense")
    want = Cref.data().copy()
    t2, h2 = pinned(A2.data)
    for _ in range(2):
        dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.0, Cg, precision="ozaki", path="dense")   # queued work on A
        Ag.set_data(h2)
        dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.0, Cg, precision="ozaki", path="dense")
        assert np.array_equal(Cg.data(), want)
        Ag.set_data(A.data)
    for M in (Ag, Bg, Cg, ref2, Cref):
        M.release()


def test_release_and_data_ptr_while_uploading():
    # a matrix released right after its create, with the copy still in flight;
    # and a device pointer taken right after a create, whose values are then
    # copied device to device on the library stream into a second matrix:
    # both wait for the copy
    import ctypes as C
    setup()
    rng = np.random.default_rng(1120)
    A = synth.dense_matrix(rng, 64, 64, 22, 22)
    tA, hA = pinned(A.data)
    for _ in range(3):
        make(A, hA).release()
    L = dbcsr.load()
    for _ in range(2):
        Ag = make(A, hA)
        ptr = Ag.data_ptr()
        rs = np.ascontiguousarray(A.row_sizes, np.int32)
        cs = np.ascontiguousarray(A.col_sizes, np.int32)
        br = np.ascontiguousarray(A.blk_row, np.int32)
        bc = np.ascontiguousarray(A.blk_col, np.int32)
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
        h = C.c_void_p()
        assert L.dbcsr_create(C.byref(h), len(rs), len(cs), ip(rs), ip(cs), len(br), ip(br), ip(bc),
                              C.c_void_p(ptr), 1) == dbcsr.OK
        copy = dbcsr.Matrix(h.value)
        assert np.array_equal(copy.data(), A.data)
        copy.release()
        Ag.release()


def test_stream_switch_with_upload_in_flight():
    # the copies were queued while one library stream was current; the multiply
    # runs on another, and still waits for them
    import torch
    setup()
    rng = np.random.default_rng(1130)
    A = synth.dense_matrix(rng, 48, 48, 22, 22)
    B = synth.dense_matrix(rng, 48, 48, 22, 22)
    Cm = synth.dense_matrix(rng, 48, 48, 22, 22)
    want = run(A, B, Cm, 0.5, (A.data, B.data, Cm.data), precision="ozaki", path="dense")
    keep = [pinned(x.data) for x in (A, B, Cm)]
    Ag, Bg, Cg = make(A, keep[0][1]), make(B, keep[1][1]), make(Cm, keep[2][1])
    s = torch.cuda.Stream()
    dbcsr.init(s)
    try:
        dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.5, Cg, precision="ozaki", path="dense")
        got = from_gpu(Cg, Cm.row_sizes, B.col_sizes)
    finally:
        dbcsr.init()
    assert np.array_equal(got.data, want.data)
    for M in (Ag, Bg, Cg):
        M.release()
