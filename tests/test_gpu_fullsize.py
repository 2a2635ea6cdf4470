"""Parity at the workloads' full sizes, in the configuration bench.py times.

The oracle cannot redo whole products of this size, so each test checks
either sampled C block rows that the oracle computes one by one (same inputs,
same definition), or, for the largest dense shapes, a property that holds at
any size: the projection C x = alpha A (B x) + beta C0 x for a random x
(Freivalds), computed by the oracle's plain loops, within the FP64 rounding
bound of the two orders of summation.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import from_gpu, setup

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def run(w, path, precision, slices=0):
    setup()
    rs = w.A.col_sizes if w.transa == "T" else w.A.row_sizes
    cs = w.B.row_sizes if w.transb == "T" else w.B.col_sizes
    Ag, Bg = dbcsr.Matrix.from_blocks(w.A), dbcsr.Matrix.from_blocks(w.B)
    Cg = dbcsr.Matrix.from_blocks(w.C) if w.C is not None else dbcsr.Matrix.create(
        rs, cs, np.zeros(0, np.int32), np.zeros(0, np.int32))
    dbcsr.multiply(w.transa, w.transb, w.alpha, Ag, Bg, w.beta, Cg, path=path, precision=precision,
                   ozaki_slices=slices)
    st = dbcsr.stats()
    got = from_gpu(Cg, rs, cs)
    for m in (Ag, Bg, Cg):
        m.release()
    return got, st


def blocks_of_rows(M, rows):
    """Sub-list (block index + data) of the blocks in the given block rows, CSR order."""
    rs = np.asarray(M.row_sizes, np.int64)
    cs = np.asarray(M.col_sizes, np.int64)
    sizes = rs[M.blk_row] * cs[M.blk_col]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    keep = np.isin(M.blk_row, rows)
    data = np.concatenate([M.data[offs[b]:offs[b + 1]] for b in np.nonzero(keep)[0]])
    return M.blk_row[keep], M.blk_col[keep], data


def frob(M):
    return float(np.linalg.norm(M.data))


def check_rows(got, ref, A, B, tol, exact=False):
    rows = np.unique(ref.blk_row)
    gbr, gbc, gdata = blocks_of_rows(got, rows)
    assert np.array_equal(gbr, ref.blk_row) and np.array_equal(gbc, ref.blk_col)
    if exact:
        assert np.array_equal(gdata, ref.data)
    else:
        err = np.linalg.norm(gdata - ref.data) / (frob(A) * frob(B))
        assert err <= tol, err


def sample_rows(n, k, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int32)


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_dense_limit_N11264(precision):
    w = synth.workload_dense_limit()
    got, st = run(w, "auto", precision)
    assert st["path"] == dbcsr.PATH_DENSE
    rows = sample_rows(512, 3, seed=1)
    if precision == "fp64":
        ref = O.multiply("N", "N", w.alpha, w.A, w.B, w.beta, w.C, rows=rows)
        check_rows(got, ref, w.A, w.B, 1e-13)
    else:
        ref = O.multiply("N", "N", w.alpha, w.A, w.B, w.beta, w.C, rows=rows, mode=1)
        check_rows(got, ref, w.A, w.B, 1e-12)


def freivalds(w, got, tol):
    """||C x - (alpha op(A) (op(B) x) + beta C0 x)|| against FP64 rounding of both sides."""
    rng = np.random.default_rng(7)
    Bd = O.densify(w.B)
    Ad = O.densify(w.A)
    Bop = Bd.T if w.transb == "T" else Bd
    Aop = Ad.T if w.transa == "T" else Ad
    x = np.asfortranarray(rng.uniform(-1, 1, (Bop.shape[1], 1)))
    bx = np.zeros((Bop.shape[0], 1), order="F")
    O.dense_gemm("N", "N", 1.0, np.asfortranarray(Bop), x, 0.0, bx)
    rhs = np.zeros((Aop.shape[0], 1), order="F")
    O.dense_gemm("N", "N", w.alpha, np.asfortranarray(Aop), bx, 0.0, rhs)
    Cd = O.densify(got)
    cx = np.zeros((Cd.shape[0], 1), order="F")
    O.dense_gemm("N", "N", 1.0, Cd, x, 0.0, cx)
    # normwise: ||C x - A B x|| / (||A||_F ||B||_F ||x||)
    err = np.linalg.norm(cx - rhs) / (np.linalg.norm(Ad) * np.linalg.norm(Bd) * np.linalg.norm(x))
    assert err <= tol, err


@pytest.mark.parametrize("variant,transb,precision", [("a", "N", "fp64"), ("b", "T", "fp64"),
                                                      ("a", "T", "ozaki"), ("b", "N", "ozaki")])
def test_tall_skinny_full(variant, transb, precision):
    w = synth.workload_tall_skinny(variant=variant, transb=transb)
    got, st = run(w, "auto", precision)
    assert st["path"] == dbcsr.PATH_DENSE
    freivalds(w, got, 1e-13 if precision == "fp64" else 1e-12)


def test_uneven_4000_fp64_stacks():
    w = synth.workload_uneven()
    got, st = run(w, "auto", "fp64")
    assert st["path"] == dbcsr.PATH_STACKS
    rows = sample_rows(4000, 24, seed=2)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows)
    check_rows(got, ref, w.A, w.B, 1e-13)


def test_uneven_4000_emulated_stacks():
    w = synth.workload_uneven()
    got, st = run(w, "stacks", "ozaki")
    rows = sample_rows(4000, 24, seed=3)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows, mode=1)
    check_rows(got, ref, w.A, w.B, 1e-12)


@pytest.mark.parametrize("precision,tol", [("ozaki", 1e-12), ("fp64", 1e-13), ("tf32", 1e-2)])
def test_precision_dense_N16384(precision, tol):
    w = synth.workload_precision_dense()
    got, st = run(w, "dense", precision)
    rows = sample_rows(512, 2, seed=4)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows, mode=1)
    check_rows(got, ref, w.A, w.B, tol)


def test_precision_sparse_1024_emulated_stacks():
    w = synth.workload_precision_sparse()
    got, st = run(w, "stacks", "ozaki")
    assert st["path"] == dbcsr.PATH_STACKS
    rows = sample_rows(1024, 8, seed=5)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows, mode=1)
    check_rows(got, ref, w.A, w.B, 1e-12)
