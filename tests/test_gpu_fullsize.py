"""Parity at the workloads' full sizes, in the configuration bench.py times.

The oracle cannot redo whole products of this size, so each test checks
sampled rows of C, which the oracle computes one by one from the same inputs
with the same definition:

* FP64: sampled C block rows (or element rows on the densified path) against
  the oracle's block product (or its densified GEMM), normwise within 1e-13
  of the sampled rows' own scale: ||C_rows - C_ref,rows||_F divided by
  ||op(A)_rows||_F ||op(B)||_F, the bar of the whole product restricted to
  those rows.
* Emulated FP64: sampled element rows bit for bit against the oracle's
  step-by-step emulation. The emulation of a row depends only on that row of
  op(A) and on all of op(B) (row exponents come from the row itself), so the
  oracle runs on the sampled rows of op(A) against the whole op(B).
* Reported precisions (emulated against the near-exact Dot2 product, TF32)
  within their gates on the same normalisation.
* FP32 (stack path): sampled C block rows against the oracle's FP32 product
  (inputs rounded to FP32, FP32 products and sums), within 2 gamma_K on the
  same normalisation, K the longest inner product of the sampled rows: each
  side is within gamma_K |A||B| of the exact product of the rounded inputs.
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


def element_rows(M, rows):
    """Dense values of the given element rows of a block matrix: (len(rows), total columns)."""
    rs, cs = np.asarray(M.row_sizes, np.int64), np.asarray(M.col_sizes, np.int64)
    ro, co = np.concatenate([[0], np.cumsum(rs)]), np.concatenate([[0], np.cumsum(cs)])
    br, bc = np.asarray(M.blk_row), np.asarray(M.blk_col)
    offs = np.concatenate([[0], np.cumsum(rs[br] * cs[bc])])
    out = np.zeros((len(rows), int(co[-1])))
    for q, r in enumerate(rows):
        bi = int(np.searchsorted(ro, r, "right") - 1)
        m = int(rs[bi])
        for b in np.nonzero(br == bi)[0]:
            j = int(bc[b])
            out[q, co[j]:co[j + 1]] = M.data[offs[b] + (r - ro[bi]) + m * np.arange(cs[j])]
    return out


def blocks_of_rows(M, rows):
    """Sub-list (block index + data) of the blocks in the given block rows, CSR order."""
    rs = np.asarray(M.row_sizes, np.int64)
    cs = np.asarray(M.col_sizes, np.int64)
    sizes = rs[M.blk_row] * cs[M.blk_col]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    keep = np.isin(M.blk_row, rows)
    data = np.concatenate([M.data[offs[b]:offs[b + 1]] for b in np.nonzero(keep)[0]])
    return M.blk_row[keep], M.blk_col[keep], data


def check_block_rows(got, ref, A, B, tol):
    """Sampled C block rows of the block product, normwise against the sampled rows of A."""
    rows = np.unique(ref.blk_row)
    gbr, gbc, gdata = blocks_of_rows(got, rows)
    assert np.array_equal(gbr, ref.blk_row) and np.array_equal(gbc, ref.blk_col)
    _, _, adata = blocks_of_rows(A, rows)
    err = np.linalg.norm(gdata - ref.data) / (np.linalg.norm(adata) * np.linalg.norm(B.data))
    assert err <= tol, err


def op_dense(M, trans):
    D = O.densify(M)
    return np.asfortranarray(D.T) if trans == "T" else D


def sample_rows(n, k, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int32)


def column_maxima(M):
    """max |M(l, j)| over each element column j of a block matrix."""
    rs, cs = np.asarray(M.row_sizes, np.int64), np.asarray(M.col_sizes, np.int64)
    co = np.concatenate([[0], np.cumsum(cs)])
    br, bc = np.asarray(M.blk_row), np.asarray(M.blk_col)
    offs = np.concatenate([[0], np.cumsum(rs[br] * cs[bc])])
    out = np.zeros(int(co[-1]))
    for b in range(len(br)):
        m, n, j = int(rs[br[b]]), int(cs[bc[b]]), int(bc[b])
        blk = np.abs(M.data[offs[b]:offs[b + 1]].reshape((m, n), order="F")).max(axis=0)
        out[co[j]:co[j + 1]] = np.maximum(out[co[j]:co[j + 1]], blk)
    return out


def sparse_subproblem(A, B, elem_rows):
    """The emulation of the sampled rows of A*B (both block-sparse, op = N) as a
    small dense problem with the same result: the sampled rows of A restricted
    to the inner indices where they are nonzero, the same rows of B, and one
    more inner index whose A entries are zero and whose B entries are B's
    column maxima. Zeros add no slices, row exponents come from the rows
    themselves, and the appended row gives every column of B its exponent over
    the whole column."""
    Arows = element_rows(A, elem_rows)
    lsel = np.nonzero(np.any(Arows != 0, axis=0))[0]
    Asub = np.zeros((len(elem_rows), len(lsel) + 1), order="F")
    Asub[:, :-1] = Arows[:, lsel]
    Bsub = np.zeros((len(lsel) + 1, int(np.sum(B.col_sizes))), order="F")
    Bsub[:-1] = element_rows(B, lsel)
    Bsub[-1] = column_maxima(B)
    return Asub, Bsub


def check_emulated_rows(w, got, elem_rows, s=7):
    """Sampled element rows equal the oracle's emulation bit for bit."""
    assert w.transa == "N"
    full_b = w.B.nblks == len(w.B.row_sizes) * len(w.B.col_sizes)
    if full_b:
        Arows = np.asfortranarray(element_rows(w.A, elem_rows))
        Bd = op_dense(w.B, w.transb)
    else:
        assert w.transb == "N"
        Arows, Bd = sparse_subproblem(w.A, w.B, elem_rows)
    Cd = np.asfortranarray(element_rows(w.C, elem_rows)) if (w.C is not None and w.beta != 0.0) else \
        np.zeros((len(elem_rows), Bd.shape[1]), order="F")
    O.ozaki_gemm(w.alpha, Arows, Bd, w.beta if w.C is not None else 0.0, Cd, s=s)
    have = element_rows(got, elem_rows)
    assert np.array_equal(have, Cd), np.abs(have - Cd).max()
    assert np.count_nonzero(Cd) > 0
    return Arows, Bd


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_dense_limit_N11264(precision):
    # emulated FP64 takes the densified GEMM under AUTO; FP64 blocks of 22
    # stay on the stack kernels there, so its dense path is asked for
    w = synth.workload_dense_limit()
    got, st = run(w, "auto" if precision == "ozaki" else "dense", precision)
    assert st["path"] == dbcsr.PATH_DENSE
    if precision == "fp64":
        rows = sample_rows(512, 3, seed=1)
        ref = O.multiply("N", "N", w.alpha, w.A, w.B, w.beta, w.C, rows=rows)
        check_block_rows(got, ref, w.A, w.B, 1e-13)
    else:
        check_emulated_rows(w, got, sample_rows(11264, 6, seed=11))
        rows = sample_rows(512, 2, seed=1)
        ref = O.multiply("N", "N", w.alpha, w.A, w.B, w.beta, w.C, rows=rows, mode=1)
        check_block_rows(got, ref, w.A, w.B, 1e-12)


@pytest.mark.parametrize("variant,transb,precision", [("a", "N", "fp64"), ("b", "T", "fp64"),
                                                      ("a", "T", "ozaki"), ("b", "N", "ozaki")])
def test_tall_skinny_full(variant, transb, precision):
    # (a) K = 131 072: eight exact-int32 K segments of 16 384 on the emulated path
    w = synth.workload_tall_skinny(variant=variant, transb=transb)
    got, st = run(w, "auto" if precision == "ozaki" else "dense", precision)
    assert st["path"] == dbcsr.PATH_DENSE
    M = int(np.sum(w.A.row_sizes))
    erows = sample_rows(M, 3 if variant == "a" else 6, seed=12)
    if precision == "ozaki":
        Arows, Bd = check_emulated_rows(w, got, erows)
        ref = np.zeros((len(erows), Bd.shape[1]), order="F")
        O.dense_gemm("N", "N", 1.0, Arows, Bd, 0.0, ref)
        tol = 1e-12
    else:
        Arows = np.asfortranarray(element_rows(w.A, erows))
        Bd = op_dense(w.B, transb)
        ref = np.zeros((len(erows), Bd.shape[1]), order="F")
        O.dense_gemm("N", "N", 1.0, Arows, Bd, 0.0, ref)
        tol = 1e-13
    err = np.linalg.norm(element_rows(got, erows) - ref) / (np.linalg.norm(Arows) * np.linalg.norm(Bd))
    assert err <= tol, err


def test_uneven_4000_fp64_stacks():
    w = synth.workload_uneven()
    got, st = run(w, "auto", "fp64")
    assert st["path"] == dbcsr.PATH_STACKS
    rows = sample_rows(4000, 24, seed=2)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows)
    check_block_rows(got, ref, w.A, w.B, 1e-13)


def test_uneven_4000_emulated_stacks():
    w = synth.workload_uneven()
    got, st = run(w, "stacks", "ozaki")
    rows = sample_rows(4000, 24, seed=3)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows, mode=1)
    check_block_rows(got, ref, w.A, w.B, 1e-12)
    M = int(np.sum(w.A.row_sizes))
    check_emulated_rows(w, got, sample_rows(M, 8, seed=13))


@pytest.mark.parametrize("precision,tol", [("ozaki", 1e-12), ("fp64", 1e-13), ("tf32", 1e-2)])
def test_precision_dense_N16384(precision, tol):
    w = synth.workload_precision_dense()
    got, st = run(w, "dense", precision)
    if precision == "ozaki":
        check_emulated_rows(w, got, sample_rows(16384, 4, seed=14))
    rows = sample_rows(512, 2, seed=4)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows, mode=1)
    check_block_rows(got, ref, w.A, w.B, tol)


def test_precision_sparse_1024_fp64_stacks():
    # FP64 stack kernels on the 1 024^2 grid of 32 x 32 blocks (two passes of 16 elements per lane)
    w = synth.workload_precision_sparse()
    got, st = run(w, "auto", "fp64")
    assert st["path"] == dbcsr.PATH_STACKS
    rows = sample_rows(1024, 8, seed=8)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows)
    check_block_rows(got, ref, w.A, w.B, 1e-13)


def test_precision_sparse_1024_emulated_stacks():
    w = synth.workload_precision_sparse()
    got, st = run(w, "stacks", "ozaki")
    assert st["path"] == dbcsr.PATH_STACKS
    rows = sample_rows(1024, 8, seed=5)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, rows=rows, mode=1)
    check_block_rows(got, ref, w.A, w.B, 1e-12)
    check_emulated_rows(w, got, sample_rows(32768, 8, seed=15))


def fp32_bar(A, rows):
    """2 gamma_K, K the longest inner product of the given C block rows (u = 2^-24)."""
    cs = np.asarray(A.col_sizes, np.int64)
    K = max(int(np.sum(cs[A.blk_col[A.blk_row == r]])) for r in rows)
    u = 2.0 ** -24
    return 2 * K * u / (1 - K * u)


@pytest.mark.parametrize("name", ["uneven", "precision-sparse", "dense-limit"])
def test_fp32_stacks_full_size(name):
    # the configuration bench.py times with --precision fp32 --path stacks (the
    # dense limit with beta = 1: the old-C term is the same FP64 step on both sides)
    if name == "uneven":
        w, rows = synth.workload_uneven(), sample_rows(4000, 24, seed=6)
    elif name == "precision-sparse":
        w, rows = synth.workload_precision_sparse(), sample_rows(1024, 8, seed=7)
    else:
        w, rows = synth.workload_dense_limit(), sample_rows(512, 3, seed=9)
    got, st = run(w, "stacks", "fp32")
    assert st["path"] == dbcsr.PATH_STACKS and st["precision"] == dbcsr.PREC_FP32
    beta = w.beta if w.C is not None else 0.0
    ref = O.multiply("N", "N", w.alpha, w.A, w.B, beta, w.C, rows=rows, mode=2)
    check_block_rows(got, ref, w.A, w.B, fp32_bar(w.A, rows))
