"""GPU parity of the emulated-FP64 path at the edges of its arithmetic.

* Non-finite inputs: a row of op(A) or a column of op(B) holding a NaN or an
  infinity has no finite maximum to scale by, so every C element of that row
  or column is NaN (where IEEE FP64 gives a NaN or an infinity); every other
  element is unchanged, and a NaN in the old C propagates where beta reads it.
* Results below the normal range: the exact level sum times its power of two
  is rounded once, at the bit of weight 2^-1074 (no second rounding), and
  results beyond the largest double are infinities.

Each case runs on the dense path with 128-wide tiles (N < 256, densified
operands), on the fused 256-wide path (fully occupied operands, N >= 256), and
on both stack kernels, and must equal the oracle's emulation bit for bit
(NaN positions equal, every other value identical).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import synth

from gpu_util import assert_same_pattern, gpu_multiply

pytestmark = pytest.mark.gpu


def poison(M, b, value):
    """Write value into element (min(3, m-1), min(1, n-1)) of stored block b of M."""
    rs, cs = np.asarray(M.row_sizes, np.int64), np.asarray(M.col_sizes, np.int64)
    sizes = rs[M.blk_row] * cs[M.blk_col]
    off = int(np.sum(sizes[:b]))
    m, n = int(rs[M.blk_row[b]]), int(cs[M.blk_col[b]])
    M.data[off + min(3, m - 1) + min(1, n - 1) * m] = value


def emul_ref(A, B, Cm, alpha, beta, s=7):
    Ad, Bd = O.densify(A), O.densify(B)
    pat = O.multiply("N", "N", 1.0, A, B, beta, Cm)
    Cd = O.densify(Cm) if Cm is not None else np.zeros((Ad.shape[0], Bd.shape[1]), order="F")
    O.ozaki_gemm(alpha, Ad, Bd, beta if Cm is not None else 0.0, Cd, s=s)
    data = O.undensify(Cd, pat.row_sizes, pat.col_sizes, pat.blk_row, pat.blk_col)
    return synth.BlockSparse(pat.row_sizes, pat.col_sizes, pat.blk_row, pat.blk_col, data)


def assert_identical(got, ref):
    assert_same_pattern(got, ref)
    g, r = np.asarray(got.data), np.asarray(ref.data)
    assert np.array_equal(np.isnan(g), np.isnan(r))
    keep = ~np.isnan(r)
    assert np.array_equal(g[keep].view(np.uint64), r[keep].view(np.uint64))


# (path, kernel, C block columns): 128-wide dense tiles, fused 256-wide dense
# path, mma.sync stacks, tcgen05 stacks
RUNS = [("dense", 0, 6), ("dense", 0, 13), ("stacks", 1, 6), ("stacks", 2, 6)]


def operands(seed, ncols, full):
    rng = np.random.default_rng(seed)
    if full:
        A = synth.dense_matrix(rng, 5, 7, 22, 22)
        B = synth.dense_matrix(rng, 7, ncols, 22, 22)
        Cm = synth.dense_matrix(rng, 5, ncols, 22, 22)
    else:
        A, B, Cm = synth.random_small(rng, 5, 7, ncols, p=0.6, sizes=(13, 22, 32), with_c=True, c_p=0.5)
    return A, B, Cm


@pytest.mark.parametrize("path,kernel,ncols", RUNS)
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_rows_and_columns(path, kernel, ncols, bad):
    A, B, Cm = operands(900, ncols, full=path == "dense")
    poison(A, A.nblks // 2, bad)                            # one row of A
    poison(B, B.nblks // 3, bad)                            # one column of B
    Cm.data[5] = np.nan                                     # an old NaN, read only when beta != 0
    for alpha, beta in ((1.0, 0.0), (-0.5, 2.0)):
        got, _ = gpu_multiply("N", "N", alpha, A, B, beta, Cm, path=path, precision="ozaki", kernel=kernel)
        ref = emul_ref(A, B, Cm, alpha, beta)
        assert_identical(got, ref)
        assert np.isnan(ref.data).any()


@pytest.mark.parametrize("path,kernel,ncols", RUNS)
@pytest.mark.parametrize("scale", [-1040, -1062, -1090, 1030])
def test_subnormal_zero_and_overflowing_results(path, kernel, ncols, scale):
    # A scaled by 2^(scale/2), B by 2^(scale/2): results near 2^scale -- in the
    # subnormal range, rounded to zero, or beyond the largest double
    A, B, Cm = operands(910 + abs(scale), ncols, full=path == "dense")
    A.data *= 2.0 ** (scale // 2)
    B.data *= 2.0 ** (scale - scale // 2)
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path=path, precision="ozaki", kernel=kernel)
    ref = emul_ref(A, B, None, 1.0, 0.0)
    assert_identical(got, ref)
    r = np.asarray(ref.data)
    if -1074 < scale < -1022:
        assert np.any((r != 0) & (np.abs(r) < 2.0 ** -1022))
    if scale > 1024:
        assert np.any(np.isinf(r))
