"""GPU parity of the stack path in emulated FP64 (batched slice products on
the tensor cores, no densification).

The level sums are exact integers, so the result must equal, bit for bit, the
oracle's emulation of the densified operands; and it must meet 1e-12 against
the plain FP64 oracle. Both kernels are checked: kernel=1 (mma.sync, blocks
padded to 16) and kernel=2 (tcgen05 with TMEM accumulators, blocks padded to
32 x 32, products in chunks of 32 per C block).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import gpu_multiply, assert_same_pattern

pytestmark = pytest.mark.gpu


def emul_ref(ta, tb, A, B, Cm, alpha, beta, s):
    Aop = synth.transpose_blocks(A) if ta == "T" else A
    Bop = synth.transpose_blocks(B) if tb == "T" else B
    Ad, Bd = O.densify(Aop), O.densify(Bop)
    pat = O.multiply(ta, tb, 1.0, A, B, beta, Cm)
    Cd = O.densify(Cm) if Cm is not None else np.zeros((Ad.shape[0], Bd.shape[1]), order="F")
    O.ozaki_gemm(alpha, Ad, Bd, beta if Cm is not None else 0.0, Cd, s=s)
    data = O.undensify(Cd, pat.row_sizes, pat.col_sizes, pat.blk_row, pat.blk_col)
    return synth.BlockSparse(pat.row_sizes, pat.col_sizes, pat.blk_row, pat.blk_col, data), Ad, Bd


KERNELS = [1, 2]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("s", [7, 3, 8, 1, 5])
def test_precision_sparse_small_bit_exact(s, kernel):
    w = synth.workload_precision_sparse(seed=5, nblk=24, occ=0.15)
    got, st = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks", precision="ozaki", ozaki_slices=s,
                           kernel=kernel)
    ref, Ad, Bd = emul_ref("N", "N", w.A, w.B, None, 1.0, 0.0, s)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)
    assert st["path"] == dbcsr.PATH_STACKS


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_uneven_blocks_transposes_beta(ta, tb, kernel):
    rng = np.random.default_rng(600)
    A, B, Cm = synth.random_small(rng, 9, 8, 10, p=0.4, sizes=(5, 13, 23, 26, 32), with_c=True, c_p=0.4)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, _ = gpu_multiply(ta, tb, 0.5, As, Bs, 2.0, Cm, path="stacks", precision="ozaki", kernel=kernel)
    ref, _, _ = emul_ref(ta, tb, As, Bs, Cm, 0.5, 2.0, 7)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("nk", [32, 33, 70])
def test_long_product_lists_chunked(nk, kernel):
    # one C block row x one C block column, nk products per C block: the
    # tcgen05 kernel's fp32 accumulators are flushed every 16 products
    rng = np.random.default_rng(630 + nk)
    A, B, Cm = synth.random_small(rng, 2, nk, 3, p=1.0, sizes=(32,), dist="wide", with_c=True, c_p=1.0)
    got, _ = gpu_multiply("N", "N", -1.5, A, B, 0.25, Cm, path="stacks", precision="ozaki", kernel=kernel)
    ref, _, _ = emul_ref("N", "N", A, B, Cm, -1.5, 0.25, 7)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)


@pytest.mark.parametrize("s", [8, 5, 4])
def test_long_product_lists_every_segment_count(s):
    # 23 products per C block: several exact fp32 stretches (16 products with
    # one or two operand segments, 10 with three at s = 8) alternating between
    # the two TMEM accumulators, on the tcgen05 kernel; wide-range values
    rng = np.random.default_rng(640 + s)
    A, B, Cm = synth.random_small(rng, 2, 23, 3, p=1.0, sizes=(32, 29), dist="wide", with_c=True, c_p=1.0)
    got, _ = gpu_multiply("N", "T", 0.75, A, synth.transpose_blocks(B), -2.0, Cm, path="stacks",
                          precision="ozaki", ozaki_slices=s, kernel=2)
    ref, _, _ = emul_ref("N", "N", A, B, Cm, 0.75, -2.0, s)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)


def test_auto_kernel_choice_matches_both():
    # 32 x 32 blocks pick the tcgen05 kernel, mixed small blocks the mma.sync one;
    # both agree bit for bit with each other
    w = synth.workload_precision_sparse(seed=7, nblk=16, occ=0.2)
    g0, _ = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks", precision="ozaki", kernel=0)
    g1, _ = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks", precision="ozaki", kernel=1)
    g2, _ = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks", precision="ozaki", kernel=2)
    assert np.array_equal(g0.data, g1.data) and np.array_equal(g1.data, g2.data)


@pytest.mark.parametrize("kernel", KERNELS)
def test_emulated_stacks_meet_1e12_and_integer_exact(kernel):
    w = synth.workload_precision_sparse(seed=6, nblk=20, occ=0.2)
    got, _ = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks", precision="ozaki", kernel=kernel)
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0)
    err = O.normwise_error(O.densify(got), O.densify(ref), O.densify(w.A), O.densify(w.B))
    assert err <= 1e-12
    rng = np.random.default_rng(610)
    A, B, _ = synth.random_small(rng, 6, 6, 6, p=0.5, sizes=(5, 13, 32), dist="int")
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="stacks", precision="ozaki", ozaki_slices=2,
                          kernel=kernel)
    assert np.array_equal(got.data, O.multiply("N", "N", 1.0, A, B, 0.0).data)


def test_emulated_stacks_reject_large_blocks():
    rng = np.random.default_rng(620)
    A, B, _ = synth.random_small(rng, 3, 3, 3, p=1.0, sizes=(40,))
    with pytest.raises(dbcsr.DbcsrError) as e:
        gpu_multiply("N", "N", 1.0, A, B, 0.0, path="stacks", precision="ozaki")
    assert e.value.code == dbcsr.ERR_ARG


@pytest.mark.parametrize("kernel", KERNELS)
def test_rounding_ties_to_even(kernel):
    # dot products 2^53 + odd and 2^54 + 2 mod 4: halfway between two doubles;
    # the exact integer sum is rounded once, to even. Every operand bit lies in
    # slices 1 and 4 (7 slices of 7 bits below the row / column maximum), so
    # no slice pair is truncated and the emulation is the exact dot product.
    from fractions import Fraction
    a_rows = [(2.0 ** 27, 1.0), (2.0 ** 27, 3.0), (-(2.0 ** 27), 1.0), (2.0 ** 28, 2.0)]
    b_cols = [(2.0 ** 26, 1.0), (2.0 ** 26, -1.0), (2.0 ** 26, 3.0)]
    Ablk = np.array(a_rows)                    # 4 x 2
    Bblk = np.array(b_cols).T                  # 2 x 3
    one = np.array([0], np.int32)
    A = synth.BlockSparse(np.array([4], np.int32), np.array([2], np.int32), one, one, Ablk.reshape(-1, order="F"))
    B = synth.BlockSparse(np.array([2], np.int32), np.array([3], np.int32), one, one, Bblk.reshape(-1, order="F"))
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="stacks", precision="ozaki", kernel=kernel)
    ref, _, _ = emul_ref("N", "N", A, B, None, 1.0, 0.0, 7)
    assert np.array_equal(got.data, ref.data)
    exact = [[float(sum(Fraction(x) * Fraction(y) for x, y in zip(r, c))) for c in b_cols] for r in a_rows]
    assert np.array_equal(got.data.reshape((4, 3), order="F"), np.array(exact))
