"""GPU parity of the stack path in emulated FP64 (batched slice products on
the tensor cores, no densification).

The level sums are exact integers, so the result must equal, bit for bit, the
oracle's emulation of the densified operands; and it must meet 1e-12 against
the plain FP64 oracle.
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


@pytest.mark.parametrize("s", [7, 3, 8])
def test_precision_sparse_small_bit_exact(s):
    w = synth.workload_precision_sparse(seed=5, nblk=24, occ=0.15)
    got, st = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks", precision="ozaki", ozaki_slices=s)
    ref, Ad, Bd = emul_ref("N", "N", w.A, w.B, None, 1.0, 0.0, s)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)
    assert st["path"] == dbcsr.PATH_STACKS


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_uneven_blocks_transposes_beta(ta, tb):
    rng = np.random.default_rng(600)
    A, B, Cm = synth.random_small(rng, 9, 8, 10, p=0.4, sizes=(5, 13, 23, 26, 32), with_c=True, c_p=0.4)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, _ = gpu_multiply(ta, tb, 0.5, As, Bs, 2.0, Cm, path="stacks", precision="ozaki")
    ref, _, _ = emul_ref(ta, tb, As, Bs, Cm, 0.5, 2.0, 7)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)


def test_emulated_stacks_meet_1e12_and_integer_exact():
    w = synth.workload_precision_sparse(seed=6, nblk=20, occ=0.2)
    got, _ = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks", precision="ozaki")
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0)
    err = O.normwise_error(O.densify(got), O.densify(ref), O.densify(w.A), O.densify(w.B))
    assert err <= 1e-12
    rng = np.random.default_rng(610)
    A, B, _ = synth.random_small(rng, 6, 6, 6, p=0.5, sizes=(5, 13, 32), dist="int")
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="stacks", precision="ozaki", ozaki_slices=2)
    assert np.array_equal(got.data, O.multiply("N", "N", 1.0, A, B, 0.0).data)


def test_emulated_stacks_reject_large_blocks():
    rng = np.random.default_rng(620)
    A, B, _ = synth.random_small(rng, 3, 3, 3, p=1.0, sizes=(40,))
    with pytest.raises(dbcsr.DbcsrError) as e:
        gpu_multiply("N", "N", 1.0, A, B, 0.0, path="stacks", precision="ozaki")
    assert e.value.code == dbcsr.ERR_ARG
