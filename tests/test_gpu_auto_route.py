"""Automatic path choice where the stack kernels do not apply (GPU).

Sec. II sends blocks beyond the small-matrix kernels' range to a GEMM. Under
DBCSR_PATH_AUTO, a sparse multiply in emulated FP64 with a block edge above 32
(the emulated stack kernels' limit), and TF32 on sparse operands (no TF32
stack kernel), take the densified GEMM of Sec. III and return the result on
the symbolic pattern; they are not refused. FP64 keeps the stack kernels,
which take any block size. Fully occupied operands take the densified GEMM
(Sec. III), except FP32 (no FP32 dense path) and FP64 with every block edge up
to 32, which stay on the stack kernels (measured faster there than the FP64
tensor-core GEMM).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import assert_same_pattern, gpu_multiply

pytestmark = pytest.mark.gpu


def emul_ref(A, B, Cm, alpha, beta, s=7):
    Ad, Bd = O.densify(A), O.densify(B)
    pat = O.multiply("N", "N", 1.0, A, B, beta, Cm)
    Cd = O.densify(Cm) if Cm is not None else np.zeros((Ad.shape[0], Bd.shape[1]), order="F")
    O.ozaki_gemm(alpha, Ad, Bd, beta if Cm is not None else 0.0, Cd, s=s)
    data = O.undensify(Cd, pat.row_sizes, pat.col_sizes, pat.blk_row, pat.blk_col)
    return synth.BlockSparse(pat.row_sizes, pat.col_sizes, pat.blk_row, pat.blk_col, data)


@pytest.mark.parametrize("sizes", [(40,), (64,), (13, 40, 22), (5, 64, 32, 48)])
def test_auto_emulated_large_blocks_take_dense(sizes):
    rng = np.random.default_rng(960 + sum(sizes))
    A, B, Cm = synth.random_small(rng, 6, 5, 7, p=0.45, sizes=sizes, with_c=True, c_p=0.4)
    got, st = gpu_multiply("N", "N", 0.5, A, B, 1.5, Cm, path="auto", precision="ozaki")
    assert st["path"] == dbcsr.PATH_DENSE
    ref = emul_ref(A, B, Cm, 0.5, 1.5)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)


@pytest.mark.parametrize("sizes", [(32,), (13, 22, 32)])
def test_auto_emulated_small_blocks_keep_stacks(sizes):
    rng = np.random.default_rng(970 + sum(sizes))
    A, B, _ = synth.random_small(rng, 6, 5, 7, p=0.45, sizes=sizes)
    got, st = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="auto", precision="ozaki")
    assert st["path"] == dbcsr.PATH_STACKS
    assert np.array_equal(got.data, emul_ref(A, B, None, 1.0, 0.0).data)


@pytest.mark.parametrize("sizes", [(40,), (64, 13)])
def test_auto_fp64_large_blocks_stacks(sizes):
    rng = np.random.default_rng(980 + sum(sizes))
    A, B, Cm = synth.random_small(rng, 5, 6, 4, p=0.5, sizes=sizes, with_c=True, c_p=0.5)
    got, st = gpu_multiply("N", "N", 1.0, A, B, -1.0, Cm, path="auto", precision="fp64")
    assert st["path"] == dbcsr.PATH_STACKS
    ref = O.multiply("N", "N", 1.0, A, B, -1.0, Cm)
    assert_same_pattern(got, ref)
    err = O.normwise_error(O.densify(got), O.densify(ref), O.densify(A), O.densify(B))
    assert err <= 1e-13


def test_auto_tf32_sparse_takes_dense():
    rng = np.random.default_rng(990)
    A, B, Cm = synth.random_small(rng, 7, 6, 5, p=0.4, sizes=(13, 22, 32), with_c=True, c_p=0.5)
    got, st = gpu_multiply("N", "N", 1.0, A, B, 0.5, Cm, path="auto", precision="tf32")
    assert st["path"] == dbcsr.PATH_DENSE
    ref = O.multiply("N", "N", 1.0, A, B, 0.5, Cm)
    assert_same_pattern(got, ref)
    Ad, Bd = O.densify(A), O.densify(B)
    # on the result pattern: the product of the TF32-rounded inputs (FP32 accumulation) plus beta * C
    want = O.densify(synth.BlockSparse(ref.row_sizes, ref.col_sizes, ref.blk_row, ref.blk_col,
                                       O.undensify(O.round_tf32(Ad) @ O.round_tf32(Bd) + 0.5 * O.densify(Cm),
                                                   ref.row_sizes, ref.col_sizes, ref.blk_row, ref.blk_col)))
    assert O.normwise_error(O.densify(got), want, Ad, Bd) <= 2e-6


@pytest.mark.parametrize("precision,bs,path", [("fp64", 22, dbcsr.PATH_STACKS), ("fp64", 32, dbcsr.PATH_STACKS),
                                               ("fp64", 33, dbcsr.PATH_DENSE), ("ozaki", 22, dbcsr.PATH_DENSE),
                                               ("tf32", 22, dbcsr.PATH_DENSE)])
def test_auto_fully_occupied(precision, bs, path):
    rng = np.random.default_rng(1000 + bs)
    A = synth.dense_matrix(rng, 6, 5, bs, bs)
    B = synth.dense_matrix(rng, 5, 7, bs, bs)
    Cm = synth.dense_matrix(rng, 6, 7, bs, bs)
    got, st = gpu_multiply("N", "N", 1.0, A, B, 0.5, Cm, path="auto", precision=precision)
    assert st["path"] == path
    if precision == "ozaki":
        ref = emul_ref(A, B, Cm, 1.0, 0.5)
        assert_same_pattern(got, ref)
        assert np.array_equal(got.data, ref.data)
        return
    ref = O.multiply("N", "N", 1.0, A, B, 0.5, Cm)
    assert_same_pattern(got, ref)
    err = O.normwise_error(O.densify(got), O.densify(ref), O.densify(A), O.densify(B))
    assert err <= (1e-13 if precision == "fp64" else 1e-2)
