"""GPU check of the TF32 variant (inputs rounded to TF32, FP32 accumulation).

Its error against FP64 is reported, not bounded by the method; what is pinned
is the input rounding: the GPU result must agree with the exact product of the
TF32-rounded inputs to FP32-accumulation accuracy, and lie within a sanity
band of the FP64 result.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import gpu_multiply, assert_same_pattern

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nb,nk,bs", [(6, 5, 22), (9, 9, 32), (3, 17, 13)])
def test_tf32_matches_rounded_inputs(nb, nk, bs):
    rng = np.random.default_rng(500 + nb)
    A = synth.dense_matrix(rng, nb, nk, bs, bs)
    B = synth.dense_matrix(rng, nk, nb + 1, bs, bs)
    Cm = synth.dense_matrix(rng, nb, nb + 1, bs, bs)
    got, st = gpu_multiply("N", "N", 1.0, A, B, 0.5, Cm, path="dense", precision="tf32")
    assert st["precision"] == dbcsr.PREC_TF32
    Ad, Bd, Cd = O.densify(A), O.densify(B), O.densify(Cm)
    exact_rounded = O.round_tf32(Ad) @ O.round_tf32(Bd) + 0.5 * Cd
    g = O.densify(got)
    e_round = O.normwise_error(g, exact_rounded, Ad, Bd)
    e_fp64 = O.normwise_error(g, Ad @ Bd + 0.5 * Cd, Ad, Bd)
    assert e_round <= 2e-6, e_round
    assert e_fp64 < 1e-2, e_fp64
    ref = O.multiply("N", "N", 1.0, A, B, 0.5, Cm)
    assert_same_pattern(got, ref)


def test_tf32_transposes_and_ragged():
    rng = np.random.default_rng(510)
    A = synth.dense_matrix(rng, 7, 3, 13, 5)       # K = 15: not a multiple of 32
    B = synth.dense_matrix(rng, 3, 11, 5, 13)
    got, _ = gpu_multiply("T", "T", 2.0, synth.transpose_blocks(A), synth.transpose_blocks(B), 0.0,
                          path="dense", precision="tf32")
    Ad, Bd = O.densify(A), O.densify(B)
    e = O.normwise_error(O.densify(got), 2.0 * (O.round_tf32(Ad) @ O.round_tf32(Bd)), Ad, Bd)
    assert e <= 2e-6


@pytest.mark.parametrize("ta,tb,beta", [("N", "N", 0.5), ("T", "N", 0.0), ("N", "T", 1.0), ("T", "T", 2.0)])
def test_tf32_fused_blocks_equal_densified(ta, tb, beta):
    # fully occupied operands of one block size per dimension (N >= 256): the
    # TF32 operands come straight from the blocks and the GEMM writes straight
    # into C's blocks. The same values through the densified path (A without
    # its first block, which is zero in the fused operand: A no longer fully
    # occupied) go through the same TF32 rounding and the same GEMM, so the two
    # results are equal bit for bit.
    rng = np.random.default_rng(520)
    Aop = synth.dense_matrix(rng, 12, 10, 22, 32)
    Bop = synth.dense_matrix(rng, 10, 12, 32, 22)
    Cm = synth.dense_matrix(rng, 12, 12, 22, 22)
    m0, n0 = int(Aop.row_sizes[0]), int(Aop.col_sizes[0])
    data = Aop.data.copy()
    data[:m0 * n0] = 0.0
    Az = synth.BlockSparse(Aop.row_sizes, Aop.col_sizes, Aop.blk_row, Aop.blk_col, data)
    As = synth.BlockSparse(Aop.row_sizes, Aop.col_sizes, Aop.blk_row[1:], Aop.blk_col[1:], data[m0 * n0:])
    store = lambda M, t: synth.transpose_blocks(M) if t == "T" else M
    fused, st = gpu_multiply(ta, tb, 1.5, store(Az, ta), store(Bop, tb), beta, Cm, path="dense", precision="tf32")
    assert st["path"] == dbcsr.PATH_DENSE
    dense, _ = gpu_multiply(ta, tb, 1.5, store(As, ta), store(Bop, tb), beta, Cm, path="dense", precision="tf32")
    assert_same_pattern(fused, dense)
    assert np.array_equal(fused.data, dense.data)
    Ad, Bd = O.densify(Az), O.densify(Bop)
    want = 1.5 * (O.round_tf32(Ad) @ O.round_tf32(Bd)) + beta * O.densify(Cm)
    assert O.normwise_error(O.densify(fused), want, Ad, Bd) <= 2e-6
