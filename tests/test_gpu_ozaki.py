"""GPU parity of the emulated-FP64 (7-bit integer slices on the tensor cores) path.

Two bars: bit-exact against the oracle's step-by-step emulation (the slices
and level sums are exact integers and the FP64 recombination order is fixed),
and <= 1e-12 normwise against the plain FP64 oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import gpu_multiply, assert_same_pattern

pytestmark = pytest.mark.gpu


def ozaki_ref(A, B, Cm, alpha, beta, s):
    """Oracle: densify, emulated GEMM, keep the blocks of the result pattern."""
    Ad, Bd = O.densify(A), O.densify(B)
    Cd = O.densify(Cm) if Cm is not None else np.zeros((Ad.shape[0], Bd.shape[1]), order="F")
    O.ozaki_gemm(alpha, Ad, Bd, beta if Cm is not None else 0.0, Cd, s=s)
    pat = O.multiply("N", "N", 1.0, A, B, beta, Cm)
    data = O.undensify(Cd, pat.row_sizes, pat.col_sizes, pat.blk_row, pat.blk_col)
    return synth.BlockSparse(pat.row_sizes, pat.col_sizes, pat.blk_row, pat.blk_col, data), Ad, Bd


@pytest.mark.parametrize("nb,nk,bs,s", [(6, 5, 22, 7), (3, 3, 32, 3), (11, 9, 13, 7), (13, 12, 22, 8), (2, 2, 5, 1)])
def test_dense_ozaki_bit_exact_vs_oracle_emulation(nb, nk, bs, s):
    rng = np.random.default_rng(400 + nb)
    A = synth.dense_matrix(rng, nb, nk, bs, bs)
    B = synth.dense_matrix(rng, nk, nb + 1, bs, bs)
    Cm = synth.dense_matrix(rng, nb, nb + 1, bs, bs)
    got, st = gpu_multiply("N", "N", 0.75, A, B, 1.5, Cm, path="dense", precision="ozaki", ozaki_slices=s)
    ref, _, _ = ozaki_ref(A, B, Cm, 0.75, 1.5, s)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)
    assert st["precision"] == dbcsr.PREC_OZAKI


def test_dense_ozaki_two_k_segments_and_ragged():
    # K = 17'000 > 16'384 (two exact int32 segments), M, N not multiples of 128
    rng = np.random.default_rng(410)
    A = synth.dense_matrix(rng, 1, 1000, 130, 17)
    B = synth.dense_matrix(rng, 1000, 1, 17, 70)
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="dense", precision="ozaki")
    ref, Ad, Bd = ozaki_ref(A, B, None, 1.0, 0.0, 7)
    assert np.array_equal(got.data, ref.data)


@pytest.mark.parametrize("dist", ["uniform", "wide"])
def test_dense_ozaki_meets_1e12_vs_fp64_oracle(dist):
    rng = np.random.default_rng(420)
    A = synth.dense_matrix(rng, 12, 14, 32, 32, dist=dist, scale_exp=4.0)
    B = synth.dense_matrix(rng, 14, 10, 32, 32, dist=dist, scale_exp=4.0)
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="dense", precision="ozaki")
    ref = O.multiply("N", "N", 1.0, A, B, 0.0)
    err = O.normwise_error(O.densify(got), O.densify(ref), O.densify(A), O.densify(B))
    assert err <= 1e-12


def test_integer_inputs_exact_ozaki():
    rng = np.random.default_rng(430)
    A = synth.make_matrix(rng, np.full(7, 13), np.full(6, 13),
                          blocks=(np.repeat(np.arange(7), 6), np.tile(np.arange(6), 7)), dist="int")
    B = synth.make_matrix(rng, np.full(6, 13), np.full(5, 13),
                          blocks=(np.repeat(np.arange(6), 5), np.tile(np.arange(5), 6)), dist="int")
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="dense", precision="ozaki", ozaki_slices=2)
    ref = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert np.array_equal(got.data, ref.data)


@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "T"), ("T", "T")])
def test_ozaki_transposes(ta, tb):
    rng = np.random.default_rng(440)
    A = synth.dense_matrix(rng, 5, 7, 22, 22)
    B = synth.dense_matrix(rng, 7, 4, 22, 22)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, _ = gpu_multiply(ta, tb, 1.0, As, Bs, 0.0, path="dense", precision="ozaki")
    ref, _, _ = ozaki_ref(A, B, None, 1.0, 0.0, 7)
    assert np.array_equal(got.data, ref.data)


def test_ozaki_on_sparse_operands_forced_dense():
    rng = np.random.default_rng(450)
    A, B, Cm = synth.random_small(rng, 9, 7, 8, p=0.4, sizes=(5, 13, 22), with_c=True)
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 1.0, Cm, path="dense", precision="ozaki")
    ref = O.multiply("N", "N", 1.0, A, B, 1.0, Cm)
    assert_same_pattern(got, ref)
    err = O.normwise_error(O.densify(got), O.densify(ref), O.densify(A), O.densify(B))
    assert err <= 1e-12


def test_ozaki_error_decreases_with_slices():
    rng = np.random.default_rng(460)
    A = synth.dense_matrix(rng, 8, 8, 32, 32, dist="wide", scale_exp=4.0)
    B = synth.dense_matrix(rng, 8, 8, 32, 32, dist="wide", scale_exp=4.0)
    ref = O.multiply("N", "N", 1.0, A, B, 0.0, mode=1)
    errs = []
    for s in range(2, 9):
        got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="dense", precision="ozaki", ozaki_slices=s)
        errs.append(O.normwise_error(O.densify(got), O.densify(ref), O.densify(A), O.densify(B)))
    assert all(errs[q + 1] <= errs[q] * 1.0001 + 1e-17 for q in range(len(errs) - 1))


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_fused_block_path_transposes_beta(ta, tb):
    # fully occupied operands with N >= 256: slices are cut straight from the
    # blocks and the result is recombined into C's blocks in place (beta != 0)
    rng = np.random.default_rng(470)
    A = synth.dense_matrix(rng, 6, 7, 22, 22)
    B = synth.dense_matrix(rng, 7, 13, 22, 22)      # N = 286
    Cm = synth.dense_matrix(rng, 6, 13, 22, 22)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, _ = gpu_multiply(ta, tb, -0.5, As, Bs, 2.0, Cm, path="dense", precision="ozaki")
    ref, _, _ = ozaki_ref(A, B, Cm, -0.5, 2.0, 7)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)


def test_fused_block_path_uneven_sizes_partial_old_c():
    # uneven block sizes (odd offsets: single bf16 stores); an old C that is not
    # fully occupied with beta != 0 takes the densifying path instead
    rng = np.random.default_rng(471)
    rs = np.array([5, 13, 23, 26, 32, 7], np.int32)
    ks = np.array([13, 23, 5, 32, 26], np.int32)
    cs = np.array([26, 32, 13, 23, 5, 32, 26, 32, 13, 23, 32, 26], np.int32)   # N = 303
    A = synth.make_matrix(rng, rs, ks, np.ones((6, 5), bool))
    B = synth.make_matrix(rng, ks, cs, np.ones((5, 12), bool))
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="dense", precision="ozaki")
    ref, _, _ = ozaki_ref(A, B, None, 1.0, 0.0, 7)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)
    Cm = synth.make_matrix(rng, rs, cs, synth.bernoulli_mask(rng, 6, 12, 0.5))
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.5, Cm, path="dense", precision="ozaki")
    ref, _, _ = ozaki_ref(A, B, Cm, 1.0, 0.5, 7)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)


# CTA-pair slice GEMM (kernel=4: 256 x 256 tiles, M and N >= 256) against the
# default one-CTA 128 x 256 kernel and the oracle: ragged M, N, K; several tile rows
# and columns; two exact-int32 K segments; fully occupied operands take the
# fused block path, sparse ones the densified one
@pytest.mark.parametrize("nbr,nbk,nbc,bsr,bsk,bsc", [(13, 9, 25, 22, 22, 22), (30, 40, 20, 22, 22, 22),
                                                     (17, 1000, 19, 16, 17, 15), (8, 3, 16, 32, 5, 32)])
def test_pair_tiles_bit_exact(nbr, nbk, nbc, bsr, bsk, bsc):
    rng = np.random.default_rng(480 + nbk)
    A = synth.dense_matrix(rng, nbr, nbk, bsr, bsk, dist="wide", scale_exp=2.0)
    B = synth.dense_matrix(rng, nbk, nbc, bsk, bsc)
    Cm = synth.dense_matrix(rng, nbr, nbc, bsr, bsc)
    assert nbr * bsr >= 256 and nbc * bsc >= 256
    ref, _, _ = ozaki_ref(A, B, Cm, 1.25, -0.5, 7)
    got, _ = gpu_multiply("N", "N", 1.25, A, B, -0.5, Cm, path="dense", precision="ozaki", kernel=4)
    one, _ = gpu_multiply("N", "N", 1.25, A, B, -0.5, Cm, path="dense", precision="ozaki")
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)
    assert np.array_equal(one.data, ref.data)


@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "T"), ("T", "T")])
def test_pair_tiles_transposes_and_sparse_forced_dense(ta, tb):
    rng = np.random.default_rng(490)
    A, B, Cm = synth.random_small(rng, 14, 11, 15, p=0.5, sizes=(13, 22, 32), with_c=True, c_p=0.6)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, _ = gpu_multiply(ta, tb, 1.0, As, Bs, 1.0, Cm, path="dense", precision="ozaki", ozaki_slices=6, kernel=4)
    ref, _, _ = ozaki_ref(A, B, Cm, 1.0, 1.0, 6)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)
