"""GPU parity of the single-precision stack path (the paper's library
accepts single precision, Sec. II): inputs rounded to FP32, FP32 products and
sums, alpha/beta in FP64.

The GPU fuses each product and sum (FMA) where the oracle rounds twice, so
the two FP32 results differ within the classical error bound of an FP32 dot
product: each is within gamma_K |A||B| of the exact product, so their
difference is within 2 gamma_K ||A||_F ||B||_F normwise (K the inner
dimension, gamma_K = K u / (1 - K u), u = 2^-24). Small-integer inputs, whose
sums are exact in FP32, must agree bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import gpu_multiply, assert_same_pattern, normwise

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def _gamma(K):
    return K * U / (1 - K * U)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_fp32_uneven_transposes_beta(ta, tb):
    rng = np.random.default_rng(900)
    A, B, Cm = synth.random_small(rng, 9, 8, 10, p=0.4, sizes=(5, 13, 23, 26, 32), with_c=True, c_p=0.4)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, st = gpu_multiply(ta, tb, 0.5, As, Bs, 2.0, Cm, path="stacks", precision="fp32")
    ref = O.multiply(ta, tb, 0.5, As, Bs, 2.0, Cm, mode=2)
    assert_same_pattern(got, ref)
    K = int(np.sum(A.col_sizes if ta == "N" else A.row_sizes))
    # alpha and beta scale both sides alike; the old-C term is identical FP64
    assert normwise(got, ref, As, Bs) <= 2 * 0.5 * _gamma(K) + 1e-15
    assert st["precision"] == dbcsr.PREC_FP32 and st["path"] == dbcsr.PATH_STACKS


def test_fp32_small_integers_bit_exact():
    rng = np.random.default_rng(901)
    A, B, _ = synth.random_small(rng, 8, 7, 9, p=0.5, sizes=(4, 9, 17, 32), dist="int")
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="stacks", precision="fp32")
    assert np.array_equal(got.data, O.multiply("N", "N", 1.0, A, B, 0.0, mode=2).data)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
def test_fp32_long_product_lists_every_class_bit_exact(ta, tb):
    # C blocks of every patch class (edges 5, 13 and 32, padded to 8, 16 and 32)
    # with about 50 products each: the products' operand offsets are read 32 at
    # a time and the staging ring runs 2 to 6 stages deep. Small integers: the
    # FP32 sums are exact, so any order of them gives the oracle's bits.
    rng = np.random.default_rng(905)
    A, B, Cm = synth.random_small(rng, 9, 72, 9, p=0.7, sizes=(5, 13, 32), dist="int", with_c=True, c_p=0.6)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, _ = gpu_multiply(ta, tb, 1.0, As, Bs, 1.0, Cm, path="stacks", precision="fp32")
    ref = O.multiply(ta, tb, 1.0, As, Bs, 1.0, Cm, mode=2)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)


def test_fp32_larger_grid_and_error_vs_fp64():
    w = synth.workload_small_sparse(0)
    got, _ = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks", precision="fp32")
    ref32 = O.multiply("N", "N", 1.0, w.A, w.B, 0.0, mode=2)
    ref64 = O.multiply("N", "N", 1.0, w.A, w.B, 0.0)
    K = int(np.sum(w.A.col_sizes))
    assert normwise(got, ref32, w.A, w.B) <= 2 * _gamma(K)
    err64 = normwise(got, ref64, w.A, w.B)
    assert 1e-12 < err64 < 1e-5      # single precision, not double


def test_fp32_dense_path_rejected():
    rng = np.random.default_rng(902)
    A, B, _ = synth.random_small(rng, 3, 3, 3, p=1.0, sizes=(8,))
    with pytest.raises(dbcsr.DbcsrError) as e:
        gpu_multiply("N", "N", 1.0, A, B, 0.0, path="dense", precision="fp32")
    assert e.value.code == dbcsr.ERR_ARG
    # automatic path choice keeps FP32 on the stacks even for full operands
    got, st = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="auto", precision="fp32")
    assert st["path"] == dbcsr.PATH_STACKS


def test_fp32_blocks_larger_than_32_use_the_generic_kernel():
    rng = np.random.default_rng(903)
    A, B, Cm = synth.random_small(rng, 4, 5, 3, p=0.7, sizes=(20, 40, 48), with_c=True, c_p=0.5)
    got, _ = gpu_multiply("N", "T", 1.0, A, synth.transpose_blocks(B), 0.5, Cm, path="stacks", precision="fp32")
    ref = O.multiply("N", "N", 1.0, A, B, 0.5, Cm, mode=2)
    assert_same_pattern(got, ref)
    K = int(np.sum(A.col_sizes))
    assert normwise(got, ref, A, B) <= 2 * _gamma(K) + 1e-15
