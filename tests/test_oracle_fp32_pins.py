"""Pins of the oracle's single-precision product (mode 2, CPU only).

The paper's library accepts single-precision matrices (Sec. II). The oracle's
FP32 mode rounds every input element to FP32, forms each product and each
addition in FP32 (k ascending, inner index ascending) and applies alpha and
beta in FP64. Pinned against a pure-Python loop over numpy float32 scalars
(bit-exact), exact integer arithmetic, the classical FP32 error bound of a
dot product, and the FP64 alpha/beta rule.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import synth

F = np.float32


def _loop_fp32(ta, tb, A, B):
    """Brute force: dense op(A), op(B) rounded to FP32, sequential FP32 sums over
    the blocks of op(A)'s row in ascending k, inside a block ascending l."""
    Aop = synth.transpose_blocks(A) if ta == "T" else A
    Bop = synth.transpose_blocks(B) if tb == "T" else B
    Ad, Bd = O.densify(Aop), O.densify(Bop)
    ks = np.asarray(Aop.col_sizes)
    koff = np.concatenate([[0], np.cumsum(ks)])
    M, N = Ad.shape[0], Bd.shape[1]
    out = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            s = F(0.0)
            for kb in range(len(ks)):
                for l in range(koff[kb], koff[kb + 1]):
                    s = F(s + F(F(Ad[i, l]) * F(Bd[l, j])))
            out[i, j] = float(s)
    return out


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
def test_fp32_mode_equals_float32_loop(ta, tb):
    rng = np.random.default_rng(80)
    # dense operands: then every (i, l, j) term is part of the sum and the
    # loop above visits exactly the oracle's terms in the oracle's order
    rs = np.array([3, 2, 4], np.int32)
    ks = np.array([2, 5, 3], np.int32)
    cs = np.array([4, 1, 3], np.int32)
    A = synth.make_matrix(rng, rs, ks, np.ones((3, 3), bool))
    B = synth.make_matrix(rng, ks, cs, np.ones((3, 3), bool))
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got = O.densify(O.multiply(ta, tb, 1.0, As, Bs, 0.0, mode=2))
    assert np.array_equal(got, _loop_fp32(ta, tb, As, Bs))


def test_fp32_mode_rounds_inputs():
    # 1 + 2^-30 rounds to 1 in FP32; the FP64 product keeps it
    rs = np.array([1], np.int32)
    A = synth.BlockSparse(rs, rs, np.array([0], np.int32), np.array([0], np.int32), np.array([1.0 + 2.0 ** -30]))
    B = synth.BlockSparse(rs, rs, np.array([0], np.int32), np.array([0], np.int32), np.array([3.0]))
    assert O.multiply("N", "N", 1.0, A, B, 0.0, mode=2).data[0] == 3.0
    assert O.multiply("N", "N", 1.0, A, B, 0.0, mode=0).data[0] == 3.0 + 3.0 * 2.0 ** -30


def test_fp32_mode_exact_on_small_integers():
    rng = np.random.default_rng(81)
    A, B, _ = synth.random_small(rng, 5, 6, 4, p=0.6, sizes=(3, 7, 11), dist="int")
    assert np.array_equal(O.multiply("N", "N", 1.0, A, B, 0.0, mode=2).data,
                          O.multiply("N", "N", 1.0, A, B, 0.0, mode=0).data)


def test_fp32_mode_within_dot_product_bound():
    rng = np.random.default_rng(82)
    A, B, _ = synth.random_small(rng, 6, 9, 5, p=0.7, sizes=(8, 16, 32))
    c32 = O.densify(O.multiply("N", "N", 1.0, A, B, 0.0, mode=2))
    c64 = O.densify(O.multiply("N", "N", 1.0, A, B, 0.0, mode=1))   # double-double: exact enough
    absab = np.abs(O.densify(A)) @ np.abs(O.densify(B))
    K = O.densify(A).shape[1]
    u = 2.0 ** -24
    # input rounding (2u) plus the recursive sum (K u), first order
    bound = ((K + 2) * u / (1 - (K + 2) * u)) * absab
    assert np.all(np.abs(c32 - c64) <= bound)
    assert np.any(c32 != c64)     # it is single precision, not double


def test_fp32_mode_alpha_beta_in_fp64():
    rng = np.random.default_rng(83)
    A, B, Cm = synth.random_small(rng, 4, 4, 4, p=0.8, sizes=(5, 6), with_c=True, c_p=1.0)
    base = O.multiply("N", "N", 1.0, A, B, 0.0, mode=2)
    full = O.multiply("N", "N", 2.5, A, B, -0.5, Cm, mode=2)
    ref = O.densify(base) * 2.5 + O.densify(Cm) * -0.5
    assert np.array_equal(O.densify(full), ref)
