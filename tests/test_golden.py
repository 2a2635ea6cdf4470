"""The oracle against hand-worked fixtures (tests/golden/): a stack list
enumerated by hand, a 2 x 2 block product worked by hand, integer slices of
values with known binary expansions, and single-precision products rounded by
hand. The paper prints no numeric example, so
every value here is derived by hand from the definitions it states (Sec. II)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def tiny_operands():
    """The A and B of stack_list_2x2x2.txt (values are irrelevant to the list)."""
    rng = np.random.default_rng(0)
    A = synth.make_matrix(rng, np.array([2, 3], np.int32), np.array([3, 2], np.int32),
                          blocks=(np.array([0, 0, 1], np.int32), np.array([0, 1, 1], np.int32)))
    B = synth.make_matrix(rng, np.array([3, 2], np.int32), np.array([2, 3], np.int32),
                          blocks=(np.array([0, 1, 1], np.int32), np.array([0, 0, 1], np.int32)))
    return A, B


def ones_2x2(vals):
    """2 x 2 grid of 1 x 1 blocks, all stored, row-major values."""
    one = np.ones(2, np.int32)
    return synth.BlockSparse(one, one.copy(), np.array([0, 0, 1, 1], np.int32), np.array([0, 1, 0, 1], np.int32),
                             np.asarray(vals, np.float64))


def test_stack_list_matches_hand_enumeration():
    want = np.array([[int(v) for v in r] for r in rows("stack_list_2x2x2.txt")], np.int32)
    A, B = tiny_operands()
    assert np.array_equal(O.stack_list("N", "N", A, B), want)


@pytest.mark.parametrize("r", rows("block_product_2x2.txt"), ids=lambda r: "".join(r[:4]))
def test_block_product_matches_hand_result(r):
    ta, tb, alpha, beta = r[0], r[1], float(r[2]), float(r[3])
    want = np.array([float(v) for v in r[4:]])
    A, B, C = ones_2x2([1, 2, 3, 4]), ones_2x2([5, 6, 7, 8]), ones_2x2([1, 1, 1, 1])
    got = O.multiply(ta, tb, alpha, A, B, beta, C)
    assert np.array_equal(O.densify(got).reshape(-1), want)


@pytest.mark.parametrize("r", rows("ozaki_slices.txt"), ids=lambda r: f"{r[0]}-{r[1]}")
def test_slices_match_hand_expansion(r):
    x, s = float(r[0]), int(r[1])
    assert O.ozaki_split(x, s) == [int(v) for v in r[2:]]


@pytest.mark.parametrize("r", rows("fp32_rounding.txt"), ids=lambda r: r[0])
def test_single_precision_matches_hand_rounding(r):
    k = int(r[1])
    a = np.array([float.fromhex(x) for x in r[2:2 + k]])
    b = np.array([float.fromhex(x) for x in r[2 + k:2 + 2 * k]])
    c32, c64 = float.fromhex(r[2 + 2 * k]), float.fromhex(r[3 + 2 * k])
    one, kk, z = np.array([1], np.int32), np.array([k], np.int32), np.zeros(1, np.int32)
    A = synth.BlockSparse(one, kk, z, z, a)
    B = synth.BlockSparse(kk, one, z, z, b)
    assert O.multiply("N", "N", 1.0, A, B, 0.0, mode=2).data[0] == c32
    assert O.multiply("N", "N", 1.0, A, B, 0.0, mode=0).data[0] == c64
