"""The GPU path against the hand-worked fixtures of tests/golden/ (through the C ABI)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr

from gpu_util import gpu_multiply, setup, to_gpu
from test_golden import ones_2x2, rows, tiny_operands

pytestmark = pytest.mark.gpu


def test_gpu_stack_list_matches_hand_enumeration():
    setup()
    want = np.array([[int(v) for v in r] for r in rows("stack_list_2x2x2.txt")], np.int32)
    A, B = tiny_operands()
    assert np.array_equal(dbcsr.get_stacks("N", "N", to_gpu(A), to_gpu(B), 30000), want)


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("r", rows("block_product_2x2.txt"), ids=lambda r: "".join(r[:4]))
def test_gpu_block_product_matches_hand_result(r, precision):
    ta, tb, alpha, beta = r[0], r[1], float(r[2]), float(r[3])
    want = np.array([float(v) for v in r[4:]])
    A, B, C = ones_2x2([1, 2, 3, 4]), ones_2x2([5, 6, 7, 8]), ones_2x2([1, 1, 1, 1])
    for path in ("stacks", "dense"):
        got, _ = gpu_multiply(ta, tb, alpha, A, B, beta, C, path=path, precision=precision)
        assert np.array_equal(O.densify(got).reshape(-1), want), (path, precision)
