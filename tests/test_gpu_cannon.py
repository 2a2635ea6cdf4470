"""The distributed schemes' local product on the GPU (one rank, no exchange):
gpu_local_mm accumulates panel products through the C ABI. Parity with the
oracle within 1e-13 (normwise), same pattern."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import cannon, synth

from gpu_util import setup

pytestmark = pytest.mark.gpu


def test_gpu_local_mm_accumulates():
    setup()
    rng = np.random.default_rng(1200)
    A, B, _ = synth.random_small(rng, 7, 9, 6, p=0.4, sizes=(5, 13, 23))
    # two inner panels multiplied in turn into one C, as a Cannon rank does
    k = cannon.split_ranges(len(A.col_sizes), 2)
    rows, cols = (0, len(A.row_sizes)), (0, len(B.col_sizes))
    C = cannon.gpu_local_mm(cannon.sub_panel(A, rows, k[0]), cannon.sub_panel(B, k[0], cols), None)
    C = cannon.gpu_local_mm(cannon.sub_panel(A, rows, k[1]), cannon.sub_panel(B, k[1], cols), C)
    ref = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert np.array_equal(C.blk_row, ref.blk_row) and np.array_equal(C.blk_col, ref.blk_col)
    assert O.normwise_error(O.densify(C), O.densify(ref), O.densify(A), O.densify(B)) <= 1e-13


def test_cannon_single_rank_on_gpu():
    setup()
    rng = np.random.default_rng(1201)
    A, B, _ = synth.random_small(rng, 6, 8, 5, p=0.5, sizes=(4, 9, 32))
    C, (r0, c0) = cannon.cannon_multiply(A, B, 0, 1)
    ref = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert (r0, c0) == (0, 0)
    assert O.normwise_error(O.densify(C), O.densify(ref), O.densify(A), O.densify(B)) <= 1e-13
