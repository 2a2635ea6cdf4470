"""GPU parity of every FP64 stack-kernel variant and of the per-shape tuning
table (mixed variants in one multiply), plus the autotuner's table round trip.
"""
import json

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import autotune, dbcsr, synth

from gpu_util import assert_same_pattern, gpu_multiply, setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", [1, 2, 3, 4])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
def test_forced_variants(kernel, ta, tb):
    rng = np.random.default_rng(800 + kernel)
    A, B, Cm = synth.random_small(rng, 10, 9, 8, p=0.5, sizes=(5, 13, 23, 32, 45), dist="int", with_c=True)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, _ = gpu_multiply(ta, tb, 1.0, As, Bs, 1.0, Cm, path="stacks", kernel=kernel)
    ref = O.multiply(ta, tb, 1.0, As, Bs, 1.0, Cm)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)
    A2, B2, _ = synth.random_small(rng, 10, 9, 8, p=0.5, sizes=(5, 13, 23, 32))
    got, _ = gpu_multiply("N", "N", 1.0, A2, B2, 0.0, path="stacks", kernel=kernel)
    ref = O.multiply("N", "N", 1.0, A2, B2, 0.0)
    assert O.normwise_error(O.densify(got), O.densify(ref), O.densify(A2), O.densify(B2)) <= 1e-13


def test_mixed_variant_table():
    setup()
    sizes = (5, 13, 23, 26, 32)
    table = [(m, n, (m * 7 + n) % 4) for m in sizes for n in sizes]
    dbcsr.set_tuning(table)
    try:
        w = synth.workload_uneven(seed=3, nblk=150, occ=0.05, width=15)
        got, _ = gpu_multiply("N", "N", 1.0, w.A, w.B, 0.0, path="stacks")
        ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0)
        assert_same_pattern(got, ref)
        assert O.normwise_error(O.densify(got), O.densify(ref), O.densify(w.A), O.densify(w.B)) <= 1e-13
    finally:
        dbcsr.set_tuning([])


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
def test_mixed_variant_table_integer_exact(ta, tb):
    # teams of 1, 2 and 4 warps in the same launch (the group sizes are read on
    # the device), blocks above 16 elements per lane in several passes:
    # integer-valued inputs make every order of the sums exact
    setup()
    sizes = (5, 13, 23, 26, 32, 45)
    table = [(m, n, (m + 3 * n) % 4) for m in sizes for n in sizes]
    dbcsr.set_tuning(table)
    try:
        rng = np.random.default_rng(821)
        A, B, Cm = synth.random_small(rng, 14, 30, 13, p=0.6, sizes=sizes, dist="int", with_c=True)
        As = synth.transpose_blocks(A) if ta == "T" else A
        Bs = synth.transpose_blocks(B) if tb == "T" else B
        got, _ = gpu_multiply(ta, tb, 2.0, As, Bs, -1.0, Cm, path="stacks")
        ref = O.multiply(ta, tb, 2.0, As, Bs, -1.0, Cm)
        assert_same_pattern(got, ref)
        assert np.array_equal(got.data, ref.data)
    finally:
        dbcsr.set_tuning([])


def test_autotune_shape_and_table_roundtrip(tmp_path):
    setup()
    best, res = autotune.tune_shape(13, 22, (5, 13), reps=1)
    assert best in res and all(v > 0 for v in res.values())
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"device": "x", "entries": [[13, 22, best, res[best], {}]]}))
    assert autotune.load_table(str(p))
    dbcsr.set_tuning([])
