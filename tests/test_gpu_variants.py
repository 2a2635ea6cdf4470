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


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T")])
def test_mnk_table_overrides_mn_table_integer_exact(ta, tb):
    # the (m, n, k) table picks the team size by the inner size of a C block's
    # first product, over the (m, n) table; teams of 1, 2 and 4 warps mix in one
    # launch. Integer-valued inputs: every order of the sums is exact.
    setup()
    sizes = (5, 13, 23, 26, 32)
    dbcsr.set_tuning([(m, n, 0) for m in sizes for n in sizes])
    dbcsr.set_tuning_mnk([(m, n, k, (m + 2 * n + 3 * k) % 4) for m in sizes for n in sizes for k in sizes])
    try:
        rng = np.random.default_rng(831)
        A, B, Cm = synth.random_small(rng, 14, 30, 13, p=0.6, sizes=sizes, dist="int", with_c=True)
        Bs = synth.transpose_blocks(B) if tb == "T" else B
        got, _ = gpu_multiply(ta, tb, 1.0, A, Bs, 1.0, Cm, path="stacks")
        ref = O.multiply(ta, tb, 1.0, A, Bs, 1.0, Cm)
        assert_same_pattern(got, ref)
        assert np.array_equal(got.data, ref.data)
    finally:
        dbcsr.set_tuning_mnk([])
        dbcsr.set_tuning([])


def test_model_table_loads_both_tables(tmp_path):
    setup()
    E = 32
    mnk = [(m, n, k, (m * n + k) % 4) for m in range(1, E + 1) for n in range(1, E + 1) for k in range(1, E + 1)]
    p = tmp_path / "m.json"
    p.write_text(json.dumps({"device": "x", "entries": [[13, 22, 2, 1.0, {}]],
                             "variants_mnk": {"max_edge": E, "variants": autotune.encode_mnk(mnk, E)}}))
    assert autotune.load_table(path=None, model_path=str(p))
    try:
        rng = np.random.default_rng(832)
        A, B, _ = synth.random_small(rng, 6, 8, 6, p=0.7, sizes=(13, 22, 5), dist="int")
        got, st = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="stacks")
        assert np.array_equal(got.data, O.multiply("N", "N", 1.0, A, B, 0.0).data)
    finally:
        dbcsr.set_tuning_mnk([])
        dbcsr.set_tuning([])


def test_table_launches_and_table_changes():
    # a table whose every choice is a one-warp team adds no launch; one with
    # teams of two or four warps adds the classify pass only; a changed table
    # takes effect on the next multiply, also after a switch of stream.
    # Integer-valued inputs: every order of the sums is exact.
    import torch
    setup()
    sizes = (5, 13, 23)
    rng = np.random.default_rng(841)
    A, B, Cm = synth.random_small(rng, 12, 16, 12, p=0.7, sizes=sizes, dist="int", with_c=True)
    ref = O.multiply("N", "N", 1.0, A, B, 1.0, Cm)

    def run():
        got, st = gpu_multiply("N", "N", 1.0, A, B, 1.0, Cm, path="stacks")
        assert_same_pattern(got, ref)
        assert np.array_equal(got.data, ref.data)
        return st["kernel_launches"]

    base = run()
    mnk = [(m, n, k) for m in sizes for n in sizes for k in sizes]
    try:
        dbcsr.set_tuning([(m, n, 1) for m in sizes for n in sizes])
        dbcsr.set_tuning_mnk([e + (0,) for e in mnk])
        assert run() == base
        # the (m, n, k) entries of every present inner size override the (m, n) ones
        dbcsr.set_tuning([(m, n, 3) for m in sizes for n in sizes])
        assert run() == base
        dbcsr.set_tuning_mnk([e + (3,) for e in mnk])
        assert run() == base + 1
        s = torch.cuda.Stream()
        dbcsr.init(s)
        try:
            dbcsr.set_tuning_mnk([e + (2,) for e in mnk])
            assert run() == base + 1
            dbcsr.set_tuning_mnk([e + ((e[2] % 2) * 3,) for e in mnk])
            assert run() == base + 1
        finally:
            dbcsr.init()
    finally:
        dbcsr.set_tuning_mnk([])
        dbcsr.set_tuning([])
