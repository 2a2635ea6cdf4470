"""GPU check of the kept stack plan and its CUDA-graph replay (FP64 stack path).

A repeated multiply of the same operand patterns (values may change) into
the C the plan produced must skip stack generation, replay one graph and
give the same result as a fresh multiply -- checked against the oracle,
bit-exactly on integer-valued inputs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import from_gpu, setup, to_gpu

pytestmark = pytest.mark.gpu


def oracle_step(A, B, Cm, alpha, beta):
    r = O.multiply("N", "N", alpha, A, B, beta, Cm)
    return synth.BlockSparse(r.row_sizes, r.col_sizes, r.blk_row, r.blk_col, r.data)


@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_replay_matches_oracle_and_tracks_values(beta):
    setup()
    rng = np.random.default_rng(700)
    A, B, Cm = synth.random_small(rng, 12, 10, 11, p=0.35, sizes=(5, 13, 22), dist="int", with_c=True)
    Ag, Bg, Cg = to_gpu(A), to_gpu(B), to_gpu(Cm)
    ref = Cm
    for step in range(4):
        if step == 2:   # new values, same pattern: the plan stays valid
            A = synth.BlockSparse(A.row_sizes, A.col_sizes, A.blk_row, A.blk_col,
                                  rng.integers(-4, 5, A.data.size).astype(np.float64))
            Ag.set_data(A.data)
        dbcsr.multiply("N", "N", 1.0, Ag, Bg, beta, Cg, path="stacks", reuse_plan=True)
        st = dbcsr.stats()
        if step >= 1:
            assert st["kernel_launches"] == 1, "a kept plan replays one graph"
        ref = oracle_step(A, B, ref, 1.0, beta)
        got = from_gpu(Cg, A.row_sizes, B.col_sizes)
        assert np.array_equal(got.blk_row, ref.blk_row) and np.array_equal(got.blk_col, ref.blk_col)
        assert np.array_equal(got.data, ref.data), f"step {step}"


def test_plan_invalidated_by_other_operand_or_scalars():
    setup()
    rng = np.random.default_rng(710)
    A, B, _ = synth.random_small(rng, 8, 8, 8, p=0.4, sizes=(4, 13))
    B2 = synth.make_matrix(rng, B.row_sizes, B.col_sizes, synth.bernoulli_mask(rng, 8, 8, 0.5))
    Ag, Bg, B2g = to_gpu(A), to_gpu(B), to_gpu(B2)
    Cg = dbcsr.Matrix.create(A.row_sizes, B.col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))
    dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.0, Cg, path="stacks", reuse_plan=True)
    dbcsr.multiply("N", "N", 1.0, Ag, B2g, 0.0, Cg, path="stacks", reuse_plan=True)   # other B
    assert dbcsr.stats()["kernel_launches"] > 1
    ref = O.multiply("N", "N", 1.0, A, B2, 0.0)
    got = from_gpu(Cg, A.row_sizes, B.col_sizes)
    assert np.array_equal(got.blk_col, ref.blk_col)
    assert O.normwise_error(O.densify(got), O.densify(ref), O.densify(A), O.densify(B2)) <= 1e-13
    dbcsr.multiply("N", "N", 2.0, Ag, B2g, 0.0, Cg, path="stacks", reuse_plan=True)   # other alpha
    assert dbcsr.stats()["kernel_launches"] > 1
    got = from_gpu(Cg, A.row_sizes, B.col_sizes)
    assert O.normwise_error(O.densify(got), 2.0 * O.densify(ref), O.densify(A), O.densify(B2)) <= 1e-13


def test_small_workload_replay_latency():
    setup()
    import torch
    w = synth.workload_small_sparse(0)
    Ag, Bg = to_gpu(w.A), to_gpu(w.B)
    Cg = dbcsr.Matrix.create(w.A.row_sizes, w.B.col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))
    dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.0, Cg, path="stacks", reuse_plan=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.0, Cg, path="stacks", reuse_plan=True)
    e1.record()
    torch.cuda.synchronize()
    ref = O.multiply("N", "N", 1.0, w.A, w.B, 0.0)
    got = from_gpu(Cg, w.A.row_sizes, w.B.col_sizes)
    assert O.normwise_error(O.densify(got), O.densify(ref), O.densify(w.A), O.densify(w.B)) <= 1e-13
    assert e0.elapsed_time(e1) / 20 < 5.0   # ms per replayed multiply, generous
