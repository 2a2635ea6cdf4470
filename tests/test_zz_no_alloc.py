"""The allocation-free emulated GEMM entry point (dbcsr_dgemm_emulated_noalloc).

It serves callers that cannot call cudaMalloc (device memory owned entirely by
another allocator, or code that must avoid the synchronisation an allocation
can imply); its scratch is a fixed array inside the library. Checked through
the C ABI against the existing entry point (dbcsr_multiply, dense path,
emulated precision): identical results -- the emulation is exact up to a
fixed FP64 recombination order, so the tolerance the other emulated tests use
is bit-equality -- on calls in a row with different inputs, against the
oracle's emulation bit for bit as well, plus the 1e-12 bar against the FP64
oracle. This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import gpu_multiply

pytestmark = pytest.mark.gpu


def run_noalloc(A, B, Cm, alpha, beta, slices):
    import torch
    Ad, Bd = O.densify(A), O.densify(B)
    Cd = O.densify(Cm)
    # column-major matrices = row-major tensors of their transposes
    tA = torch.from_numpy(np.ascontiguousarray(Ad.T)).cuda()
    tB = torch.from_numpy(np.ascontiguousarray(Bd.T)).cuda()
    tC = torch.from_numpy(np.ascontiguousarray(Cd.T)).cuda()
    dbcsr.dgemm_emulated_noalloc(alpha, tA, tB, beta, tC, slices=slices)
    torch.cuda.synchronize()
    return tC.cpu().numpy().T


# (block rows of A, block columns of A = block rows of B, block size, seed, slices,
# block columns of B): the last case has M = 512, N = 320, K = 512, where
# dbcsr_multiply takes its 128 x 256 tiles and the fused block recombination
# while this entry point keeps 128 x 128 tiles -- the results must still agree
CASES = [(9, 7, 22, 0, 7, 11), (5, 11, 13, 1, 6, 7), (16, 16, 32, 2, 7, 10)]


def test_noalloc_matches_existing_entry_point_twice():
    dbcsr.init()
    for call, (nb, nk, bs, seed, s, nc) in enumerate(CASES):
        rng = np.random.default_rng(900 + seed)
        A = synth.dense_matrix(rng, nb, nk, bs, bs, dist="wide", scale_exp=3.0)
        B = synth.dense_matrix(rng, nk, nc, bs, bs)
        Cm = synth.dense_matrix(rng, nb, nc, bs, bs)
        got = run_noalloc(A, B, Cm, 0.5, 2.0, s)
        ref_blocks, _ = gpu_multiply("N", "N", 0.5, A, B, 2.0, Cm, path="dense", precision="ozaki",
                                     ozaki_slices=s)
        ref = O.densify(ref_blocks)
        assert np.array_equal(got, ref), f"call {call}: differs from dbcsr_multiply"
        # and the oracle's step-by-step emulation itself
        want = O.densify(Cm)
        O.ozaki_gemm(0.5, O.densify(A), O.densify(B), 2.0, want, s=s)
        assert np.array_equal(got, want), f"call {call}: differs from the oracle's emulation"
        fp64 = O.multiply("N", "N", 0.5, A, B, 2.0, Cm)
        err = O.normwise_error(got, O.densify(fp64), O.densify(A), O.densify(B))
        assert err <= 1e-12


def test_noalloc_rejects_oversize():
    import torch
    dbcsr.init()
    M = N = K = 2048
    tA = torch.zeros((K, M), dtype=torch.float64, device="cuda")
    tB = torch.zeros((N, K), dtype=torch.float64, device="cuda")
    tC = torch.zeros((N, M), dtype=torch.float64, device="cuda")
    with pytest.raises(dbcsr.DbcsrError) as e:
        dbcsr.dgemm_emulated_noalloc(1.0, tA, tB, 0.0, tC)
    assert e.value.code == dbcsr.ERR_OVERFLOW
    assert "scratch" in str(e.value)
