"""GPU parity of the hybrid path: per panel of block rows of op(A), a
densified GEMM where the panel (and op(B)) is occupied at least the threshold,
the stack kernels elsewhere (Sec. III's densification applied to parts of a
sparse matrix).

FP64: within 1e-13 (normwise) of the oracle, same result pattern. Emulated
FP64: both the dense panels and the stack panels compute exact level sums
with the exponents of whole rows of op(A) and columns of op(B), so the result
is bit-identical to the oracle's emulation of the densified operands.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import gpu_multiply, assert_same_pattern, normwise
from test_gpu_smm_emul import emul_ref

pytestmark = pytest.mark.gpu


def _mats(seed, nbr=24, nbk=20, nbc=18, panel=4, sizes=(5, 13, 23, 26, 32), b_occ=0.9, with_c=False):
    rng = np.random.default_rng(seed)
    rsz = rng.choice(np.asarray(sizes, np.int32), nbr).astype(np.int32)
    ksz = rng.choice(np.asarray(sizes, np.int32), nbk).astype(np.int32)
    csz = rng.choice(np.asarray(sizes, np.int32), nbc).astype(np.int32)
    A = synth.make_matrix(rng, rsz, ksz, synth.panel_mask(rng, nbr, nbk, panel, 2, 0.1))
    B = synth.make_matrix(rng, ksz, csz, synth.bernoulli_mask(rng, nbk, nbc, b_occ))
    Cm = synth.make_matrix(rng, rsz, csz, synth.bernoulli_mask(rng, nbr, nbc, 0.3)) if with_c else None
    return A, B, Cm


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("beta", [0.0, 0.75])
def test_hybrid_fp64_matches_oracle(ta, tb, beta):
    A, B, Cm = _mats(700, with_c=beta != 0.0)
    As = synth.transpose_blocks(A) if ta == "T" else A
    Bs = synth.transpose_blocks(B) if tb == "T" else B
    got, st = gpu_multiply(ta, tb, 1.25, As, Bs, beta, Cm, path="hybrid", hybrid_panel=4, hybrid_fill_pct=50)
    ref = O.multiply(ta, tb, 1.25, As, Bs, beta, Cm)
    assert_same_pattern(got, ref)
    assert normwise(got, ref, As, Bs, ta, tb) <= 1e-13
    assert st["path"] == dbcsr.PATH_HYBRID
    assert 0 < st["dense_panels"] < 6          # 24 block rows in panels of 4: half dense


def test_hybrid_emulated_bit_exact():
    A, B, Cm = _mats(701, with_c=True, sizes=(13, 22, 32))
    got, st = gpu_multiply("N", "N", 0.5, A, B, 2.0, Cm, path="hybrid", precision="ozaki", hybrid_panel=4)
    ref, _, _ = emul_ref("N", "N", A, B, Cm, 0.5, 2.0, 7)
    assert_same_pattern(got, ref)
    assert np.array_equal(got.data, ref.data)
    assert st["dense_panels"] > 0


@pytest.mark.parametrize("pct,panel", [(100, 4), (1, 4), (50, 1), (50, 0)])
def test_hybrid_thresholds_and_panels(pct, panel):
    A, B, _ = _mats(702, b_occ=1.0)
    got, st = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="hybrid", hybrid_panel=panel, hybrid_fill_pct=pct)
    ref = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert_same_pattern(got, ref)
    assert normwise(got, ref, A, B) <= 1e-13
    if pct == 1:
        assert st["dense_panels"] == 6           # every panel is at least 1 % full
    if pct == 100:
        assert st["dense_panels"] == 3           # exactly the fully occupied panels


def test_hybrid_sparse_b_keeps_stacks():
    # op(B) below the threshold: no panel is densified
    A, B, _ = _mats(703, b_occ=0.2)
    got, st = gpu_multiply("N", "N", 1.0, A, B, 0.0, path="hybrid", hybrid_panel=4, hybrid_fill_pct=50)
    ref = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert normwise(got, ref, A, B) <= 1e-13
    assert st["dense_panels"] == 0


def test_hybrid_rejects_tf32():
    A, B, _ = _mats(704)
    with pytest.raises(dbcsr.DbcsrError) as e:
        gpu_multiply("N", "N", 1.0, A, B, 0.0, path="hybrid", precision="tf32")
    assert e.value.code == dbcsr.ERR_ARG
