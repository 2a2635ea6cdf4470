"""Bounded waits of the tensor-core pipelines run out on purpose (no GPU fault).

The stages of the tcgen05 kernels (the emulated-FP64 GEMMs on one CTA or on
CTA pairs, the TF32 GEMMs and the emulated stack kernel) hand work to each other through shared-memory
barriers, and every wait on them gives up after a limit (4 s by default). With
the limit set to a few nanoseconds the first waits give up before the copies
or the tensor-core work they wait for can finish: the kernel stops every role,
waits (with its own fixed 4 s limit) for its copies and MMAs in flight, frees
its tensor memory and returns, and the call reports DBCSR_ERR_TIMEOUT. The
library then stays usable: with the default limit restored, the same multiply
in the same process matches the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import assert_same_pattern, gpu_multiply, setup

pytestmark = pytest.mark.gpu


def operands(case):
    rng = np.random.default_rng(950)
    if case == "stacks":
        w = synth.workload_precision_sparse(seed=9, nblk=24, occ=0.3)
        return w.A, w.B
    ncols = 5 if case == "dense-128" else 20               # N = 160 (128 x 128 tiles) or 640
    return synth.dense_matrix(rng, 12, 64, 32, 32), synth.dense_matrix(rng, 64, ncols, 32, 32)


@pytest.mark.parametrize("case,precision", [("dense-256", "ozaki"), ("dense-pair", "ozaki"), ("dense-128", "ozaki"),
                                            ("dense-256", "tf32"), ("dense-128", "tf32"), ("stacks", "ozaki")])
def test_wait_expiry_reports_timeout_then_recovers(case, precision):
    setup()
    A, B = operands(case)
    path = "stacks" if case == "stacks" else "dense"
    # kernel 2: the tcgen05 stack kernel; 4: the slice GEMM on CTA pairs (M = 384, N = 640)
    kw = dict(path=path, precision=precision, kernel={"stacks": 2, "dense-pair": 4}.get(case, 0))
    dbcsr.set_wait_limit(2)
    try:
        with pytest.raises(dbcsr.DbcsrError) as e:
            gpu_multiply("N", "N", 1.0, A, B, 0.0, **kw)
        assert e.value.code == dbcsr.ERR_TIMEOUT
        assert "timed out" in str(e.value)
    finally:
        dbcsr.set_wait_limit(0)
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0, **kw)
    ref = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert_same_pattern(got, ref)
    err = O.normwise_error(O.densify(got), O.densify(ref), O.densify(A), O.densify(B))
    assert err <= (1e-12 if precision == "ozaki" else 1e-2)
