"""Allocation failures on the GPU, injected on the host (no GPU fault).

The allocator hook refuses the (q+1)-th device allocation, for q = 0, 1, 2, ...
until a whole create + multiply + read-back succeeds, so every allocation that
path makes fails once. Every refusal must come back as DBCSR_ERR_ALLOC with the
hook's message, and the library must stay usable: the run that succeeds under
the hook, and a plain run afterwards, give the right product.

The hook hands out PyTorch caching-allocator memory on the library's stream.
What a failed call hands back stays mapped and is reused only by work ordered
after it on that stream, so kernels queued before a refusal finish on valid
memory. Every matrix is created afresh in each attempt and released after it.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import assert_same_pattern, from_gpu, gpu_multiply, normwise, setup

pytestmark = pytest.mark.gpu


class Refusing:
    """Hands out the first ``grant`` allocations, then refuses every one."""

    def __init__(self, grant):
        self.grant, self.calls, self.refused = grant, 0, 0

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.calls > self.grant:
            self.refused += 1
            return None
        return torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)

    def free(self, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)


CASES = [
    ("stacks", "fp64", {}, 1e-13),
    ("dense", "fp64", {}, 1e-13),
    ("stacks", "ozaki", {}, 1e-12),
    ("dense", "ozaki", {}, 1e-12),
    ("hybrid", "fp64", {"hybrid_panel": 4, "hybrid_fill_pct": 50}, 1e-13),
    ("dense", "tf32", {}, None),
]


@pytest.mark.parametrize("path,precision,kw,tol", CASES, ids=[f"{c[0]}-{c[1]}" for c in CASES])
def test_every_allocation_failure_is_reported_and_recovered(path, precision, kw, tol):
    setup()
    rng = np.random.default_rng(61)
    A, B, Cm = synth.random_small(rng, 8, 6, 7, p=0.6, sizes=(13, 22, 32), with_c=True, c_p=0.5)
    alpha, beta = 0.75, 1.5
    refusals = 0
    for grant in range(500):
        hook = Refusing(grant)
        made = []
        dbcsr.set_allocator(hook.alloc, hook.free)
        try:
            for M in (A, B, Cm):
                made.append(dbcsr.Matrix.from_blocks(M))
            dbcsr.multiply("N", "N", alpha, made[0], made[1], beta, made[2], path=path, precision=precision, **kw)
            got = from_gpu(made[2], Cm.row_sizes, Cm.col_sizes)
        except dbcsr.DbcsrError as e:
            assert e.code == dbcsr.ERR_ALLOC, str(e)
            assert "allocator hook returned NULL" in str(e)
            assert hook.refused == 1, "the library must stop at the first refusal"
            refusals += 1
            continue
        finally:
            for m in made:
                m.release()
            dbcsr.set_allocator(None, None)
            dbcsr.sync()
        break
    else:
        pytest.fail("no attempt succeeded within 500 granted allocations")
    assert hook.refused == 0 and refusals == grant and grant > 0

    plain, _ = gpu_multiply("N", "N", alpha, A, B, beta, Cm, path=path, precision=precision, **kw)
    assert_same_pattern(got, plain)
    if tol is None:
        assert normwise(got, plain, A, B) <= 1e-6
    else:
        ref = O.multiply("N", "N", alpha, A, B, beta, Cm)
        assert_same_pattern(got, ref)
        assert normwise(got, ref, A, B) <= tol
        assert normwise(plain, ref, A, B) <= tol
