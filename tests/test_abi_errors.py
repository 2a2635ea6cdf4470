"""Argument checks of the C ABI that run before any device call (CPU only).

Every entry point reports a bad argument as a negative DBCSR_ERR_* code with a
message in dbcsr_last_error(), leaves its outputs cleared, and touches neither
the device nor the arrays it was handed when an earlier check already fails
(the overflow case passes a block count far larger than its arrays).
"""
import ctypes as C

import numpy as np
import pytest

from paper_1910_04796_gb300 import dbcsr


@pytest.fixture(scope="module")
def L():
    return dbcsr.load(build_if_missing=True)


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def last(L):
    return L.dbcsr_last_error().decode()


def create(L, nbr, nbc, rs, cs, nblks, br, bc, out=True):
    h = C.c_void_p(12345)   # must be cleared on failure
    rc = L.dbcsr_create(C.byref(h) if out else None, nbr, nbc, rs, cs, nblks, br, bc, None, 0)
    return rc, h.value


def test_create_rejects_bad_arguments(L):
    rs = np.array([2, 3], np.int32)
    cs = np.array([4], np.int32)
    br = np.array([0, 1], np.int32)
    bc = np.array([0, 0], np.int32)
    cases = [
        (dict(out=False), dbcsr.ERR_ARG, "out is NULL"),
        (dict(nbr=-1), dbcsr.ERR_ARG, "negative size"),
        (dict(nblks=-1), dbcsr.ERR_ARG, "negative size"),
        (dict(rs=None), dbcsr.ERR_ARG, "block size array is NULL"),
        (dict(bc=None), dbcsr.ERR_ARG, "block index array is NULL"),
        # int32 guard: block ids are int32 in every kernel
        (dict(nblks=2 ** 31 - 1), dbcsr.ERR_OVERFLOW, "too many blocks"),
        (dict(nblks=2 ** 40), dbcsr.ERR_OVERFLOW, "too many blocks"),
        (dict(rs=_ip(np.array([2, 0], np.int32))), dbcsr.ERR_ARG, "row block size < 1 at 1"),
        (dict(cs=_ip(np.array([-4], np.int32))), dbcsr.ERR_ARG, "col block size < 1 at 0"),
        (dict(br=_ip(np.array([0, 2], np.int32))), dbcsr.ERR_ARG, "block coordinate out of range at 1"),
        (dict(bc=_ip(np.array([0, 1], np.int32))), dbcsr.ERR_ARG, "block coordinate out of range at 1"),
    ]
    for over, code, msg in cases:
        kw = dict(nbr=2, nbc=1, rs=_ip(rs), cs=_ip(cs), nblks=2, br=_ip(br), bc=_ip(bc), out=True)
        kw.update(over)
        rc, h = create(L, **kw)
        assert rc == code, (over, rc, last(L))
        assert msg in last(L), (over, last(L))
        if kw["out"]:
            assert h is None, "the handle must be cleared on failure"


def test_null_handles_rejected(L):
    n = C.c_int64()
    checks = [
        (lambda: L.dbcsr_multiply(b"N", b"N", 1.0, None, None, 0.0, None, None), "multiply: NULL matrix"),
        (lambda: L.dbcsr_get_stacks(b"N", b"N", None, None, 30000, None, 0, C.byref(n)), "get_stacks: NULL"),
        (lambda: L.dbcsr_get_info(None, None, None, None, None), "get_info: NULL matrix"),
        (lambda: L.dbcsr_get_index(None, None, None, None), "get_index: NULL matrix"),
        (lambda: L.dbcsr_get_data(None, None, 0), "get_data: NULL argument"),
        (lambda: L.dbcsr_set_data(None, None, 0), "set_data: NULL argument"),
        (lambda: L.dbcsr_data_ptr(None, None), "data_ptr: NULL argument"),
        (lambda: L.dbcsr_get_block(None, 0, 0, None, None), "get_block: NULL argument"),
        (lambda: L.dbcsr_get_stats(None), "get_stats: NULL"),
        (lambda: L.dbcsr_set_tuning(None, None, None, -1), "set_tuning: bad arguments"),
        (lambda: L.dbcsr_set_tuning(None, None, None, 3), "set_tuning: bad arguments"),
        (lambda: L.dbcsr_set_tuning_mnk(None, None, None, None, 3), "set_tuning_mnk: bad arguments"),
        (lambda: L.dbcsr_set_tuning_mnk(None, None, None, None, -1), "set_tuning_mnk: bad arguments"),
    ]
    for call, msg in checks:
        assert call() == dbcsr.ERR_ARG, msg
        assert msg in last(L)


def test_release_of_nothing_is_a_no_op(L):
    h = C.c_void_p()
    assert L.dbcsr_release(None) == dbcsr.OK
    assert L.dbcsr_release(C.byref(h)) == dbcsr.OK


def test_allocator_hooks_come_in_pairs(L):
    fa = dbcsr.ALLOC_FN(lambda nbytes, stream, ctx: None)
    assert L.dbcsr_set_allocator(fa, dbcsr.FREE_FN(), None) == dbcsr.ERR_ARG
    assert "both be set or both be NULL" in last(L)
    assert L.dbcsr_set_allocator(dbcsr.ALLOC_FN(), dbcsr.FREE_FN(), None) == dbcsr.OK


def test_noalloc_gemm_argument_checks(L):
    d = (C.c_double * 4)()
    f = L.dbcsr_dgemm_emulated_noalloc
    cases = [
        ((2, 2, 2, 1.0, d, 2, d, 2, 0.0, d, 2, 9, None), dbcsr.ERR_ARG, "slices must be 1..8"),
        ((-1, 2, 2, 1.0, d, 2, d, 2, 0.0, d, 2, 0, None), dbcsr.ERR_ARG, "negative size"),
        ((2, 2, 2, 1.0, d, 1, d, 2, 0.0, d, 2, 0, None), dbcsr.ERR_ARG, "leading dimension"),
        ((2, 2, 2, 1.0, d, 2, d, 2, 0.0, d, 1, 0, None), dbcsr.ERR_ARG, "leading dimension"),
        ((2, 2, 2, 1.0, None, 2, d, 2, 0.0, d, 2, 0, None), dbcsr.ERR_ARG, "NULL matrix pointer"),
        ((2 ** 25, 2, 2, 1.0, d, 2 ** 25, d, 2, 0.0, d, 2 ** 25, 0, None), dbcsr.ERR_OVERFLOW,
         "exceeds the fixed scratch"),
    ]
    for args, code, msg in cases:
        assert f(*args) == code, (args, last(L))
        assert msg in last(L)
    # empty products are complete without any device work
    assert f(0, 5, 3, 1.0, None, 1, None, 3, 0.0, None, 1, 0, None) == dbcsr.OK


def test_binding_allocator_hooks_come_in_pairs(L):
    with pytest.raises(ValueError):
        dbcsr.set_allocator(lambda nbytes, stream: None, None)
    with pytest.raises(ValueError):
        dbcsr.set_allocator(None, lambda ptr, nbytes, stream: None)
    dbcsr.set_allocator(None, None)   # the built-in pool: accepted without a GPU


def test_tuning_mnk_entries_out_of_range(L):
    # m, n, k in 1..32 and variant in 0..3 (host checks, no GPU needed)
    for bad in ([33, 5, 5, 0], [5, 0, 5, 0], [5, 5, 40, 0], [5, 5, 5, 4], [5, 5, 5, -1]):
        a = [np.array([x], np.int32) for x in bad]
        assert L.dbcsr_set_tuning_mnk(*[_ip(x) for x in a], 1) == dbcsr.ERR_ARG
        assert "out of range" in last(L)
    assert L.dbcsr_set_tuning_mnk(None, None, None, None, 0) == dbcsr.OK   # clears the table
