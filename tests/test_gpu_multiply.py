"""GPU parity: the CUDA library against the CPU oracle, through the C ABI.

Bars: result patterns identical; FP64 values within 1e-13 normwise
(||C - C_ref||_F / (||A||_F ||B||_F)) and bit-exact for integer-valued inputs
(every partial sum is an integer below 2^53, so any summation order is exact).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import dbcsr, synth

from gpu_util import assert_same_pattern, gpu_multiply, normwise, setup, to_gpu, empty_like_c

pytestmark = pytest.mark.gpu
TOL = 1e-13


def check(ta, tb, alpha, A, B, beta, Cm=None, exact=False, **kw):
    got, st = gpu_multiply(ta, tb, alpha, A, B, beta, Cm, **kw)
    ref = O.multiply(ta, tb, alpha, A, B, beta, Cm)
    assert_same_pattern(got, ref)
    if exact:
        assert np.array_equal(got.data, ref.data)
    else:
        assert normwise(got, ref, A, B) <= TOL
    return got, ref, st


@pytest.mark.parametrize("path", ["stacks", "dense"])
def test_small_sparse_workload(path):
    w = synth.workload_small_sparse(0)
    got, ref, st = check("N", "N", 1.0, w.A, w.B, 0.0, path=path)
    assert st["kernel_launches"] > 0


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("sizes", [(1, 2, 3, 4, 5), (5, 13, 22, 23, 26, 32)])
def test_integer_inputs_bit_exact(seed, sizes):
    rng = np.random.default_rng(300 + seed)
    A, B, Cm = synth.random_small(rng, 7, 6, 8, p=0.5, sizes=sizes, dist="int", with_c=True)
    check("N", "N", 1.0, A, B, 0.0, exact=True)
    check("N", "N", 2.0, A, B, 1.0, Cm, exact=True)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T"), ("C", "N")])
@pytest.mark.parametrize("path", ["stacks", "dense"])
def test_transposes(ta, tb, path):
    rng = np.random.default_rng(31)
    A, B, _ = synth.random_small(rng, 6, 5, 7, p=0.5, sizes=(3, 5, 13), dist="int")
    As = synth.transpose_blocks(A) if ta in "TC" else A
    Bs = synth.transpose_blocks(B) if tb in "TC" else B
    check(ta, tb, 1.0, As, Bs, 0.0, exact=True, path=path)
    rng = np.random.default_rng(32)
    A, B, _ = synth.random_small(rng, 6, 5, 7, p=0.6, sizes=(4, 22, 32))
    As = synth.transpose_blocks(A) if ta in "TC" else A
    Bs = synth.transpose_blocks(B) if tb in "TC" else B
    check(ta, tb, 0.75, As, Bs, 0.0, path=path)


@pytest.mark.parametrize("path", ["stacks", "dense"])
def test_beta_union_and_scaling(path):
    rng = np.random.default_rng(33)
    A, B, Cm = synth.random_small(rng, 8, 6, 9, p=0.4, sizes=(2, 13, 22), with_c=True, c_p=0.5)
    check("N", "N", -1.5, A, B, 0.25, Cm, path=path)


@pytest.mark.parametrize("path", ["stacks", "dense"])
def test_beta_zero_ignores_nan(path):
    rng = np.random.default_rng(34)
    A, B, Cm = synth.random_small(rng, 5, 5, 5, p=0.5, sizes=(3, 13), with_c=True, c_p=0.9)
    Cm.data[:] = np.nan
    got, ref, _ = check("N", "N", 1.0, A, B, 0.0, Cm, path=path)
    assert not np.isnan(got.data).any()


def test_empty_operands():
    rng = np.random.default_rng(35)
    _, B, Cm = synth.random_small(rng, 4, 5, 3, p=0.6, with_c=True, c_p=0.5)
    A = synth.BlockSparse(Cm.row_sizes, B.row_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    check("N", "N", 1.0, A, B, 0.5, Cm, exact=True)
    got, _, _ = check("N", "N", 1.0, A, B, 0.0, Cm)
    assert got.blk_row.size == 0


def test_zero_sized_grids():
    setup()
    rs = np.array([3, 4], np.int32)
    A = synth.BlockSparse(rs, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = synth.BlockSparse(np.zeros(0, np.int32), rs, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    got, _ = gpu_multiply("N", "N", 1.0, A, B, 0.0)
    assert got.blk_row.size == 0


@pytest.mark.parametrize("nb,bs", [(7, 13), (5, 22), (3, 32), (9, 5)])
def test_dense_path_ragged_tiles(nb, bs):
    # dense limit with tiles that do not divide 64: exercises GEMM edges
    rng = np.random.default_rng(36 + nb)
    A = synth.dense_matrix(rng, nb, nb + 2, bs, bs)
    B = synth.dense_matrix(rng, nb + 2, nb + 1, bs, bs)
    Cm = synth.dense_matrix(rng, nb, nb + 1, bs, bs)
    _, _, st = check("N", "N", 1.0, A, B, 1.0, Cm, path="dense")
    assert st["path"] == dbcsr.PATH_DENSE
    # FP64 blocks up to 32 x 32 stay on the stack kernels under AUTO
    _, _, st = check("N", "N", 1.0, A, B, 1.0, Cm)
    assert st["path"] == dbcsr.PATH_STACKS


def test_uneven_banded_small():
    w = synth.workload_uneven(seed=3, nblk=120, occ=0.05, width=12)
    check("N", "N", 1.0, w.A, w.B, 0.0)


@pytest.mark.parametrize("cap", [30000, 7, 1])
def test_stack_list_bit_exact(cap):
    setup()
    rng = np.random.default_rng(37)
    A, B, _ = synth.random_small(rng, 9, 8, 7, p=0.5, sizes=(5, 13, 23))
    Ag, Bg = to_gpu(A), to_gpu(B)
    got = dbcsr.get_stacks("N", "N", Ag, Bg, cap)
    ref = O.stack_list("N", "N", A, B, cap)
    assert np.array_equal(got, ref)
    got_t = dbcsr.get_stacks("T", "N", to_gpu(synth.transpose_blocks(A)), Bg, cap)
    assert np.array_equal(got_t, ref)


def test_stack_list_workload_counts():
    setup()
    w = synth.workload_small_sparse(0)
    got = dbcsr.get_stacks("N", "N", to_gpu(w.A), to_gpu(w.B))
    ref = O.stack_list("N", "N", w.A, w.B)
    assert np.array_equal(got, ref)


def test_get_block_and_info():
    setup()
    rng = np.random.default_rng(38)
    A, _, _ = synth.random_small(rng, 4, 5, 2, p=0.5, sizes=(2, 3))
    Ag = to_gpu(A)
    nbr, nbc, n, e = Ag.info()
    assert (nbr, nbc, n, e) == (4, 5, A.nblks, A.data.size)
    pos = 0
    for i, j in zip(A.blk_row, A.blk_col):
        m, nn = int(A.row_sizes[i]), int(A.col_sizes[j])
        blk = Ag.get_block(int(i), int(j), m, nn)
        assert np.array_equal(blk, A.data[pos:pos + m * nn].reshape((m, nn), order="F"))
        pos += m * nn
    present = set(zip(A.blk_row.tolist(), A.blk_col.tolist()))
    for i in range(4):
        for j in range(5):
            if (i, j) not in present:
                assert Ag.get_block(i, j, int(A.row_sizes[i]), int(A.col_sizes[j])) is None


def test_create_unsorted_and_device_data():
    import torch
    setup()
    rng = np.random.default_rng(39)
    A, _, _ = synth.random_small(rng, 5, 5, 2, p=0.6, sizes=(2, 3, 4))
    perm = rng.permutation(A.nblks)
    # reorder the blocks and their data
    sizes = A.row_sizes[A.blk_row].astype(np.int64) * A.col_sizes[A.blk_col]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    data = np.concatenate([A.data[offs[b]:offs[b + 1]] for b in perm]) if A.nblks else np.zeros(0)
    M1 = dbcsr.Matrix.create(A.row_sizes, A.col_sizes, A.blk_row[perm], A.blk_col[perm], data)
    M2 = dbcsr.Matrix.create(A.row_sizes, A.col_sizes, A.blk_row[perm], A.blk_col[perm],
                             torch.from_numpy(data).cuda())
    for M in (M1, M2):
        br, bc, _ = M.index()
        assert np.array_equal(br, A.blk_row) and np.array_equal(bc, A.blk_col)
        assert np.array_equal(M.data(), A.data)


def test_errors_are_reported():
    setup()
    rng = np.random.default_rng(40)
    A, B, _ = synth.random_small(rng, 3, 4, 3, p=0.6)
    Ag, Bg = to_gpu(A), to_gpu(B)
    Cbad = empty_like_c(A.row_sizes, A.row_sizes[:2])
    with pytest.raises(dbcsr.DbcsrError) as e:
        dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.0, Cbad)
    assert e.value.code == dbcsr.ERR_DIM
    with pytest.raises(dbcsr.DbcsrError) as e:
        dbcsr.multiply("X", "N", 1.0, Ag, Bg, 0.0, empty_like_c(A.row_sizes, B.col_sizes))
    assert e.value.code == dbcsr.ERR_ARG
    with pytest.raises(dbcsr.DbcsrError) as e:
        dbcsr.Matrix.create([2, 2], [2], [0, 0], [0, 0], np.zeros(8))
    assert e.value.code == dbcsr.ERR_ARG
    with pytest.raises(dbcsr.DbcsrError) as e:
        dbcsr.Matrix.create([2, 2], [2], [0, 5], [0, 0], np.zeros(8))
    assert e.value.code == dbcsr.ERR_ARG


def test_torch_allocator_hooks():
    setup()
    rng = np.random.default_rng(41)
    A, B, Cm = synth.random_small(rng, 6, 5, 6, p=0.5, sizes=(3, 13), with_c=True)
    dbcsr.use_torch_allocator(True)
    try:
        check("N", "N", 1.0, A, B, 1.0, Cm)
        check("N", "N", 1.0, A, B, 1.0, Cm, path="dense")
    finally:
        dbcsr.use_torch_allocator(False)
