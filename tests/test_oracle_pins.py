"""Pins of the CPU oracle against references other than itself (CPU only).

Each test fixes a fact the mathematics or the paper fixes, so that a plausible
mistake in the oracle (a dropped block, a transposed operand, a wrong index,
alpha/beta swapped, a wrong stack cut) fails at least one of them:

* brute-force dense triple loop in pure Python on the densified matrices,
  bit-exact (same summation order: block k ascending then inner index);
* numpy's matmul (library routine) within 1e-14 normwise;
* exact integer arithmetic for integer-valued inputs;
* identity, block-row permutation and transpose invariants, bit-exact;
* alpha/beta linearity, the beta = 0 convention (old C never read), empty A;
* brute-force enumeration of block-product triples and the count identity
  sum_k colnnz_A(k) * rownnz_B(k) for the stack list (Sec. II);
* double-double accumulation against exact rational arithmetic.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_04796_gb300 import synth


def dense_triple_loop(Ad, Bd):
    """Pure-Python C = A*B, summing the inner index ascending (no FMA)."""
    M, K = Ad.shape
    K2, N = Bd.shape
    assert K == K2
    Cd = np.zeros((M, N), order="F")
    for r in range(M):
        for c in range(N):
            s = 0.0
            for l in range(K):
                s = s + float(Ad[r, l]) * float(Bd[l, c])
            Cd[r, c] = s
    return Cd


def dense_of(res):
    return O.densify(res)


@pytest.mark.parametrize("seed", range(6))
def test_oracle_equals_dense_triple_loop_bitexact(seed):
    rng = np.random.default_rng(100 + seed)
    nbr, nbk, nbc = rng.integers(1, 7, 3)
    A, B, _ = synth.random_small(rng, nbr, nbk, nbc, p=0.5)
    res = O.multiply("N", "N", 1.0, A, B, 0.0)
    ref = dense_triple_loop(O.densify(A), O.densify(B))
    got = dense_of(res)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "T"), ("T", "T"), ("C", "N")])
def test_oracle_op_transpose_bitexact(ta, tb):
    rng = np.random.default_rng(7)
    A, B, _ = synth.random_small(rng, 4, 5, 3, p=0.6)
    As = synth.transpose_blocks(A) if ta in "TC" else A
    Bs = synth.transpose_blocks(B) if tb in "TC" else B
    res = O.multiply(ta, tb, 1.0, As, Bs, 0.0)
    ref = dense_triple_loop(O.densify(A), O.densify(B))
    assert np.array_equal(dense_of(res), ref)


def test_oracle_matches_numpy_matmul():
    rng = np.random.default_rng(11)
    A, B, _ = synth.random_small(rng, 12, 15, 10, p=0.4, sizes=(3, 7, 13, 22))
    res = O.multiply("N", "N", 1.0, A, B, 0.0)
    Ad, Bd = O.densify(A), O.densify(B)
    ref = Ad @ Bd
    assert O.normwise_error(dense_of(res), ref, Ad, Bd) < 1e-14


def test_oracle_integer_inputs_exact():
    rng = np.random.default_rng(12)
    A, B, _ = synth.random_small(rng, 8, 9, 7, p=0.5, sizes=(5, 13, 22), dist="int")
    res = O.multiply("N", "N", 1.0, A, B, 0.0)
    Ai = O.densify(A).astype(np.int64)
    Bi = O.densify(B).astype(np.int64)
    assert np.array_equal(dense_of(res).astype(np.int64), Ai @ Bi)


def test_pattern_is_symbolic_product_not_numeric():
    # blocks whose product cancels to zero are still part of the pattern
    rs = np.array([1, 1], np.int32)
    A = synth.BlockSparse(rs, rs, np.array([0, 0], np.int32), np.array([0, 1], np.int32),
                          np.array([1.0, 1.0]))
    B = synth.BlockSparse(rs, rs, np.array([0, 1], np.int32), np.array([0, 0], np.int32),
                          np.array([1.0, -1.0]))
    res = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert list(res.blk_row) == [0] and list(res.blk_col) == [0]
    assert res.data[0] == 0.0


def test_identity_left_and_right():
    rng = np.random.default_rng(13)
    A, B, _ = synth.random_small(rng, 5, 6, 4, p=0.6)
    ks = B.row_sizes
    # block-diagonal identity I with the k sizes of B: I*B = B exactly
    ii = np.arange(len(ks), dtype=np.int32)
    data = np.concatenate([np.eye(int(k)).reshape(-1, order="F") for k in ks])
    I = synth.BlockSparse(ks, ks, ii, ii, data)
    res = O.multiply("N", "N", 1.0, I, B, 0.0)
    assert np.array_equal(dense_of(res), O.densify(B))
    cs = A.col_sizes
    ii = np.arange(len(cs), dtype=np.int32)
    I2 = synth.BlockSparse(cs, cs, ii, ii, np.concatenate([np.eye(int(k)).reshape(-1, order="F") for k in cs]))
    res2 = O.multiply("N", "N", 1.0, A, I2, 0.0)
    assert np.array_equal(dense_of(res2), O.densify(A))


def test_block_row_permutation_permutes_c():
    rng = np.random.default_rng(14)
    A, B, _ = synth.random_small(rng, 6, 5, 4, p=0.6)
    perm = rng.permutation(6).astype(np.int32)          # new row perm[i] holds old row i
    Ap = synth.BlockSparse(A.row_sizes[np.argsort(perm)].astype(np.int32), A.col_sizes,
                           perm[A.blk_row], A.blk_col, A.data)
    r0 = O.multiply("N", "N", 1.0, A, B, 0.0)
    r1 = O.multiply("N", "N", 1.0, Ap, B, 0.0)
    d0 = {(int(i), int(j)): r0.data[o:o + A.row_sizes[i] * B.col_sizes[j]]
          for i, j, o in zip(r0.blk_row, r0.blk_col, r0.blk_off)}
    d1 = {(int(i), int(j)): r1.data[o:o + Ap.row_sizes[i] * B.col_sizes[j]]
          for i, j, o in zip(r1.blk_row, r1.blk_col, r1.blk_off)}
    assert set(d1) == {(int(perm[i]), j) for (i, j) in d0}
    for (i, j), v in d0.items():
        assert np.array_equal(d1[(int(perm[i]), j)], v)


def test_transpose_of_product_bitexact():
    # (A B)^T = B^T A^T: multiply(T, T, B, A) is the transpose of multiply(N, N, A, B)
    rng = np.random.default_rng(15)
    A, B, _ = synth.random_small(rng, 5, 4, 6, p=0.6)
    r = O.multiply("N", "N", 1.0, A, B, 0.0)
    rt = O.multiply("T", "T", 1.0, B, A, 0.0)
    assert np.array_equal(dense_of(rt), dense_of(r).T)


def test_alpha_beta_linearity():
    rng = np.random.default_rng(16)
    A, B, Cm = synth.random_small(rng, 5, 4, 6, p=0.6, with_c=True, c_p=0.5)
    r1 = dense_of(O.multiply("N", "N", 1.0, A, B, 0.0))
    r2 = dense_of(O.multiply("N", "N", 2.0, A, B, 0.0))
    assert np.array_equal(r2, 2.0 * r1)
    # beta != 0: C = alpha*acc + beta*Cold, pattern = product pattern U old pattern
    r3 = O.multiply("N", "N", 0.5, A, B, -3.0, Cm)
    Cd = O.densify(Cm)
    ref = (0.5 * r1) + (-3.0 * Cd)
    assert np.array_equal(dense_of(r3), ref)
    pat = set(zip(r3.blk_row.tolist(), r3.blk_col.tolist()))
    p1 = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert pat == set(zip(p1.blk_row.tolist(), p1.blk_col.tolist())) | set(
        zip(Cm.blk_row.tolist(), Cm.blk_col.tolist()))


def test_beta_zero_never_reads_old_c():
    rng = np.random.default_rng(17)
    A, B, Cm = synth.random_small(rng, 4, 4, 4, p=0.6, with_c=True, c_p=0.8)
    Cm.data[:] = np.nan
    r = O.multiply("N", "N", 1.0, A, B, 0.0, Cm)
    assert not np.isnan(r.data).any()
    p1 = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert np.array_equal(r.blk_row, p1.blk_row) and np.array_equal(r.blk_col, p1.blk_col)


def test_empty_a_gives_beta_c():
    rng = np.random.default_rng(18)
    _, B, Cm = synth.random_small(rng, 4, 5, 3, p=0.6, with_c=True, c_p=0.5)
    rs = Cm.row_sizes
    A = synth.BlockSparse(rs, B.row_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    r = O.multiply("N", "N", 1.0, A, B, 0.25, Cm)
    assert np.array_equal(dense_of(r), 0.25 * O.densify(Cm))
    r0 = O.multiply("N", "N", 1.0, A, B, 0.0, Cm)
    assert r0.blk_row.size == 0


def test_dimension_mismatch_rejected():
    rng = np.random.default_rng(19)
    A, B, _ = synth.random_small(rng, 3, 4, 3, p=0.6)
    Bbad = synth.BlockSparse(B.row_sizes[:-1], B.col_sizes, B.blk_row[B.blk_row < len(B.row_sizes) - 1],
                             B.blk_col[B.blk_row < len(B.row_sizes) - 1], np.zeros(0))
    with pytest.raises(ValueError):
        O.multiply("N", "N", 1.0, A, Bbad, 0.0)


def test_inner_block_size_mismatch_rejected():
    # same number of block columns in A as block rows in B, but one k block of
    # A is narrower than B's: no block product is defined (Sec. II)
    one = np.array([2], np.int32)
    z = np.zeros(1, np.int32)
    A = synth.BlockSparse(one, np.array([2, 3], np.int32), np.zeros(2, np.int32), np.array([0, 1], np.int32),
                          np.ones(2 * 2 + 2 * 3))
    B = synth.BlockSparse(np.array([3, 3], np.int32), one, np.array([0, 1], np.int32), np.zeros(2, np.int32),
                          np.ones(3 * 2 + 3 * 2))
    with pytest.raises(ValueError):
        O.multiply("N", "N", 1.0, A, B, 0.0)
    with pytest.raises(ValueError):
        O.stack_list("N", "N", A, B)
    # the same check through op(): A^T with A stored 3 x 2 has a k size of 2
    At = synth.BlockSparse(np.array([2, 3], np.int32), one, np.array([0, 1], np.int32), z.repeat(2),
                           np.ones(2 * 2 + 3 * 2))
    with pytest.raises(ValueError):
        O.multiply("T", "N", 1.0, At, B, 0.0)


def test_duplicate_block_rejected():
    # a block index names each (row, column) at most once (blocked CSR, Sec. II)
    rs = np.array([2, 2], np.int32)
    A = synth.BlockSparse(rs, rs, np.array([0, 1, 0], np.int32), np.array([1, 0, 1], np.int32), np.ones(12))
    B = synth.BlockSparse(rs, rs, np.array([0, 1], np.int32), np.array([0, 1], np.int32), np.ones(8))
    with pytest.raises(ValueError):
        O.multiply("N", "N", 1.0, A, B, 0.0)
    with pytest.raises(ValueError):
        O.multiply("N", "N", 1.0, B, A, 0.0)
    with pytest.raises(ValueError):
        O.stack_list("N", "N", A, B)


def test_row_subset_equals_full_rows():
    rng = np.random.default_rng(20)
    A, B, Cm = synth.random_small(rng, 7, 5, 6, p=0.5, with_c=True)
    full = O.multiply("N", "N", 1.0, A, B, 1.0, Cm)
    sub = O.multiply("N", "N", 1.0, A, B, 1.0, Cm, rows=[1, 4, 5])
    keep = np.isin(full.blk_row, [1, 4, 5])
    assert np.array_equal(sub.blk_row, full.blk_row[keep])
    assert np.array_equal(sub.blk_col, full.blk_col[keep])
    ref = np.concatenate([full.data[o:o + A.row_sizes[i] * B.col_sizes[j]]
                          for i, j, o in zip(full.blk_row[keep], full.blk_col[keep], full.blk_off[keep])])
    assert np.array_equal(sub.data, ref)


# ----------------------------------------------------------------------------
# stack list (Sec. II: Traversal + Generation, at most 30'000 products a batch)
# ----------------------------------------------------------------------------
def brute_force_stacks(A, B, cap):
    pa = set(zip(A.blk_row.tolist(), A.blk_col.tolist()))
    pb = set(zip(B.blk_row.tolist(), B.blk_col.tolist()))
    ent = []
    for i in range(len(A.row_sizes)):
        for j in range(len(B.col_sizes)):
            for k in range(len(A.col_sizes)):
                if (i, k) in pa and (k, j) in pb:
                    ent.append((int(A.row_sizes[i]), int(B.col_sizes[j]), int(A.col_sizes[k]), i, j, k))
    ent.sort()
    out = []
    sid, run, prev = -1, 0, None
    for e in ent:
        if e[:3] != prev or run == cap:
            sid += 1
            run = 0
        prev = e[:3]
        run += 1
        out.append((sid,) + e)
    return np.array(out, np.int32).reshape(-1, 7)


@pytest.mark.parametrize("seed,cap", [(0, 30000), (1, 3), (2, 1), (3, 7)])
def test_stack_list_brute_force(seed, cap):
    rng = np.random.default_rng(200 + seed)
    A, B, _ = synth.random_small(rng, 6, 5, 6, p=0.5, sizes=(2, 3, 5))
    got = O.stack_list("N", "N", A, B, cap)
    ref = brute_force_stacks(A, B, cap)
    assert np.array_equal(got, ref)


def test_stack_count_identity_and_cap():
    w = synth.workload_small_sparse(0)
    A, B = w.A, w.B
    st = O.stack_list("N", "N", A, B)
    colnnz_a = np.bincount(A.blk_col, minlength=20)
    rownnz_b = np.bincount(B.blk_row, minlength=20)
    assert len(st) == int((colnnz_a * rownnz_b).sum())
    # one shape (13,13,13) -> one stack below the cap; flops = 2*13^3 per entry
    assert len(np.unique(st[:, 0])) == (1 if len(st) else 0)
    assert np.all(st[:, 1:4] == 13)


def test_stack_list_transposed_ops():
    rng = np.random.default_rng(21)
    A, B, _ = synth.random_small(rng, 5, 4, 6, p=0.6, sizes=(2, 3))
    ref = O.stack_list("N", "N", A, B, 5)
    got = O.stack_list("T", "T", synth.transpose_blocks(A), synth.transpose_blocks(B), 5)
    assert np.array_equal(got, ref)


# ----------------------------------------------------------------------------
# double-double accumulation (Dot2) against exact rational arithmetic
# ----------------------------------------------------------------------------
def test_dot2_against_exact_rationals():
    rng = np.random.default_rng(22)
    n = 40
    # ill-conditioned dot products: large cancelling terms plus small ones
    big = rng.uniform(-1, 1, n) * 10.0 ** rng.integers(-8, 9, n)
    a = big.copy()
    b = rng.uniform(-1, 1, n)
    a = np.concatenate([a, -a[:10]])
    b = np.concatenate([b, b[:10] * (1 + 2.0 ** -30)])
    K = len(a)
    one = np.array([1], np.int32)
    A = synth.BlockSparse(one, np.array([K], np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32), a)
    B = synth.BlockSparse(np.array([K], np.int32), one, np.zeros(1, np.int32), np.zeros(1, np.int32), b)
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    r2 = O.multiply("N", "N", 1.0, A, B, 0.0, mode=1).data[0]
    r1 = O.multiply("N", "N", 1.0, A, B, 0.0, mode=0).data[0]
    u = 2.0 ** -53
    absum = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(a, b))
    gamma = (K * u) / (1 - K * u)
    # Ogita-Rump-Oishi: |dot2 - exact| <= u|exact| + gamma_n^2 * sum|a_i b_i|
    bound = u * abs(exact) + Fraction(gamma) ** 2 * absum
    assert abs(Fraction(r2) - exact) <= bound
    # plain FP64 obeys the classical gamma_n bound, and Dot2 is strictly better here
    assert abs(Fraction(r1) - exact) <= Fraction(gamma) * absum
    assert abs(Fraction(r2) - exact) <= abs(Fraction(r1) - exact)


# ----------------------------------------------------------------------------
# densification (Sec. III)
# ----------------------------------------------------------------------------
def test_densify_roundtrip_and_placement():
    rng = np.random.default_rng(23)
    A, _, _ = synth.random_small(rng, 5, 6, 2, p=0.5, sizes=(1, 3, 4))
    D = O.densify(A)
    back = O.undensify(D, A.row_sizes, A.col_sizes, A.blk_row, A.blk_col)
    assert np.array_equal(back, A.data)
    # an element placed by hand: first block's (0,0) entry sits at its block's corner
    if A.nblks:
        i, j = int(A.blk_row[0]), int(A.blk_col[0])
        assert D[int(A.row_sizes[:i].sum()), int(A.col_sizes[:j].sum())] == A.data[0]
    assert np.count_nonzero(D) <= A.data.size


def test_dense_gemm_against_numpy_and_loop():
    rng = np.random.default_rng(24)
    Ad = np.asfortranarray(rng.uniform(-1, 1, (7, 5)))
    Bd = np.asfortranarray(rng.uniform(-1, 1, (5, 6)))
    Cd = np.asfortranarray(rng.uniform(-1, 1, (7, 6)))
    out = O.dense_gemm("N", "N", 1.0, Ad, Bd, 0.0, Cd.copy(order="F"))
    assert np.array_equal(out, dense_triple_loop(Ad, Bd))
    out2 = O.dense_gemm("T", "T", 2.0, np.asfortranarray(Ad.T), np.asfortranarray(Bd.T), 1.0, Cd.copy(order="F"))
    assert np.allclose(out2, 2 * Ad @ Bd + Cd, rtol=0, atol=1e-14)


def test_dense_limit_block_oracle_equals_dense_gemm():
    # Sec. III: the densified product equals the block product (same sum order)
    rng = np.random.default_rng(25)
    A = synth.dense_matrix(rng, 4, 3, 5, 5)
    B = synth.dense_matrix(rng, 3, 4, 5, 5)
    res = O.multiply("N", "N", 1.0, A, B, 0.0)
    Ad, Bd = O.densify(A), O.densify(B)
    Cd = np.zeros((Ad.shape[0], Bd.shape[1]), order="F")
    O.dense_gemm("N", "N", 1.0, Ad, Bd, 0.0, Cd)
    assert np.array_equal(dense_of(res), Cd)
