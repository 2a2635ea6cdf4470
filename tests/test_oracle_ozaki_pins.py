"""Pins of the oracle's emulated-FP64 (integer-slice) product (CPU only).

The emulation is not in the paper; it follows Ozaki, Ogita, Oishi & Rump
(2012) in integer form. Pinned against: exact integer arithmetic (inputs that
the leading slice captures whole), exact rational arithmetic within the
method's own truncation bound, the exact reconstruction of a value from 8
slices of 7 bits (56 >= 53 bits), monotone error decrease in the slice count,
and the level-sum identity against an int64 matmul of slices built here.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import oracle as O


def test_split_properties():
    rng = np.random.default_rng(50)
    for x in rng.uniform(-1, 1, 200):
        sl = O.ozaki_split(x, 8)
        assert all(-127 <= v <= 127 for v in sl)
        assert all(v == 0 or (v > 0) == (x > 0) for v in sl)       # truncation keeps the sign
        rec = sum(Fraction(v) * Fraction(2) ** (-7 * (t + 1)) for t, v in enumerate(sl))
        if abs(x) >= 2 ** -4:                                      # 53 bits all inside 56
            assert rec == Fraction(float(x))
        r5 = sum(Fraction(v) * Fraction(2) ** (-7 * (t + 1)) for t, v in enumerate(O.ozaki_split(x, 5)))
        assert abs(Fraction(float(x)) - r5) < Fraction(2) ** -35   # |r_s| < 2^-7s
        assert abs(r5) <= abs(Fraction(float(x)))                  # truncation toward zero


def test_split_known_values():
    # 0.5 = 64 * 2^-7; -0.75 = -96 * 2^-7; 2^-8 = 64 * 2^-14
    assert O.ozaki_split(0.5, 3) == [64, 0, 0]
    assert O.ozaki_split(-0.75, 3) == [-96, 0, 0]
    assert O.ozaki_split(2.0 ** -8, 3) == [0, 64, 0]
    assert O.ozaki_split(1 - 2.0 ** -21, 3) == [127, 127, 127]


def test_exponents_frexp():
    A = np.asfortranarray(np.array([[0.5, -3.0], [0.0, 0.0], [1.0, 0.25]]))
    B = np.asfortranarray(np.array([[7.9, 0.0], [-8.0, 0.0]]))
    e, f = O.ozaki_exponents(A, B)
    assert list(e) == [2, 0, 1]       # 3 = 0.75*2^2; zero row -> 0; 1 = 0.5*2^1
    assert list(f) == [4, 0]          # 8 = 0.5*2^4


@pytest.mark.parametrize("s", [1, 3, 7])
def test_integer_inputs_exact(s):
    rng = np.random.default_rng(51)
    A = rng.integers(-8, 9, (17, 23)).astype(np.float64)
    B = rng.integers(-8, 9, (23, 13)).astype(np.float64)
    Cd = np.zeros((17, 13), order="F")
    O.ozaki_gemm(1.0, A, B, 0.0, Cd, s=s)
    assert np.array_equal(Cd, A @ B)


def test_levels_equal_int_matmul_of_slices():
    rng = np.random.default_rng(52)
    M, K, N, s = 6, 9, 5, 4
    A = np.asfortranarray(rng.uniform(-1, 1, (M, K)))
    B = np.asfortranarray(rng.uniform(-1, 1, (K, N)))
    e, f = O.ozaki_exponents(A, B)
    SA = np.zeros((s, M, K), np.int64)
    SB = np.zeros((s, K, N), np.int64)
    for i in range(M):
        for l in range(K):
            SA[:, i, l] = O.ozaki_split(math.ldexp(A[i, l], -int(e[i])), s)
    for l in range(K):
        for j in range(N):
            SB[:, l, j] = O.ozaki_split(math.ldexp(B[l, j], -int(f[j])), s)
    _, lv = O.ozaki_gemm(1.0, A, B, 0.0, np.zeros((M, N), order="F"), s=s, want_levels=True)
    for d in range(2, s + 2):
        G = sum(SA[t - 1] @ SB[d - t - 1] for t in range(1, d) if 1 <= d - t <= s)
        assert np.array_equal(lv[d - 2], G)


def test_error_within_truncation_bound_exact_rationals():
    rng = np.random.default_rng(53)
    M, K, N = 5, 30, 4
    A = np.asfortranarray(rng.uniform(-1, 1, (M, K)) * 10.0 ** rng.uniform(-4, 4, (M, K)))
    B = np.asfortranarray(rng.uniform(-1, 1, (K, N)) * 10.0 ** rng.uniform(-4, 4, (K, N)))
    e, f = O.ozaki_exponents(A, B)
    for s in (3, 5, 7):
        Cd = np.zeros((M, N), order="F")
        O.ozaki_gemm(1.0, A, B, 0.0, Cd, s=s)
        for i in range(M):
            for j in range(N):
                exact = sum(Fraction(float(A[i, l])) * Fraction(float(B[l, j])) for l in range(K))
                # per scaled product: truncation (2.01 * 2^-7s) + dropped levels (s * 2^-7s)
                trunc = Fraction(2) ** (int(e[i]) + int(f[j])) * K * (Fraction(s) + Fraction(201, 100)) \
                    * Fraction(2) ** (-7 * s)
                rounding = Fraction(2) ** -50 * (abs(exact) + Fraction(2) ** (int(e[i]) + int(f[j])) * K)
                assert abs(Fraction(float(Cd[i, j])) - exact) <= trunc + rounding


def test_error_decreases_with_slices_and_meets_1e12():
    rng = np.random.default_rng(54)
    M = K = N = 64
    A = np.asfortranarray(rng.uniform(-1, 1, (M, K)) * 10.0 ** rng.uniform(-4, 4, (M, K)))
    B = np.asfortranarray(rng.uniform(-1, 1, (K, N)) * 10.0 ** rng.uniform(-4, 4, (K, N)))
    ref = np.zeros((M, N), order="F")
    O.dense_gemm("N", "N", 1.0, A, B, 0.0, ref)
    errs = []
    for s in range(2, 9):
        Cd = np.zeros((M, N), order="F")
        O.ozaki_gemm(1.0, A, B, 0.0, Cd, s=s)
        errs.append(O.normwise_error(Cd, ref, A, B))
    assert all(errs[q + 1] <= errs[q] * 1.0001 + 1e-17 for q in range(len(errs) - 1))
    assert errs[7 - 2] <= 1e-12


def test_alpha_beta_and_row_subset():
    rng = np.random.default_rng(55)
    A = np.asfortranarray(rng.uniform(-1, 1, (9, 11)))
    B = np.asfortranarray(rng.uniform(-1, 1, (11, 7)))
    C0 = np.asfortranarray(rng.uniform(-1, 1, (9, 7)))
    full = C0.copy(order="F")
    O.ozaki_gemm(0.5, A, B, 2.0, full, s=6)
    base = np.zeros((9, 7), order="F")
    O.ozaki_gemm(1.0, A, B, 0.0, base, s=6)
    assert np.array_equal(full, (0.5 * base) + (2.0 * C0))
    sub = C0.copy(order="F")
    O.ozaki_gemm(0.5, A, B, 2.0, sub, s=6, rows=[1, 4])
    assert np.array_equal(sub[[1, 4]], full[[1, 4]])
    assert np.array_equal(np.delete(sub, [1, 4], 0), np.delete(C0, [1, 4], 0))


def test_beta_zero_never_reads_old_c():
    # beta = 0: C is output only, as in the plain product -- a NaN there does not propagate
    rng = np.random.default_rng(56)
    A = np.asfortranarray(rng.uniform(-1, 1, (6, 9)))
    B = np.asfortranarray(rng.uniform(-1, 1, (9, 5)))
    nan = np.full((6, 5), np.nan, order="F")
    O.ozaki_gemm(1.0, A, B, 0.0, nan, s=7)
    zero = np.zeros((6, 5), order="F")
    O.ozaki_gemm(1.0, A, B, 0.0, zero, s=7)
    assert np.array_equal(nan, zero)


def test_round_tf32_known_values():
    # TF32 keeps 10 mantissa bits: ulp(1) = 2^-10; 2^-11 is a tie, rounded away from zero
    assert O.round_tf32([1.0 + 2.0 ** -11])[0] == 1.0 + 2.0 ** -10
    assert O.round_tf32([-(1.0 + 2.0 ** -11)])[0] == -(1.0 + 2.0 ** -10)
    assert O.round_tf32([1.0 + 2.0 ** -12])[0] == 1.0
    assert O.round_tf32([1.0 + 3 * 2.0 ** -12])[0] == 1.0 + 2.0 ** -10
    assert O.round_tf32([0.0])[0] == 0.0
    rng = np.random.default_rng(56)
    x = rng.uniform(-1, 1, 1000)
    r = O.round_tf32(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -11 * 1.0001)
    # the result has at most 11 significant bits
    m, _ = np.frexp(r)
    assert np.all(m * 2 ** 11 == np.round(m * 2 ** 11))


@pytest.mark.parametrize("s", [3, 7, 8])
def test_recombination_is_exact_sum_rounded_once(s):
    # C = alpha * round(sum_d G_d 2^-7d) * 2^(e+f): with alpha = 1, beta = 0 each
    # C(i,j) must be the correctly rounded value of the exact rational sum
    # (Python's float(Fraction) rounds to nearest, ties to even)
    rng = np.random.default_rng(57 + s)
    M, K, N = 4, 40, 5
    A = np.asfortranarray(rng.uniform(-1, 1, (M, K)) * 10.0 ** rng.uniform(-3, 3, (M, K)))
    B = np.asfortranarray(rng.uniform(-1, 1, (K, N)) * 10.0 ** rng.uniform(-3, 3, (K, N)))
    e, f = O.ozaki_exponents(A, B)
    Cd, lv = O.ozaki_gemm(1.0, A, B, 0.0, np.zeros((M, N), order="F"), s=s, want_levels=True)
    for i in range(M):
        for j in range(N):
            exact = sum(Fraction(int(lv[d - 2][i][j])) * Fraction(2) ** (-7 * d) for d in range(2, s + 2))
            exact *= Fraction(2) ** (int(e[i]) + int(f[j]))
            assert Cd[i, j] == float(exact)


def _exact_scaled(S, k):
    """S * 2^k as Python rounds it (int / int and int -> float round to nearest, ties to even)."""
    try:
        return float(S << k) if k >= 0 else S / (1 << -k)
    except OverflowError:
        return math.copysign(math.inf, S)


def _bits(x):
    return np.array([x], np.float64).view(np.uint64)[0]


def test_round_scaled_matches_exact_rationals():
    rng = np.random.default_rng(58)
    cases = []
    for _ in range(3000):
        n = int(rng.integers(1, 127))
        S = int(rng.integers(1 << 30)) | (1 << (n - 1)) if n > 30 else int(rng.integers(1, 1 << n))
        S = (S << max(0, n - 31)) | int(rng.integers(0, 1 << min(n, 62))) if n > 30 else S
        S = S % (1 << 126) or 1
        if rng.random() < 0.5:
            S = -S
        # k around the normal range, the subnormal range and overflow
        lead = S.bit_length() - 1 if S > 0 else (-S).bit_length() - 1
        k = int(rng.choice([rng.integers(-1200, 1100) - lead, -1022 - lead - rng.integers(0, 60),
                            -1074 - lead + rng.integers(-3, 3), 1023 - lead + rng.integers(-1, 2)]))
        cases.append((S, k))
    # a tie created by rounding first to 53 bits and then again at the subnormal
    # precision: rounded once, the remainder below the last kept bit (2^76 of S)
    # is less than half of it, so the result is (2^23 + 1) 2^-1074
    S_dr = (1 << 99) + (1 << 76) + ((1 << 75) - (1 << 46))
    cases += [(S_dr, -1150), (-S_dr, -1150), (1, -1075), (3, -1075), (-1, -1076), (1, -1074),
              ((1 << 53) - 1, 971), ((1 << 54) - 1, 970), (1 << 126, -2000), (5, 0), (0, 3)]
    assert O.round_scaled(S_dr, -1150) == (2 ** 23 + 1) * 2.0 ** -1074
    for S, k in cases:
        got, want = O.round_scaled(S, k), _exact_scaled(S, k)
        assert _bits(got) == _bits(want), (S, k, got, want)


def _py_emulated_gemm(A, B, s):
    """The integer-slice emulation on tiny inputs with Python integers and
    fractions only: exponents from math.frexp of the line maxima, slices by
    truncation of the exact scaled values, level sums t + u <= s + 1, the exact
    sum S rounded once by Python's exact int / int division."""
    M, K = A.shape
    N = B.shape[1]
    e = [math.frexp(max(abs(float(v)) for v in A[i])) [1] if np.any(A[i]) else 0 for i in range(M)]
    f = [math.frexp(max(abs(float(v)) for v in B[:, j]))[1] if np.any(B[:, j]) else 0 for j in range(N)]

    def slices(x, ex):
        q = Fraction(float(x)) / Fraction(2) ** ex * (1 << (7 * s))
        a = int(abs(q))                        # truncation toward zero
        sg = -1 if q < 0 else 1
        return [sg * ((a >> (7 * (s - t))) & 127) for t in range(1, s + 1)]

    SA = [[slices(A[i, l], e[i]) for l in range(K)] for i in range(M)]
    SB = [[slices(B[l, j], f[j]) for j in range(N)] for l in range(K)]
    C = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            S = 0
            for d in range(2, s + 2):
                G = sum(SA[i][l][t - 1] * SB[l][j][d - t - 1] for l in range(K) for t in range(1, d) if d - t <= s)
                S += G << (7 * (s + 1 - d))
            C[i, j] = _exact_scaled(S, e[i] + f[j] - 7 * (s + 1))
    return C


@pytest.mark.parametrize("scale_a,scale_b", [(0, 0), (-560, -480), (-540, -520), (-700, -362), (-600, -500),
                                             (530, 500)])
def test_emulation_against_python_integers(scale_a, scale_b):
    # (0, 0): ordinary values; then results in the subnormal range (rounded at
    # the bit of weight 2^-1074), below it (signed zeros) and beyond the
    # largest double (infinities)
    rng = np.random.default_rng(59 + abs(scale_a))
    M, K, N, s = 3, 5, 4, 5
    A = np.asfortranarray(rng.uniform(-1, 1, (M, K)) * 2.0 ** scale_a)
    B = np.asfortranarray(rng.uniform(-1, 1, (K, N)) * 2.0 ** scale_b)
    got = np.zeros((M, N), order="F")
    O.ozaki_gemm(1.0, A, B, 0.0, got, s=s)
    want = _py_emulated_gemm(A, B, s)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    if -1074 < scale_a + scale_b < -1030:
        assert np.any((got != 0) & (np.abs(got) < 2.0 ** -1022))   # the subnormal range is exercised
    if scale_a + scale_b > 1024:
        assert np.any(np.isinf(got))


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_lines_give_nan(bad):
    # a NaN or an infinity in row i of A (column j of B) makes C's row i
    # (column j) NaN -- where IEEE FP64 gives a NaN or an infinity -- and leaves
    # every other element as it is without that line
    rng = np.random.default_rng(60)
    M, K, N = 6, 7, 5
    A = np.asfortranarray(rng.uniform(-1, 1, (M, K)))
    B = np.asfortranarray(rng.uniform(-1, 1, (K, N)))
    A[2, 3] = bad
    B[4, 1] = bad
    C0 = np.asfortranarray(rng.uniform(-1, 1, (M, N)))
    C0[0, 4] = np.nan                                   # an old NaN propagates where beta reads it
    for alpha, beta in ((1.0, 0.0), (0.5, 2.0), (0.0, 1.0)):
        got = C0.copy(order="F")
        O.ozaki_gemm(alpha, A, B, beta, got, s=7)
        with np.errstate(invalid="ignore"):
            ieee = A @ B
        poisoned = ~np.isfinite(ieee)
        assert poisoned[2].all() and poisoned[:, 1].all() and poisoned.sum() == N + M - 1
        want_nan = poisoned | (np.isnan(C0) if beta != 0.0 else False)
        assert np.array_equal(np.isnan(got), want_nan)
        A0, B0 = A.copy(order="F"), B.copy(order="F")
        A0[2, 3] = 0.0
        B0[4, 1] = 0.0
        clean = C0.copy(order="F")
        O.ozaki_gemm(alpha, A0, B0, beta, clean, s=7)
        keep = ~want_nan
        assert np.array_equal(got[keep], clean[keep])
    e, f = O.ozaki_exponents(A, B)
    assert e[2] == O.OZ_NONFINITE and f[1] == O.OZ_NONFINITE
    assert all(v != O.OZ_NONFINITE for q, v in enumerate(e) if q != 2)
