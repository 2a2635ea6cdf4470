// emul_common.cuh -- device helpers of the emulated-FP64 product shared by
// the dense (emul.cu) and block-sparse (smm_emul.cu) paths.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace dbcsr {
namespace emul {

// floor(|x| 2^(7s - e)) with the sign of x, from the bit pattern of x
// (integer operations only). |x| 2^-e < 1 guarantees the result is below
// 2^(7s) <= 2^56. Its 7-bit groups, most significant first, are the slices
// sigma_1 .. sigma_s of x 2^-e obtained by repeated truncation.
__device__ __forceinline__ long long fixed_point(double x, int e, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    unsigned long long m = b & 0xfffffffffffffull;
    int E;   // |x| = m * 2^E
    if (ex == 0) {
        E = -1074;
    } else {
        m |= 1ull << 52;
        E = ex - 1075;
    }
    const int sh = E - e + 7 * s;
    unsigned long long q;
    if (m == 0) q = 0;
    else if (sh >= 0) q = m << sh;
    else if (sh > -64) q = m >> (-sh);
    else q = 0;
    return (b >> 63) ? -(long long)q : (long long)q;
}

// slice t (1-based) of the fixed-point value q, as an exact bf16. The integer
// v (|v| <= 127) becomes a float without the quarter-rate conversion unit:
// the bit pattern of 1.5 * 2^23 plus v is the float 1.5 * 2^23 + v (ulp 1 in
// [2^23, 2^24) for |v| < 2^22), and subtracting 1.5 * 2^23 is exact. v has at
// most 7 significant bits, so the float's upper half is its exact bf16.
__device__ __forceinline__ __nv_bfloat16 slice_bf16(long long q, int t, int s) {
    const unsigned long long a = (unsigned long long)(q < 0 ? -q : q);
    int v = (int)((a >> (7 * (s - t))) & 127ull);
    if (q < 0) v = -v;
    const float fv = __int_as_float(0x4B400000 + v) - 12582912.0f;
    return __ushort_as_bfloat16((unsigned short)(__float_as_uint(fv) >> 16));
}

// Exponent marker of a line (row of op(A) / column of op(B)) that holds a NaN
// or an infinity: the line has no finite maximum to scale by. Its slices come
// out zero (the shift in fixed_point is far below -64) and every C element of
// the line is NaN. Real exponents lie in [-1073, 1024], so a sum e_i + f_j
// above NONFINITE_EXP / 2 means that one of the two lines is marked.
constexpr int NONFINITE_EXP = 1 << 20;

// frexp exponent of a magnitude given by its bit pattern (0 for zero;
// NONFINITE_EXP for an infinity or a NaN, whose patterns are the largest)
__device__ __forceinline__ int exponent_of_bits(unsigned long long bits) {
    if (bits >= 0x7ff0000000000000ull) return NONFINITE_EXP;
    const double mu = __longlong_as_double((long long)bits);
    int ex = 0;
    if (mu != 0.0) frexp(mu, &ex);
    return ex;
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// |S| 2^k with the sign for a result below the normal range: rounded once, to
// nearest with ties to even, at the bit of weight 2^-1074 (bit d = -1074 - k
// of |S|, d > msb - 52; for d <= 0 every bit is kept and |S| < 2^52). The kept
// integer q is at most 2^52, so it is the double's bit pattern as it stands
// (q = 2^52 is the smallest normal). A call of its own: inlined, the rare
// branch would cost every element registers.
static __device__ __noinline__ double round_subnormal(unsigned long long hi, unsigned long long lo, int k,
                                                      bool neg) {
    const int d = -1074 - k;
    unsigned long long q = 0;
    if (d <= 0) {
        q = lo << (-d);
    } else if (d < 128) {
        const unsigned __int128 a = ((unsigned __int128)hi << 64) | lo;
        q = (unsigned long long)(a >> d);
        const unsigned __int128 rem = a - ((unsigned __int128)q << d);
        const unsigned __int128 half = (unsigned __int128)1 << (d - 1);
        if (rem > half || (rem == half && (q & 1ull))) q += 1;
    }   // d >= 128: |S| < 2^127 <= half of the last bit: zero
    return __longlong_as_double((long long)(((unsigned long long)neg << 63) | q));
}

// Recombination of the level sums: S = sum_d G_d 2^(7(s+1-d)) is an exact
// 128-bit integer; the result is the real number S 2^k rounded once to FP64
// (to nearest, ties to even): 53 significant bits when it is normal, down to
// the bit of weight 2^-1074 when it is subnormal, +-infinity beyond the
// largest double. Integer operations only.
__device__ __forceinline__ double round_i128_scaled(__int128 S, int k) {
    if (S == 0) return 0.0;
    const bool neg = S < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-S) : (unsigned __int128)S;
    const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
    const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);   // leading one
    if (msb + k < -1022) return round_subnormal(hi, lo, k, neg);
    unsigned long long mant;   // significand in [2^52, 2^53)
    int ex;                    // |S| rounded = mant * 2^ex
    if (msb <= 52) {
        mant = lo << (52 - msb);
        ex = msb - 52;
    } else {
        // drop d = msb - 52 low bits; 64-bit shifts only (a variable 128-bit
        // shift costs a branchy sequence). mant < 2^53 in both cases.
        const int d = msb - 52;
        bool up;
        if (d < 64) {
            mant = (hi << (64 - d)) | (lo >> d);
            const unsigned long long rem = lo & ((1ull << d) - 1ull), half = 1ull << (d - 1);
            up = rem > half || (rem == half && (mant & 1ull));
        } else {
            const int e = d - 64;   // 0 .. 63
            mant = hi >> e;
            const unsigned long long rh = e ? (hi & ((1ull << e) - 1ull)) : 0ull;
            // half = 2^(d-1): in the high word when d > 64, else the top bit of the low word
            bool gt, eq;
            if (e == 0) {
                gt = lo > (1ull << 63);
                eq = lo == (1ull << 63);
            } else {
                const unsigned long long hh = 1ull << (e - 1);
                gt = rh > hh || (rh == hh && lo != 0ull);
                eq = rh == hh && lo == 0ull;
            }
            up = gt || (eq && (mant & 1ull));
        }
        ex = d;
        if (up) {
            mant += 1;
            if (mant >> 53) {   // carried into a new power of two
                mant >>= 1;
                ex += 1;
            }
        }
    }
    const int E = ex + k + 52;   // result = mant / 2^52 * 2^E, E >= -1022 here
    if (E > 1023) return __longlong_as_double((long long)(((unsigned long long)neg << 63) | 0x7ff0000000000000ull));
    const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)(E + 1023) << 52) |
                                    (mant & 0xfffffffffffffull);
    return __longlong_as_double((long long)bits);
}

// The recombined value of one C element: S 2^(ef - shift) rounded once, with
// ef = e_i + f_j; NaN when either line holds a non-finite value.
__device__ __forceinline__ double recombined(__int128 S, int ef, int shift) {
    if (ef > NONFINITE_EXP / 2) return __longlong_as_double(0x7ff8000000000000ll);
    return round_i128_scaled(S, ef - shift);
}

}  // namespace emul
}  // namespace dbcsr
