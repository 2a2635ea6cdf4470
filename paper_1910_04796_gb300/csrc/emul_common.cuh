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

// slice t (1-based) of the fixed-point value q, as an exact bf16
__device__ __forceinline__ __nv_bfloat16 slice_bf16(long long q, int t, int s) {
    const unsigned long long a = (unsigned long long)(q < 0 ? -q : q);
    int v = (int)((a >> (7 * (s - t))) & 127ull);
    if (q < 0) v = -v;
    return __float2bfloat16_rn((float)v);   // |v| <= 127: exact
}

// frexp exponent of a magnitude given by its bit pattern (0 for zero)
__device__ __forceinline__ int exponent_of_bits(unsigned long long bits) {
    const double mu = __longlong_as_double((long long)bits);
    int ex = 0;
    if (mu != 0.0) frexp(mu, &ex);
    return ex;
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

}  // namespace emul
}  // namespace dbcsr
