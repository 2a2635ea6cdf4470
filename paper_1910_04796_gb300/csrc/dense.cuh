// dense.cuh -- densification (Sec. III) and the dense GEMM kernels.
#pragma once
#include "internal.cuh"

namespace dbcsr {

// Write op(m) as a dense column-major array with leading dimension ld
// (zero-filled first when zero_first, so absent blocks read as 0).
int densify(const dbcsr_matrix_s* m, bool trans, double* dense, int64_t ld, bool zero_first);
// Fill every stored block of m from the dense column-major array.
int undensify(dbcsr_matrix_s* m, const double* dense, int64_t ld);

// C = alpha*A*B + beta*C, column-major FP64, on the FP64 tensor-core MMA.
int dgemm_fp64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
               int64_t ldb, double beta, double* C, int64_t ldc);

}  // namespace dbcsr
