// dense.cuh -- densification (Sec. III) and the dense GEMM kernels.
#pragma once
#include "internal.cuh"

namespace dbcsr {

// Write op(m) as a dense column-major array with leading dimension ld
// (zero-filled first when zero_first, so absent blocks read as 0).
int densify(const dbcsr_matrix_s* m, bool trans, double* dense, int64_t ld, bool zero_first);
// Fill every stored block of m from the dense column-major array.
int undensify(dbcsr_matrix_s* m, const double* dense, int64_t ld);

// Block rows [lo, hi) of op(m) into a dense column-major array (leading
// dimension ld), the first element row of block row lo at dense row `at`;
// only stored blocks are written (the caller zero-fills the array first).
int densify_rows(const dbcsr_matrix_s* m, bool trans, int lo, int hi, double* dense, int64_t ld, int64_t at);
// Fill blocks b0..b1-1 of an index (row_of, col, off into data; sizes and
// offsets of `shape`) from a dense array whose row 0 is element row `base`.
int undensify_blocks(int64_t b0, int64_t b1, const int* row_of, const int* col, const int64_t* off, double* data,
                     const dbcsr_matrix_s* shape, const double* dense, int64_t ld, int64_t base);

// C = alpha*A*B + beta*C, column-major FP64, on the FP64 tensor-core MMA.
int dgemm_fp64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
               int64_t ldb, double beta, double* C, int64_t ldc);

}  // namespace dbcsr
