// emul.cuh -- emulated-FP64 (integer slices on the tensor cores) and TF32 paths.
#pragma once
#include "internal.cuh"
#include "smm.cuh"

namespace dbcsr {

// Dense C = alpha*A*B + beta*C (column-major FP64 in and out) computed in the
// precision o.precision selects (DBCSR_PREC_OZAKI or DBCSR_PREC_TF32).
// main_flops (optional): tensor-core arithmetic issued (all slice GEMMs, padded tiles).
int dgemm_emulated(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double beta, double* C, int64_t ldc, const dbcsr_opts& o, double* main_flops);

// Emulated-FP64 product of fully occupied block matrices without densifying:
// slices are cut straight from op(A)'s and op(B)'s blocks, and the result is
// recombined straight into C's storage, which must already be the fully
// occupied layout (blocks in CSR order) holding the old values when beta != 0.
// Only where ozaki_blocks_ok(N) (the 256-wide slice GEMMs).
bool ozaki_blocks_ok(int64_t N);
// kernel: dbcsr_opts.kernel (4 = 256 x 256 tiles on CTA pairs instead of 128 x 256 tiles, one CTA each)
int dgemm_ozaki_blocks(dbcsr_matrix_s* A, bool ta, dbcsr_matrix_s* B, bool tb, dbcsr_matrix_s* C, double alpha,
                       double beta, int s, double* main_flops, int kernel);

// TF32 dense product of fully occupied operands with one block size per
// dimension, written straight into C's block storage (no dense copies);
// tf32_blocks_ok: whether it applies (N >= 256, the 256-wide kernel usable)
bool tf32_blocks_ok(const dbcsr_matrix_s* A, const dbcsr_matrix_s* B, int64_t N);
int dgemm_tf32_blocks(dbcsr_matrix_s* A, bool ta, dbcsr_matrix_s* B, bool tb, dbcsr_matrix_s* C, double alpha,
                      double beta, double* main_flops);

// TF32 variant of the dense GEMM (tf32.cu).
int dgemm_tf32(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
               int64_t ldb, double beta, double* C, int64_t ldc, double* main_flops);

// Stack path in emulated FP64 (same contract as smm_fp64_generic); A, B are
// the stored operands (op() given by ta, tb), C the result matrix whose sizes
// and offsets describe the new blocks. Blocks up to 32 x 32. nprod: products
// computed; main_flops (optional): tensor-core arithmetic issued. ranges
// (optional): only the plan's C blocks [first, second) of each range (the
// operands are cut into slices once for all of them).
int smm_emulated(const SmmArgs& g, dbcsr_matrix_s* A, bool ta, dbcsr_matrix_s* B, bool tb, dbcsr_matrix_s* C,
                 const dbcsr_opts& o, int64_t nprod, double* main_flops, const CRanges* ranges = nullptr);

}  // namespace dbcsr
