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

// Stack path in emulated precision (same contract as smm_fp64_generic).
int smm_emulated(const SmmArgs& g, int max_m, int max_n, int max_k, const dbcsr_opts& o);

}  // namespace dbcsr
