// smm.cuh -- arguments of the batched small-matrix product kernels.
#pragma once
#include <utility>
#include <vector>

#include "internal.cuh"

namespace dbcsr {

// One launch covers every C block of the plan: C block cb = (c_row, c_col) at
// element offset c_off, its products prod[c_pstart[cb] .. c_pstart[cb+1]).
struct SmmArgs {
    int64_t nC;
    const int* c_row;
    const int* c_col;
    const int64_t* c_off;
    const int* c_old;          // stored position in old C, -1 none (nullptr: no old C)
    const int64_t* c_pstart;
    const int2* prod;
    OpView A, B;               // op(A), op(B); off[] has a sentinel entry at nblks
    const int* rsC;
    const int* csC;
    double* Cd;                // new C data
    const double* Cold;        // old C data (beta != 0)
    const int64_t* Cold_off;
    double alpha, beta;
    unsigned long long* counter;  // zeroed work counter
    const float* A32;          // FP32 copies of op(A)'s and op(B)'s stored data (FP32 path only)
    const float* B32;
};

// ranges [first, second) of a plan's C blocks
using CRanges = std::vector<std::pair<int64_t, int64_t>>;

// FP64 stack-kernel variants (the autotuner's search space), see smm_fp64.cu
constexpr int SMM_NUM_VARIANTS = 4;

// variant 0 over every C block
int smm_fp64_generic(const SmmArgs& g, int max_mn);
// kernel = 0: the tuning tables (variant 0 where untuned); kernel = v >= 1:
// variant v-1. team_bound: the largest team index (0: one warp, 1: two, 2:
// four) the tables can give these C blocks (smm_table_team_bound); with 0 the
// table path launches the one-warp kernel directly.
int smm_fp64_dispatch(const SmmArgs& g, int max_mn, int kernel, int team_bound = 2);
// Largest team index the tuning tables give a C block of m in ms, n in ns whose
// products have inner sizes in ks (host check, conservative: 2 when unsure)
int smm_table_team_bound(const std::vector<int>& ms, const std::vector<int>& ns, const std::vector<int>& ks);
// (m, n) -> variant entries of the tuning table (replaces the table)
int smm_set_table(const int* m, const int* n, const int* variant, int count);
// (m, n, k) -> variant entries, m, n, k in 1..32 (replaces that table; count 0 clears it)
int smm_set_table_mnk(const int* m, const int* n, const int* k, const int* variant, int count);

// FP32 stack kernels over every C block (g.A32, g.B32 set), one warp per C
// block; max_edge: the largest block edge of op(A) and op(B)
int smm_fp32_dispatch(const SmmArgs& g, int max_mn, int max_edge);
// FP64 -> FP32 copy, round to nearest even
int to_f32(const double* in, int64_t n, float* out);

}  // namespace dbcsr
