// stackgen.cuh -- result pattern and product (stack) list of one multiply.
#pragma once
#include "internal.cuh"

namespace dbcsr {

// C's new index and the product list, grouped by C block (CSR order of C),
// each C block's products in ascending inner block index k.
struct StackPlan {
    int nbr = 0, nbc = 0;
    int64_t nC = 0;          // blocks of the result
    int64_t nelem = 0;       // elements of the result
    int64_t nprod = 0;       // block products
    int64_t aentries = 0;    // entries of the op(A) view
    int* c_rowptr = nullptr; // [nbr+1]
    int* c_col = nullptr;    // [nC]
    int* c_row = nullptr;    // [nC]
    int64_t* c_off = nullptr;   // [nC] element offset in the new data
    int* c_old = nullptr;    // [nC] stored position in the old C, -1 if none
    int64_t* c_pstart = nullptr;  // [nC+1] product range of each C block
    int2* prod = nullptr;    // [nprod] (stored position in A, stored position in B)
    void reset();
    ~StackPlan() { reset(); }
};

int build_stacks(const OpView& A, const OpView& B, const dbcsr_matrix_s* oldC, const int* d_rsC,
                 const int* d_csC, StackPlan& P);
int export_stacks(const OpView& A, const StackPlan& P, const int* d_rsC, const int* d_csC,
                  const std::vector<int>& h_sizes_all, int stack_cap, int* h_out, int64_t* n_stacks,
                  int64_t* n_shapes);

}  // namespace dbcsr
