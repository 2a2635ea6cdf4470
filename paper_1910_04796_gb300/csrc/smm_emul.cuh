// smm_emul.cuh -- what the two emulated-FP64 stack kernels share: the view of
// a stored block through op() used to cut it into slices, and the tcgen05
// variant's entry point.
#pragma once
#include "internal.cuh"
#include "smm.cuh"

namespace dbcsr {

// largest block edge the emulated stack kernels take (blocks are padded to 32
// x 32 on the tcgen05 kernel, to multiples of 16 up to 32 on the mma.sync one)
constexpr int EMUL_STACK_MAX_EDGE = 32;

// One matrix seen through op(): stored block b, element (x, l) of its op()
// "row-like" view is data[off[b] + x*xs + l*ls]: x indexes op(A)'s rows (or
// op(B)'s columns), l the inner dimension.
struct SliceGeom {
    const int* row_of;
    const int* col;
    const int64_t* off;
    const double* data;
    const int* rs;          // stored block row sizes
    const int* cs;          // stored block column sizes
    const int64_t* roff;    // stored element row offsets
    const int64_t* coff;    // stored element column offsets
    int64_t nblks;
    int x_is_row;           // x runs over the stored rows (else stored columns)
};

__device__ __forceinline__ void geom_block(const SliceGeom& G, int64_t b, int& X, int& L, int& xs, int& ls,
                                           int64_t& xbase) {
    const int sr = G.rs[G.row_of[b]], sc = G.cs[G.col[b]];
    if (G.x_is_row) {
        X = sr; L = sc; xs = 1; ls = sr; xbase = G.roff[G.row_of[b]];
    } else {
        X = sc; L = sr; xs = sr; ls = 1; xbase = G.coff[G.col[b]];
    }
}

inline SliceGeom slice_geom(dbcsr_matrix_s* M, bool x_is_row) {
    return SliceGeom{M->d_row_of, M->d_col, M->d_off, M->d_data, M->d_rs, M->d_cs, M->d_roff, M->d_coff,
                     M->nblks, x_is_row ? 1 : 0};
}

// frexp exponents of the maximum |x| of each op() line of M (element rows of
// op(A) when x_is_row describes op(A)'s rows, element columns of op(B)), from
// the stored blocks; nlines entries
int line_exponents(dbcsr_matrix_s* M, bool x_is_row, int64_t nlines, DBuf<int>& ex);

// tcgen05 variant (smm_emul_tc.cu): every block padded to 32 x 32; e, f are the
// exponents of op(A)'s element rows and op(B)'s element columns. issued_flops
// receives the tensor-core arithmetic issued (padded operand shapes).
bool smm_emul_tc_usable();
int smm_emul_tc(const SmmArgs& g, dbcsr_matrix_s* A, bool ta, dbcsr_matrix_s* B, bool tb, dbcsr_matrix_s* C,
                const int* e, const int* f, int s, int64_t nprod, double* issued_flops,
                const CRanges* ranges = nullptr);

}  // namespace dbcsr
