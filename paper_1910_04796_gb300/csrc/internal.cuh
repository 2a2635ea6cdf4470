// internal.cuh -- shared definitions of the GB300 block-sparse multiply library.
//
// Layout of one matrix in HBM (blocked CSR, Sec. II of the paper):
//   rs[nbr], cs[nbc]        block row / column sizes (int32)
//   roff[nbr+1], coff[nbc+1] element offsets of block rows / columns (int64)
//   rowptr[nbr+1]           CSR row pointers into the block arrays (int32)
//   col[nblks]              block column of each stored block (int32)
//   row_of[nblks]           block row of each stored block (int32)
//   off[nblks]              element offset of each block in data (int64)
//   data[nelems]            FP64, blocks in CSR order, each column-major
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/dbcsr_gb.h"

namespace dbcsr {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define DB_CUDA(call)                                                                 \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return ::dbcsr::fail(DBCSR_ERR_CUDA, std::string(#call) + ": " +          \
                                 cudaGetErrorString(e_) + " at " + __FILE__ + ":" +   \
                                 std::to_string(__LINE__));                           \
    } while (0)

// after every kernel launch: count it and surface launch errors
void count_launch();
// CUDA events around the dominant kernel of a multiply (no-ops unless timing)
void timer_kernel_begin();
void timer_kernel_end();
#define DB_KCHECK()                 \
    do {                            \
        ::dbcsr::count_launch();    \
        DB_CUDA(cudaGetLastError()); \
    } while (0)

#define DB_TRY(call)                    \
    do {                                \
        int r_ = (call);                \
        if (r_ != DBCSR_OK) return r_;  \
    } while (0)

// ---------------------------------------------------------------- context
struct Context {
    cudaStream_t stream = nullptr;
    dbcsr_alloc_fn alloc = nullptr;
    dbcsr_free_fn free = nullptr;
    void* alloc_ctx = nullptr;
    int device = -1;
    int num_sms = 0;
    int pool_ready = 0;
    // device scratch reused across calls (error flag, work counters)
    int* d_flags = nullptr;
    int64_t* d_counters = nullptr;
    // limit of each bounded wait in the tensor-core pipelines (dbcsr_set_wait_limit)
    uint64_t wait_ns = 4000000000ull;
    // uploads of matrix values from host memory run on their own stream, so
    // that they overlap the library stream's work (Sec. II: host-to-device
    // transfers double-buffered against computation with CUDA streams)
    cudaStream_t xfer = nullptr;
    cudaEvent_t order_ev = nullptr;   // library-stream point the next upload starts after
};
Context& ctx();
int ensure_device();

// stream-ordered device allocation through the configured allocator
int dev_alloc(void** p, size_t bytes);
void dev_free(void* p, size_t bytes);

template <class T>
int dalloc(T** p, size_t n) {
    return dev_alloc(reinterpret_cast<void**>(p), n * sizeof(T));
}
template <class T>
void dfree(T*& p, size_t n) {
    if (p) dev_free(p, n * sizeof(T));
    p = nullptr;
}

// Scoped device buffer (freed stream-ordered at scope exit).
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { reset(); }
    int alloc(size_t count) {
        reset();
        n = count;
        return dalloc(&p, count ? count : 1);
    }
    void reset() {
        if (p) dfree(p, n ? n : 1);
        p = nullptr;
        n = 0;
    }
    T* release() {
        T* q = p;
        p = nullptr;
        n = 0;
        return q;
    }
};

}  // namespace dbcsr

// ---------------------------------------------------------------- matrix
struct dbcsr_matrix_s {
    int nbr = 0, nbc = 0;
    int64_t nblks = 0, nelems = 0;
    std::vector<int> h_rs, h_cs;
    std::vector<int> u_rs, u_cs;   // distinct block sizes, ascending
    std::vector<int64_t> h_roff, h_coff;
    int max_rs = 0, max_cs = 0;
    int* d_rs = nullptr;
    int* d_cs = nullptr;
    int64_t* d_roff = nullptr;
    int64_t* d_coff = nullptr;
    int* d_rowptr = nullptr;
    int* d_col = nullptr;
    int* d_row_of = nullptr;
    int64_t* d_off = nullptr;
    double* d_data = nullptr;
    // lazily built column view (CSC) used for op = 'T'
    int* d_tptr = nullptr;   // [nbc+1]
    int* d_tidx = nullptr;   // [nblks] block row of each entry, column-sorted
    int* d_tpos = nullptr;   // [nblks] stored position of each entry
    bool t_valid = false;
    // lazily downloaded host mirror of the index
    bool h_valid = false;
    std::vector<int> h_rowptr, h_col;
    std::vector<int64_t> h_off;
    // with the host index: per block row the sum of its blocks' column sizes and
    // their count, per block column the sum of row sizes and the count
    std::vector<double> h_row_cs, h_col_rs;
    std::vector<int64_t> h_row_n, h_col_n;
    uint64_t version = 0;    // bumped whenever the pattern changes
    uint64_t uid = 0;
    void* plan = nullptr;    // reusable stack plan + CUDA graph (api.cu)
    // an upload of the values on the transfer stream that the library stream
    // has not been ordered after yet; `ready` is recorded when it completes
    cudaEvent_t ready = nullptr;
    bool pending = false;
};

namespace dbcsr {

// View of op(M) as block rows: entries of row i are [ptr[i], ptr[i+1]),
// each with block column idx[e] and stored block position pos[e]
// (pos == nullptr: identity). trans = 1 when the stored block is the
// transpose of the op() block.
struct OpView {
    const int* ptr;
    const int* idx;
    const int* pos;
    const int64_t* off;
    const double* data;
    const int* rs;   // sizes of op(M)'s block rows
    const int* cs;   // sizes of op(M)'s block columns
    int nrows, ncols;
    int64_t nentries;
    int trans;
};

int build_transpose_index(dbcsr_matrix_s* m);
OpView make_view(dbcsr_matrix_s* m, bool trans);

int download_index(dbcsr_matrix_s* m);
void free_index(dbcsr_matrix_s* m);  // index + data + caches, not sizes
// Order the library stream after a pending upload of m's values (no-op
// otherwise); every use of m->d_data on the library stream comes after it.
int await_data(dbcsr_matrix_s* m);

// ------------------------------------------------------------ primitives
// exclusive scan of n int64 values (in may alias out); total to *d_total (device, may be null)
int scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* d_total);
// exclusive scan of int32 counts into int32 output; returns through d_total (int64)
int scan_i32(const int* in, int* out, int64_t n, int64_t* d_total);
// stable LSD radix sort of (key, value) pairs by the low `bits` bits of key
int radix_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n, int bits);

// copy helpers
int h2d(void* dst, const void* src, size_t bytes);
int d2h(void* dst, const void* src, size_t bytes);
int sync_stream();

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// The BLAS update of a C element: alpha * x + beta * old, each product and
// the sum rounded once, in that order. A factor of exactly 1 is skipped --
// 1 * x == x for every double, so the result is the same -- which keeps the
// common alpha = 1 / beta = 1 updates off the narrow FP64 pipe. The tests on
// alpha and beta compare bit patterns (integer instructions: the compiler may
// re-evaluate them per element, and FP64 comparisons would take the FP64 pipe).
__device__ __forceinline__ unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    return 0ull;   // host pass of a device-only helper: never executed
#endif
}

struct BlasUpd {
    double alpha, beta;
    bool a1, b1, old;   // alpha == 1, beta == 1, beta != 0 (the old C is read)
    __device__ __forceinline__ BlasUpd(double a, double b)
        : alpha(a),
          beta(b),
          a1(dbits(a) == 0x3FF0000000000000ull),
          b1(dbits(b) == 0x3FF0000000000000ull),
          old((dbits(b) << 1) != 0ull) {}   // +-0: no old C
    // the general forms are calls: inlined, the compiler evaluates both arms
    // of the selects and the skipped multiplies still occupy the FP64 pipe
    __device__ __forceinline__ double scale(double x) const { return a1 ? x : scale_any(alpha, x); }
    __device__ __forceinline__ double update(double x, double c) const {
        return (a1 && b1) ? __dadd_rn(x, c) : update_any(alpha, x, beta, c, a1, b1);
    }
    static __device__ __noinline__ double scale_any(double alpha, double x) { return __dmul_rn(alpha, x); }
    static __device__ __noinline__ double update_any(double alpha, double x, double beta, double c, bool a1,
                                                     bool b1) {
        return __dadd_rn(a1 ? x : __dmul_rn(alpha, x), b1 ? c : __dmul_rn(beta, c));
    }
};

}  // namespace dbcsr
