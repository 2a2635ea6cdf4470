/*
 * dbcsr_gb.h -- C ABI of the GB300 (sm_103a) local block-sparse matrix product.
 *
 * The library computes, on one GPU,
 *
 *     C = alpha * op(A) * op(B) + beta * C,      op(X) in {X, X^T}
 *
 * for matrices stored in the blocked compressed sparse row layout that the
 * paper describes (Sivkov, Lazzaro, Hutter, "DBCSR: A Library for Dense Matrix
 * Multiplications on Distributed GPU-Accelerated Systems", Sec. II: "DBCSR
 * matrices are stored in a blocked compressed sparse row (CSR) format"; the
 * paper states that a C API is provided). Every stored block is a dense
 * sub-matrix, column-major (the library the paper describes is Fortran), of
 * size row_blk_sizes[i] x col_blk_sizes[j].
 *
 * The product is the paper's local multiplication (Sec. II): pairwise block
 * products A_ik * B_kj, organised in stacks of block products grouped by block
 * shape (m, n, k) and executed by batched small-matrix kernels; or, when both
 * operands are dense, the densified path of Sec. III (all blocks coalesced into
 * one large block, one GEMM, then the result split back into the original
 * block sizes).
 *
 * Conventions for every entry point:
 *   - Return value: DBCSR_OK (0) or a negative DBCSR_ERR_* code. The message of
 *     the last error on the calling thread is available from dbcsr_last_error().
 *     No C++ exception ever crosses this interface.
 *   - All GPU work is ordered on the stream given to dbcsr_init() (default: the
 *     legacy default stream), except the copies of matrix values from
 *     page-locked host memory made by dbcsr_create() and dbcsr_set_data():
 *     those run on a transfer stream of the library, so that they overlap
 *     work already queued (Sec. II: host-to-device transfers double-buffered
 *     against the computation with CUDA streams), and every later use of the
 *     matrix waits for its copy. Entry points that return host data synchronise the library
 *     stream before returning; dbcsr_sync() waits for both streams.
 *   - Device memory is obtained through the allocator set with
 *     dbcsr_set_allocator(), else from CUDA's stream-ordered pool
 *     (cudaMallocAsync on the library stream; freed blocks stay in the pool).
 *   - Matrices are opaque handles owned by the library; dbcsr_release() frees
 *     them. A handle may be used by one host thread at a time.
 *   - Sizes and counts are int64_t where they can exceed 2^31; block counts of
 *     one matrix must stay below 2^31 (DBCSR_ERR_OVERFLOW otherwise).
 */
#ifndef DBCSR_GB_H
#define DBCSR_GB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DBCSR_API __attribute__((visibility("default")))
#else
#define DBCSR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define DBCSR_OK            0
#define DBCSR_ERR_ARG      -1  /* invalid argument (NULL handle, bad trans char, bad index) */
#define DBCSR_ERR_DIM      -2  /* block grids or block sizes of A, B, C do not conform */
#define DBCSR_ERR_ALLOC    -3  /* the device allocator returned NULL */
#define DBCSR_ERR_OVERFLOW -4  /* a count exceeds what the index types can hold */
#define DBCSR_ERR_TIMEOUT  -5  /* a bounded device-side wait gave up */
#define DBCSR_ERR_CUDA     -6  /* a CUDA runtime call failed */
#define DBCSR_ERR_STATE    -7  /* library not initialised / no device */

typedef struct dbcsr_matrix_s *dbcsr_matrix;

/* Device allocator hooks. alloc returns device memory of `bytes` usable in
 * stream order on `stream` (a cudaStream_t), or NULL on failure. free releases
 * a pointer returned by alloc; `bytes` is the size that was requested. */
typedef void *(*dbcsr_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*dbcsr_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

/* Execution path of dbcsr_multiply (Sec. II stacks vs Sec. III densification). */
#define DBCSR_PATH_AUTO   0  /* dense path when op(A) and op(B) are 100% occupied (FP32:
                                always stacks; FP64 with every block edge up to 32: stacks,
                                measured faster there than the FP64 dense GEMM); else
                                stacks, except where the stack kernels do not apply:
                                emulated FP64 with a block edge above 32 and TF32 take the
                                dense path (Sec. II: blocks beyond the small kernels' range
                                go to a GEMM) */
#define DBCSR_PATH_STACKS 1  /* stacks of block products, batched small-GEMM kernels. FP64
                                and FP32: any block size. Emulated FP64: block edges up
                                to 32 (DBCSR_ERR_ARG above). TF32: none (DBCSR_ERR_ARG) */
#define DBCSR_PATH_DENSE  2  /* densify, one GEMM, undensify (any occupancy; absent blocks = 0) */
#define DBCSR_PATH_HYBRID 3  /* per panel of block rows of op(A): densified GEMM where the panel
                                (and op(B)) is at least hybrid_fill_pct % occupied, stacks elsewhere
                                (Sec. III's densification applied to parts of a sparse matrix) */

/* Arithmetic of the multiply. */
#define DBCSR_PREC_FP64  0   /* IEEE FP64 products and sums (DFMA / DMMA) */
#define DBCSR_PREC_OZAKI 1   /* FP64 emulated with 7-bit integer slices on the tensor cores,
                                exact integer accumulation, FP64 recombination */
#define DBCSR_PREC_TF32  2   /* inputs rounded to TF32, FP32 accumulation (error reported only) */
#define DBCSR_PREC_FP32  3   /* single precision (Sec. II: the library accepts single): inputs rounded
                                to FP32, FP32 products and sums (FMA), alpha/beta in FP64; stack
                                path only (the dense path offers TF32) */

typedef struct {
    int path;          /* DBCSR_PATH_*                                        */
    int precision;     /* DBCSR_PREC_*                                        */
    int ozaki_slices;  /* slices per operand for DBCSR_PREC_OZAKI; 0 = default (7) */
    int kernel;        /* FP64 stack kernel: 0 = per-shape tables set with
                          dbcsr_set_tuning_mnk and dbcsr_set_tuning (variant
                          0 for untuned shapes);
                          v = 1..4 forces variant v-1 for every block:
                          0: one warp per C block;
                          1: the same as 0 (kept for tables that name it);
                          2: two warps per C block (products split);
                          3: four warps per C block.
                          Every C block of a multiply runs in one launch.
                          Emulated-FP64 stack kernel: 0 = tcgen05 when the mean
                          block edge is at least 12, else mma.sync; 1 = mma.sync
                          (blocks padded to 16); 2 = tcgen05 (blocks padded to
                          32 x 32, fp32 accumulators in tensor memory).
                          Emulated-FP64 dense GEMM: 0 = 128 x 256 output
                          tiles, one CTA each (128 x 128 when N < 256); 4 =
                          256 x 256 tiles on pairs of CTAs where M and N reach
                          256 (same results bit for bit)                   */
    int timing;        /* nonzero: time the phases with CUDA events on the
                          library stream (reported by dbcsr_get_stats)        */
    int reuse_plan;    /* nonzero (FP64 stack path): keep this multiply's stack
                          plan with C and capture its product kernel in a CUDA
                          graph; a later multiply of the same A and B handles
                          (patterns unchanged, values may change), same op(),
                          alpha and beta, into the C it produced, skips stack
                          generation and replays the graph, updating C in place */
    int hybrid_panel;  /* DBCSR_PATH_HYBRID: block rows per panel; 0 = about 1024 element rows */
    int hybrid_fill_pct; /* DBCSR_PATH_HYBRID: occupancy (percent of elements) from which a panel
                            is densified; 0 = 50                                   */
} dbcsr_opts;

/* Statistics of the last dbcsr_multiply on the calling thread. */
typedef struct {
    int64_t n_products;      /* block products (stack entries)                   */
    int64_t n_stacks;        /* stacks of <= 30000 entries per (m,n,k) shape      */
    int64_t n_shapes;        /* distinct (m,n,k) shapes                           */
    int64_t c_blocks;        /* blocks in the result C                            */
    double useful_flops;     /* sum over block products of 2*m*n*k                */
    int path;                /* path taken (DBCSR_PATH_STACKS or _DENSE)          */
    int precision;           /* precision used                                    */
    int kernel_launches;     /* kernels this library launched during the call     */
    int dense_panels;        /* DBCSR_PATH_HYBRID: panels computed densely        */
    /* with dbcsr_opts.timing: milliseconds per phase, CUDA events on the stream */
    float ms_setup;          /* stack generation, or densification of A, B, C    */
    float ms_main;           /* the product kernels (batched small GEMM / GEMM)   */
    float ms_finish;         /* undensification / index hand-over                 */
    float ms_total;          /* whole call                                        */
    double main_flops;       /* arithmetic the main kernels executed (2*M*N*K per
                                GEMM issued, incl. slices / padding)             */
    double main_bytes;       /* algorithmic HBM bytes of the main kernels         */
    float ms_kernel;         /* the dominant kernel alone (GEMM / batched SMM)    */
    float reserved_f;
} dbcsr_stats;

/* Select the stream (a cudaStream_t, may be NULL for the legacy default
 * stream) on which all following work is ordered, and the current CUDA
 * device. Call once before anything else; may be called again to switch.
 * (Sec. III: the GPU execution keeps one library context per thread -- the
 * paper initialises a cuBLAS context once per thread and draws buffers from
 * memory pools; here the context is the stream, the device and the pool.) */
DBCSR_API int dbcsr_init(void *cuda_stream);

/* Route device allocations through the given hooks (NULL, NULL restores the
 * built-in stream-ordered pool). Every allocation is later returned to the
 * hook (or pool) that made it, so the hooks may be switched at any time; the
 * hook's ctx must stay valid while memory it allocated is alive. (Sec. III:
 * the GPU execution draws its buffers from memory pools; here the pool can be
 * the caller's.) */
DBCSR_API int dbcsr_set_allocator(dbcsr_alloc_fn alloc, dbcsr_free_fn free_fn, void *ctx);

/* Create a matrix (Sec. II: a blocked CSR matrix with per-row and per-column
 * block sizes).
 *   nblkrows, nblkcols  : block grid (>= 0)
 *   row_blk_sizes       : host int32[nblkrows], each >= 1
 *   col_blk_sizes       : host int32[nblkcols], each >= 1
 *   nblks               : number of stored blocks (>= 0)
 *   blk_row, blk_col    : host int32[nblks], block coordinates in any order,
 *                         no duplicates (DBCSR_ERR_ARG on a duplicate or an
 *                         out-of-range coordinate)
 *   data                : the blocks' values concatenated in the order of
 *                         blk_row/blk_col, each block column-major; host
 *                         memory if data_on_device == 0, device memory
 *                         otherwise; NULL creates all-zero blocks
 * The library copies everything; the caller keeps ownership of its arrays.
 * Host values in CSR order from page-locked (pinned) memory are copied on the
 * library's transfer stream: the call returns while they copy, the matrix's
 * next use waits for the copy, and `data` must stay unchanged until a call
 * that synchronises has returned (dbcsr_sync(), dbcsr_release() of the
 * matrix, or any call that returns the matrix's values to the host). From pageable memory the copy is complete
 * when the call returns.
 * Blocks are stored in CSR order (row, then column ascending). */
DBCSR_API int dbcsr_create(dbcsr_matrix *out, int nblkrows, int nblkcols,
                 const int *row_blk_sizes, const int *col_blk_sizes,
                 int64_t nblks, const int *blk_row, const int *blk_col,
                 const double *data, int data_on_device);

/* Free a matrix and set *m to NULL. NULL or *m == NULL is a no-op. Its device
 * memory returns to the pool it came from (Sec. III: memory-pool buffers on
 * the GPU reduce the time spent in allocations). A copy of its values from
 * page-locked host memory still in flight is waited for first, so the
 * caller may free that memory once this call returns. */
DBCSR_API int dbcsr_release(dbcsr_matrix *m);

/* Block grid, number of stored blocks and of stored elements of a matrix in
 * the blocked CSR format of Sec. II (block rows and columns of the grid, the
 * stored blocks of the index). Any output pointer may be NULL. */
DBCSR_API int dbcsr_get_info(dbcsr_matrix m, int *nblkrows, int *nblkcols, int64_t *nblks,
                   int64_t *nelems);

/* Block index in storage (CSR) order, to host arrays of length nblks:
 * block row, block column, element offset of the block in the data array.
 * Any output pointer may be NULL. (Sec. II: the blocked CSR index of the
 * stored blocks, each a dense sub-matrix at an offset of the data array.) */
DBCSR_API int dbcsr_get_index(dbcsr_matrix m, int *blk_row, int *blk_col, int64_t *blk_off);

/* All stored values in storage order (nelems doubles) to `out`, which is host
 * memory if out_on_device == 0 and device memory otherwise. (Sec. II: the
 * blocks' values, each block column-major, concatenated in CSR order.) */
DBCSR_API int dbcsr_get_data(dbcsr_matrix m, double *out, int out_on_device);

/* Overwrite all stored values (nelems doubles, storage order) from `data`,
 * host memory if data_on_device == 0, else device memory. The pattern is
 * unchanged, so a kept stack plan (dbcsr_opts.reuse_plan) stays valid. Host
 * values are copied as in dbcsr_create() (from page-locked memory on the
 * transfer stream: `data` must stay unchanged until a call that synchronises
 * has returned); device values are copied before the call returns. (Sec. II:
 * the blocks' values in CSR order, as dbcsr_get_data returns them.) */
DBCSR_API int dbcsr_set_data(dbcsr_matrix m, const double *data, int data_on_device);

/* Device pointer of the stored values (valid until the next call that changes
 * the matrix) -- for callers that keep data resident on the GPU. A copy of
 * host values still in flight is waited for before the call returns. (Sec. II:
 * the data array of the blocked CSR format.) */
DBCSR_API int dbcsr_data_ptr(dbcsr_matrix m, double **dev_ptr);

/* Copy block (row, col) to host `out_colmajor` (row_blk_size x col_blk_size
 * doubles, column-major). *found = 1 if the block is stored, else 0 and `out`
 * is left untouched. DBCSR_ERR_ARG for coordinates outside the grid.
 * (Sec. II: a matrix is a set of small dense blocks stored in blocked CSR
 * form; this reads one of them back, with absent blocks meaning zero.) */
DBCSR_API int dbcsr_get_block(dbcsr_matrix m, int row, int col, double *out_colmajor, int *found);

/* C = alpha * op(A) * op(B) + beta * C (Sec. II local multiplication; Sec. III
 * densification when the dense path is taken).
 *   transa, transb : 'N' (op = identity), 'T' or 'C' (op = transpose; for real
 *                    data 'C' equals 'T')
 *   A, B, C        : existing matrices; C must have block rows = those of
 *                    op(A), block columns = those of op(B), and the inner
 *                    block sizes of op(A) and op(B) must agree one by one
 *                    (DBCSR_ERR_DIM otherwise). C must differ from A and B.
 *   opts           : NULL = DBCSR_PATH_AUTO, DBCSR_PREC_FP64.
 * The result pattern is the set of (i,j) reached by at least one block
 * product, united with C's old pattern when beta != 0. With beta == 0 the old
 * C values are never read (NaN in them does not propagate). Blocks whose
 * value cancels to zero stay stored. C's index and data are replaced. */
DBCSR_API int dbcsr_multiply(char transa, char transb, double alpha, dbcsr_matrix A, dbcsr_matrix B,
                   double beta, dbcsr_matrix C, const dbcsr_opts *opts);

/* Statistics of the last dbcsr_multiply of this thread: block products,
 * stacks, shapes, the path taken and phase times (Sec. IV-B compares the
 * blocked and densified runs by their numbers of stacks and their times). */
DBCSR_API int dbcsr_get_stats(dbcsr_stats *out);

/* Per-shape choice of the FP64 stack kernel (the paper's LIBCUSMM is
 * auto-tuned per (m, n, k); Sec. II). count entries: C blocks of size
 * m[q] x n[q] (1..128) use variant[q] (0..3, see dbcsr_opts.kernel).
 * Replaces the previous table; count = 0 clears it. Host arrays. */
DBCSR_API int dbcsr_set_tuning(const int *m, const int *n, const int *variant, int count);

/* Per-(m, n, k) choice of the FP64 stack kernel, over the (m, n) table of
 * dbcsr_set_tuning (Sec. II: LIBCUSMM's kernels are tuned per block shape
 * m, n, k). count entries: a C block of size m[q] x n[q] whose first product
 * has inner size k[q] (all 1..32) uses variant[q] (0..3). C blocks of shapes
 * without an entry fall back to the (m, n) table. Replaces the previous
 * (m, n, k) table; count = 0 clears it. Host arrays; DBCSR_ERR_ARG for NULL
 * arrays with count > 0 or an entry out of range (the table is then left as
 * it was). The tables reach the GPU once per change, before the next
 * multiply that reads them. */
DBCSR_API int dbcsr_set_tuning_mnk(const int *m, const int *n, const int *k, const int *variant, int count);

/* The stack list of Sec. II (Traversal + Generation), as the GPU builds it
 * for op(A) * op(B): one entry per block product, 7 int32 each:
 *   stack id, m, n, k, block row i, block column j, inner block index k.
 * Canonical order: shape (m, n, k) ascending, then i, j, k ascending. A stack
 * is a run of one shape, cut every `stack_cap` entries (the paper's batches
 * hold at most 30'000 multiplications; stack_cap <= 0 means 30000).
 * out: host int32[7*cap]; *n_out receives the number of entries. When
 * out == NULL or cap < *n_out only the count is returned. */
DBCSR_API int dbcsr_get_stacks(char transa, char transb, dbcsr_matrix A, dbcsr_matrix B, int stack_cap,
                     int *out, int64_t cap, int64_t *n_out);

/* Allocation-free emulated-FP64 dense GEMM. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- for
 * example applications whose device memory is entirely owned by another
 * allocator (a framework that reserved the HBM up front), or code that must
 * not perform the device-wide synchronisation cudaMalloc/cudaFree may imply.
 *
 * Computes C = alpha*A*B + beta*C with the same emulation as
 * DBCSR_PREC_OZAKI (7-bit integer slices on the tensor cores, exact integer
 * level sums, FP64 recombination); results are identical to the dense path of
 * dbcsr_multiply with that precision.
 *   M, N, K        : sizes (>= 0); A is M x K, B is K x N, C is M x N
 *   A, B, C        : DEVICE pointers, column-major, leading dimensions
 *                    lda >= M, ldb >= K, ldc >= M; owned by the caller
 *   slices         : 1..8, 0 = 7
 *   stream         : cudaStream_t the work is ordered on; the call returns
 *                    after that stream has finished it
 * Scratch comes from one fixed 128 MiB device array inside the library
 * (every GPU that loads the library holds it until the process exits); the
 * call allocates nothing. Sizes whose scratch exceeds it (about
 * M = N = K = 1024 with 7 slices) return DBCSR_ERR_OVERFLOW with a message.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture begins. Every call
 * waits for its stream to finish the work before it returns. All calls share
 * the array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it, so callers serialise them. */
DBCSR_API int dbcsr_dgemm_emulated_noalloc(int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                                           int64_t lda, const double *B, int64_t ldb, double beta, double *C,
                                           int64_t ldc, int slices, void *stream);

/* Limit, in nanoseconds, of each bounded wait inside the tensor-core
 * pipelines (the emulated-FP64 and TF32 GEMMs and the emulated stack kernel);
 * ns <= 0 restores the default of 4 s. The paper has no counterpart: the
 * kernels' stages hand work to each other through shared-memory barriers,
 * and a wait that runs out makes the kernel stop every role, wait (always up
 * to 4 s) for its own copies and tensor-core operations in flight, release
 * its tensor memory and return; the call then fails with DBCSR_ERR_TIMEOUT
 * and the library stays usable. A limit far below the pipeline's normal
 * latency (a few microseconds) makes multiplies fail that way on purpose,
 * which is what the failure tests use it for. Applies to calls made after it
 * on any thread; not to dbcsr_dgemm_emulated_noalloc (fixed 4 s). */
DBCSR_API int dbcsr_set_wait_limit(int64_t ns);

/* Wait for all work the library queued on its stream and its transfer stream
 * (Sec. II: the GPU work and the host-device transfers are ordered on CUDA
 * streams). */
DBCSR_API int dbcsr_sync(void);

/* Message of the last error on the calling thread ("" if none). The paper has
 * no counterpart: it is the error channel of this C ABI. */
DBCSR_API const char *dbcsr_last_error(void);

/* Library version string. The paper has no counterpart. */
DBCSR_API const char *dbcsr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DBCSR_GB_H */
