/*
 * dbcsr_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, slow, obviously correct CPU statement of what the GPU library
 * computes, written from the paper (Sivkov, Lazzaro, Hutter: "DBCSR: A Library
 * for Dense Matrix Multiplications on Distributed GPU-Accelerated Systems").
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg and
 * reference arm (the oracle timed on the host cores) may load it. It shares no
 * code, header or table with the CUDA library.
 *
 * What it states:
 *   - the local block-sparse product C = alpha*op(A)*op(B) + beta*C on the
 *     blocked-CSR layout: "pairwise multiplications of small dense matrix
 *     blocks, (m x k) for A blocks and (k x n) for B blocks" (Sec. II);
 *   - the stack list of Sec. II (Traversal / Generation: batches of at most
 *     30'000 block multiplications), in one canonical order;
 *   - a double-double (Dot2, Ogita-Rump-Oishi 2005) accumulation mode used as
 *     the near-exact reference for the precision studies;
 *   - the INT8-slice emulation of FP64 (Ozaki et al. 2012 scheme, integer form)
 *     step by step, so the GPU's emulated path can be checked slice by slice.
 *
 * Arithmetic: IEEE FP64, compiled with -ffp-contract=off so every a*b+c is a
 * rounded product followed by a rounded sum, in the order written.
 * Intra-block storage is column-major (the library is Fortran, Sec. II).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One matrix as the tests hand it over: a block index in any order and the
 * blocks' data concatenated in that same order, each block column-major. */
typedef struct {
    int nbr, nbc;              /* number of block rows / block columns        */
    const int *rs, *cs;        /* block row sizes [nbr], block col sizes [nbc] */
    int64_t nblks;             /* number of stored blocks                     */
    const int *br, *bc;        /* block coordinates [nblks]                   */
    const double *data;        /* sum over blocks of rs[br]*cs[bc] doubles    */
} ob_mat;

/* Internal row-wise view: for block row i, the stored blocks sorted by column,
 * each with a pointer to its (already op()-applied) column-major data. */
typedef struct {
    int nbr, nbc;
    int *rs, *cs;
    int64_t *rowptr;           /* [nbr+1]                                     */
    int *col;                  /* [nblks] column of each block, row-sorted    */
    const double **blk;        /* [nblks] data pointer of each block          */
    double *own;               /* storage for transposed blocks, or NULL      */
} ob_rows;

static int cmp_i64pair(const void *x, const void *y)
{
    const int64_t *a = (const int64_t *)x, *b = (const int64_t *)y;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

static void rows_free(ob_rows *v)
{
    free(v->rs); free(v->cs); free(v->rowptr); free(v->col);
    free((void *)v->blk); free(v->own);
    memset(v, 0, sizeof(*v));
}

/* Build the row view of op(M). For op = 'N' the block (i,k) of op(M) is the
 * stored block (i,k). For op = 'T' (or 'C', identical for real data) the block
 * (i,k) of op(M) is the transpose of the stored block (k,i): the block grid is
 * transposed and the row/column size arrays swap roles. Transposed blocks are
 * copied element by element into owned storage. Returns 0, or -1 on a
 * duplicate block / allocation failure. */
static int rows_build(const ob_mat *M, char op, ob_rows *v)
{
    int tr = (op == 'T' || op == 't' || op == 'C' || op == 'c');
    memset(v, 0, sizeof(*v));
    v->nbr = tr ? M->nbc : M->nbr;
    v->nbc = tr ? M->nbr : M->nbc;
    v->rs = (int *)malloc(sizeof(int) * (size_t)(v->nbr + 1));
    v->cs = (int *)malloc(sizeof(int) * (size_t)(v->nbc + 1));
    v->rowptr = (int64_t *)calloc((size_t)v->nbr + 1, sizeof(int64_t));
    v->col = (int *)malloc(sizeof(int) * (size_t)(M->nblks + 1));
    v->blk = (const double **)malloc(sizeof(double *) * (size_t)(M->nblks + 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(M->nblks + 1));
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M->nblks + 1));
    if (!v->rs || !v->cs || !v->rowptr || !v->col || !v->blk || !order || !off) {
        free(order); free(off); rows_free(v); return -1;
    }
    for (int i = 0; i < v->nbr; i++) v->rs[i] = tr ? M->cs[i] : M->rs[i];
    for (int j = 0; j < v->nbc; j++) v->cs[j] = tr ? M->rs[j] : M->cs[j];

    /* data offset of every stored block, in the order given */
    int64_t total = 0;
    for (int64_t b = 0; b < M->nblks; b++) {
        off[b] = total;
        total += (int64_t)M->rs[M->br[b]] * M->cs[M->bc[b]];
    }
    /* sort (row, col) of op(M) -- stored block b sits at (bc,br) if transposed */
    for (int64_t b = 0; b < M->nblks; b++) {
        int64_t r = tr ? M->bc[b] : M->br[b];
        int64_t c = tr ? M->br[b] : M->bc[b];
        order[3 * b + 0] = r * (int64_t)(v->nbc + 1) + c;
        order[3 * b + 1] = b;
        order[3 * b + 2] = 0;
    }
    qsort(order, (size_t)M->nblks, 3 * sizeof(int64_t), cmp_i64pair);
    if (tr) {
        v->own = (double *)malloc(sizeof(double) * (size_t)(total + 1));
        if (!v->own) { free(order); free(off); rows_free(v); return -1; }
    }
    int64_t pos = 0;
    for (int64_t q = 0; q < M->nblks; q++) {
        int64_t b = order[3 * q + 1];
        int r = (int)(order[3 * q + 0] / (v->nbc + 1));
        int c = (int)(order[3 * q + 0] % (v->nbc + 1));
        if (q > 0 && order[3 * q + 0] == order[3 * (q - 1) + 0]) {
            free(order); free(off); rows_free(v); return -1;   /* duplicate */
        }
        v->rowptr[r + 1]++;
        v->col[q] = c;
        if (!tr) {
            v->blk[q] = M->data + off[b];
        } else {
            /* stored block is (sr x sc) = (cs_op[c] x rs_op[r]); op block is its transpose */
            int sr = M->rs[M->br[b]], sc = M->cs[M->bc[b]];
            const double *src = M->data + off[b];
            double *dst = v->own + pos;
            for (int x = 0; x < sc; x++)          /* op row    x = stored col */
                for (int y = 0; y < sr; y++)      /* op column y = stored row */
                    dst[x + (int64_t)y * sc] = src[y + (int64_t)x * sr];
            v->blk[q] = dst;
            pos += (int64_t)sr * sc;
        }
    }
    for (int i = 0; i < v->nbr; i++) v->rowptr[i + 1] += v->rowptr[i];
    free(order); free(off);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Local block-sparse product, Sec. II.
 *
 *   C_ij = alpha * sum_k op(A)_ik * op(B)_kj  +  beta * C_ij(old)
 *
 * The result pattern is the set of (i,j) reached by at least one product
 * op(A)_ik op(B)_kj, united with the old C pattern when beta != 0. With
 * beta == 0 the old C is never read (a NaN in it does not propagate).
 * Every element sum runs over k ascending and, inside a block product, over
 * the inner index l ascending: acc += a[r,l]*b[l,c], then
 * C = (alpha*acc) + (beta*Cold). mode 1 carries the sum in double-double.
 * mode 2 is the single-precision product the paper's library also accepts
 * (Sec. II): each input element rounded to FP32 (nearest, ties to even), each
 * product and each addition rounded to FP32, the same order; alpha and beta
 * applied in FP64 to the FP32 sum.
 *
 * Rows: rows_sel (ascending, distinct) restricts the computation to those
 * block rows of C (NULL = all rows). Output in row order, columns ascending.
 * Call first with out_br == NULL to get *out_nblks and *out_nelems.
 * ------------------------------------------------------------------------- */

/* Dot2 building blocks (Ogita, Rump, Oishi 2005): TwoSum (Knuth) and
 * TwoProduct (via a fused multiply-add, which returns the exact error). */
static inline void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}
static inline void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

typedef struct {
    int64_t nblks, nelems;
} row_count;

/* pattern of C row i: mark[j] = 1 for every reached column; returns count */
static void row_pattern(const ob_rows *a, const ob_rows *b, const ob_rows *cold,
                        int use_old, int i, unsigned char *mark)
{
    memset(mark, 0, (size_t)b->nbc);
    for (int64_t p = a->rowptr[i]; p < a->rowptr[i + 1]; p++) {
        int k = a->col[p];
        for (int64_t q = b->rowptr[k]; q < b->rowptr[k + 1]; q++) mark[b->col[q]] = 1;
    }
    if (use_old)
        for (int64_t q = cold->rowptr[i]; q < cold->rowptr[i + 1]; q++) mark[cold->col[q]] = 1;
}

int oracle_multiply(char ta, char tb, double alpha, const ob_mat *A, const ob_mat *B,
                    double beta, const ob_mat *C, const int *rows_sel, int nrows_sel,
                    int mode, int nthreads,
                    int64_t *out_nblks, int64_t *out_nelems,
                    int *out_br, int *out_bc, int64_t *out_off, double *out_data)
{
    ob_rows a, b, c;
    int use_old = (beta != 0.0) && C && C->nblks > 0;
    if (rows_build(A, ta, &a)) return -1;
    if (rows_build(B, tb, &b)) { rows_free(&a); return -1; }
    memset(&c, 0, sizeof(c));
    if (C && rows_build(C, 'N', &c)) { rows_free(&a); rows_free(&b); return -1; }
    if (a.nbc != b.nbr) { rows_free(&a); rows_free(&b); rows_free(&c); return -2; }
    for (int k = 0; k < a.nbc; k++)
        if (a.cs[k] != b.rs[k]) { rows_free(&a); rows_free(&b); rows_free(&c); return -2; }
    if (C && (c.nbr != a.nbr || c.nbc != b.nbc)) { rows_free(&a); rows_free(&b); rows_free(&c); return -2; }
    if (C) {
        for (int i = 0; i < a.nbr; i++) if (c.rs[i] != a.rs[i]) { rows_free(&a); rows_free(&b); rows_free(&c); return -2; }
        for (int j = 0; j < b.nbc; j++) if (c.cs[j] != b.cs[j]) { rows_free(&a); rows_free(&b); rows_free(&c); return -2; }
    }
    int nsel = rows_sel ? nrows_sel : a.nbr;
    row_count *cnt = (row_count *)calloc((size_t)nsel + 1, sizeof(row_count));
    if (!cnt) { rows_free(&a); rows_free(&b); rows_free(&c); return -1; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif

    /* phase 1: per row, the number of C blocks and elements */
#pragma omp parallel
    {
        unsigned char *mark = (unsigned char *)malloc((size_t)b.nbc + 1);
#pragma omp for schedule(dynamic, 1)
        for (int s = 0; s < nsel; s++) {
            int i = rows_sel ? rows_sel[s] : s;
            row_pattern(&a, &b, &c, use_old, i, mark);
            int64_t nb = 0, ne = 0;
            for (int j = 0; j < b.nbc; j++)
                if (mark[j]) { nb++; ne += (int64_t)a.rs[i] * b.cs[j]; }
            cnt[s].nblks = nb; cnt[s].nelems = ne;
        }
        free(mark);
    }
    int64_t tb_ = 0, te_ = 0;
    for (int s = 0; s < nsel; s++) { tb_ += cnt[s].nblks; te_ += cnt[s].nelems; }
    *out_nblks = tb_; *out_nelems = te_;
    if (!out_br) { free(cnt); rows_free(&a); rows_free(&b); rows_free(&c); return 0; }

    /* row start positions (blocks, elements) */
    int64_t *bstart = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nsel + 1));
    int64_t *estart = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nsel + 1));
    bstart[0] = 0; estart[0] = 0;
    for (int s = 0; s < nsel; s++) {
        bstart[s + 1] = bstart[s] + cnt[s].nblks;
        estart[s + 1] = estart[s] + cnt[s].nelems;
    }

    /* phase 2: values */
#pragma omp parallel
    {
        unsigned char *mark = (unsigned char *)malloc((size_t)b.nbc + 1);
        double **acc = (double **)calloc((size_t)b.nbc + 1, sizeof(double *));
        double **cmp = (double **)calloc((size_t)b.nbc + 1, sizeof(double *));
#pragma omp for schedule(dynamic, 1)
        for (int s = 0; s < nsel; s++) {
            int i = rows_sel ? rows_sel[s] : s;
            int m = a.rs[i];
            row_pattern(&a, &b, &c, use_old, i, mark);
            /* place the row's blocks and zero their accumulators */
            int64_t bp = bstart[s], ep = estart[s];
            for (int j = 0; j < b.nbc; j++) {
                if (!mark[j]) continue;
                out_br[bp] = i; out_bc[bp] = j; out_off[bp] = ep;
                acc[j] = out_data + ep;
                size_t ne = (size_t)m * (size_t)b.cs[j];
                memset(acc[j], 0, ne * sizeof(double));
                if (mode == 1) cmp[j] = (double *)calloc(ne + 1, sizeof(double));
                bp++; ep += (int64_t)ne;
            }
            /* k ascending over op(A)'s row i, then op(B)'s row k */
            for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; p++) {
                int k = a.col[p], kk = a.cs[k];
                const double *ablk = a.blk[p];               /* m x kk */
                for (int64_t q = b.rowptr[k]; q < b.rowptr[k + 1]; q++) {
                    int j = b.col[q], n = b.cs[j];
                    const double *bblk = b.blk[q];           /* kk x n */
                    double *x = acc[j];
                    for (int cc = 0; cc < n; cc++)
                        for (int r = 0; r < m; r++) {
                            if (mode == 1) {
                                double sh = x[r + (int64_t)cc * m], sl = cmp[j][r + (int64_t)cc * m];
                                for (int l = 0; l < kk; l++) {
                                    double pr, pe, t, te;
                                    two_prod(ablk[r + (int64_t)l * m], bblk[l + (int64_t)cc * kk], &pr, &pe);
                                    two_sum(sh, pr, &t, &te);
                                    sh = t;
                                    sl = sl + (pe + te);
                                }
                                x[r + (int64_t)cc * m] = sh;
                                cmp[j][r + (int64_t)cc * m] = sl;
                            } else if (mode == 2) {
                                float sum = (float)x[r + (int64_t)cc * m];   /* holds an FP32 value */
                                for (int l = 0; l < kk; l++) {
                                    float pa = (float)ablk[r + (int64_t)l * m];
                                    float pb = (float)bblk[l + (int64_t)cc * kk];
                                    float pr = pa * pb;
                                    sum = sum + pr;
                                }
                                x[r + (int64_t)cc * m] = (double)sum;
                            } else {
                                double sum = x[r + (int64_t)cc * m];
                                for (int l = 0; l < kk; l++)
                                    sum = sum + ablk[r + (int64_t)l * m] * bblk[l + (int64_t)cc * kk];
                                x[r + (int64_t)cc * m] = sum;
                            }
                        }
                }
            }
            /* C = alpha*acc + beta*Cold */
            int64_t q0 = use_old ? c.rowptr[i] : 0, q1 = use_old ? c.rowptr[i + 1] : 0;
            for (int j = 0; j < b.nbc; j++) {
                if (!mark[j]) continue;
                size_t ne = (size_t)m * (size_t)b.cs[j];
                const double *old = NULL;
                for (int64_t q = q0; q < q1; q++) if (c.col[q] == j) { old = c.blk[q]; break; }
                for (size_t e = 0; e < ne; e++) {
                    double v = (mode == 1) ? acc[j][e] + cmp[j][e] : acc[j][e];
                    double r = alpha * v;
                    if (old) r = r + beta * old[e];
                    acc[j][e] = r;
                }
                if (mode == 1) { free(cmp[j]); cmp[j] = NULL; }
            }
        }
        free(mark); free(acc); free(cmp);
    }
    free(bstart); free(estart); free(cnt);
    rows_free(&a); rows_free(&b); rows_free(&c);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Stack list, Sec. II (Traversal + Generation).
 *
 * One entry per block product op(A)_ik op(B)_kj with both blocks stored. The
 * paper fixes only the content of a batch (at most 30'000 multiplications of
 * one kind); the canonical order used for comparison is: shape (m,n,k)
 * ascending, then i, then j, then k. A stack is a maximal run of entries of
 * one shape, cut every stack_cap entries. Each entry is written as 7 ints:
 * stack id, m, n, k, i, j, kblk. Returns the number of entries, or <0
 * (-1 duplicate block, -2 block grids or inner block sizes that disagree).
 * ------------------------------------------------------------------------- */
static int cmp_entry(const void *x, const void *y)
{
    const int *a = (const int *)x, *b = (const int *)y;
    for (int f = 1; f < 7; f++)
        if (a[f] != b[f]) return a[f] < b[f] ? -1 : 1;
    return 0;
}

int64_t oracle_stack_list(char ta, char tb, const ob_mat *A, const ob_mat *B,
                          int stack_cap, int *out, int64_t cap)
{
    ob_rows a, b;
    if (rows_build(A, ta, &a)) return -1;
    if (rows_build(B, tb, &b)) { rows_free(&a); return -1; }
    if (a.nbc != b.nbr) { rows_free(&a); rows_free(&b); return -2; }
    for (int k = 0; k < a.nbc; k++)   /* every product needs A's k size == B's */
        if (a.cs[k] != b.rs[k]) { rows_free(&a); rows_free(&b); return -2; }
    int64_t n = 0;
    for (int i = 0; i < a.nbr; i++)
        for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; p++) {
            int k = a.col[p];
            n += b.rowptr[k + 1] - b.rowptr[k];
        }
    if (!out) { rows_free(&a); rows_free(&b); return n; }
    if (n > cap) { rows_free(&a); rows_free(&b); return -3; }
    int64_t e = 0;
    for (int i = 0; i < a.nbr; i++)
        for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; p++) {
            int k = a.col[p];
            for (int64_t q = b.rowptr[k]; q < b.rowptr[k + 1]; q++) {
                int j = b.col[q];
                int *x = out + 7 * e;
                x[0] = 0; x[1] = a.rs[i]; x[2] = b.cs[j]; x[3] = a.cs[k];
                x[4] = i; x[5] = j; x[6] = k;
                e++;
            }
        }
    qsort(out, (size_t)n, 7 * sizeof(int), cmp_entry);
    int sid = -1, run = 0;
    for (int64_t q = 0; q < n; q++) {
        int *x = out + 7 * q;
        int newshape = (q == 0) || x[1] != x[1 - 7] || x[2] != x[2 - 7] || x[3] != x[3 - 7];
        if (newshape || run == stack_cap) { sid++; run = 0; }
        x[0] = sid; run++;
    }
    rows_free(&a); rows_free(&b);
    return n;
}

/* ---------------------------------------------------------------------------
 * Dense column-major GEMM, plain triple loop: C = alpha*op(A)*op(B) + beta*C
 * with op(A) M x K and op(B) K x N, summing l ascending. Used to state the
 * densified product of Sec. III (one large block, batch size 1).
 * lda/ldb/ldc are the column strides of the stored arrays.
 * ------------------------------------------------------------------------- */
void oracle_dense_gemm(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha,
                       const double *A, int64_t lda, const double *B, int64_t ldb,
                       double beta, double *C, int64_t ldc, int nthreads)
{
    int trA = (ta == 'T' || ta == 't' || ta == 'C' || ta == 'c');
    int trB = (tb == 'T' || tb == 't' || tb == 'C' || tb == 'c');
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < N; c++)
        for (int64_t r = 0; r < M; r++) {
            double s = 0.0;
            for (int64_t l = 0; l < K; l++) {
                double x = trA ? A[l + r * lda] : A[r + l * lda];
                double y = trB ? B[c + l * ldb] : B[l + c * ldb];
                s = s + x * y;
            }
            double v = alpha * s;
            if (beta != 0.0) v = v + beta * C[r + c * ldc];
            C[r + c * ldc] = v;
        }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Emulated FP64 product with integer slices (not in the paper: the precision
 * form of the dense / large-block path). Scheme: Ozaki, Ogita, Oishi & Rump
 * (2012), error-free splitting, in its integer form (Ootomo, Ozaki & Yokota
 * 2024), stated here step by step:
 *
 *  1. Row scaling of A: mu_i = max_l |A(i,l)|, e_i = the exponent with
 *     mu_i = f * 2^e_i, 1/2 <= f < 1 (frexp), so |A(i,l)| * 2^-e_i < 1.
 *     e_i = 0 for a zero row. Column scaling of B likewise, exponents f_j.
 *  2. Slices by truncation: x = A(i,l) * 2^-e_i, r_0 = x, and for
 *     t = 1..s:  sigma_t = trunc(r_{t-1} * 2^(7t)),
 *                r_t = r_{t-1} - sigma_t * 2^(-7t).
 *     Every sigma_t is an integer in [-127, 127] with the sign of x; every
 *     step is exact in FP64. So x = sum_t sigma_t 2^(-7t) + r_s, |r_s| < 2^-7s.
 *  3. Integer products, kept exactly: for each level d = t + u with
 *     2 <= d <= s+1 (the triangular truncation: pairs with t + u > s + 1 are
 *     dropped), G_d(i,j) = sum over t+u=d of sum_l sigmaA_t(i,l) sigmaB_u(l,j).
 *  4. Recombination, exact then rounded once: the integer
 *     S = sum_{d=2}^{s+1} G_d * 2^(7(s+1-d)) is formed exactly (128-bit), and
 *     the real number S * 2^(e_i + f_j - 7(s+1)) is rounded once to the
 *     nearest double (ties to even) -- 53 significant bits for a normal
 *     result, fewer for a subnormal one, +-infinity beyond the largest double.
 *  5. C(i,j) = alpha * that value + beta * C(i,j).
 *
 * Non-finite inputs (a reading: the scheme is defined for finite values). A
 * row of A, or a column of B, that holds a NaN or an infinity has no finite
 * maximum to scale by. Its exponent is the marker OZ_NONFINITE, its slices are
 * not formed, and every C(i,j) of that row i or column j is NaN -- whatever
 * alpha, beta and the old C(i,j). (IEEE FP64 gives a NaN or an infinity in
 * exactly those elements of a dense product: one non-finite term in a dot
 * product makes it non-finite.)
 * ------------------------------------------------------------------------- */
#define OZ_NONFINITE (1 << 20)
static int frexp_exp(double mu)
{
    int e = 0;
    if (mu == 0.0) return 0;
    (void)frexp(mu, &e);
    return e;
}

/* slices of one pre-scaled value x (|x| < 1): out[t-1] = sigma_t */
void oracle_ozaki_split(double x, int s, int *out)
{
    double r = x;
    for (int t = 1; t <= s; t++) {
        double sg = trunc(ldexp(r, 7 * t));
        out[t - 1] = (int)sg;
        r = r - ldexp(sg, -7 * t);
    }
}

/* row exponents of column-major A (M x K), column exponents of column-major B
 * (K x N); OZ_NONFINITE for a row / column holding a NaN or an infinity */
void oracle_ozaki_exponents(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                            const double *B, int64_t ldb, int *e_row, int *f_col)
{
    for (int64_t i = 0; i < M; i++) {
        double mu = 0.0;
        int finite = 1;
        for (int64_t l = 0; l < K; l++) {
            double v = fabs(A[i + l * lda]);
            if (!isfinite(v)) finite = 0;
            else if (v > mu) mu = v;
        }
        e_row[i] = finite ? frexp_exp(mu) : OZ_NONFINITE;
    }
    for (int64_t j = 0; j < N; j++) {
        double nu = 0.0;
        int finite = 1;
        for (int64_t l = 0; l < K; l++) {
            double v = fabs(B[l + j * ldb]);
            if (!isfinite(v)) finite = 0;
            else if (v > nu) nu = v;
        }
        f_col[j] = finite ? frexp_exp(nu) : OZ_NONFINITE;
    }
}

/* The real number S * 2^k rounded once to the nearest double, ties to even:
 * keep the bits of |S| down to the last one a double can hold -- the 53rd
 * significant bit, or the bit of weight 2^-1074 when the result is subnormal
 * -- and round at that bit. The kept integer q (at most 2^53) times 2^(k+drop)
 * is then exactly a double, or beyond the largest one (infinity, which is the
 * correctly rounded result there). A nonzero S that rounds to zero gives a
 * zero with its sign. */
double oracle_round_scaled(__int128 S, int k)
{
    if (S == 0) return 0.0;
    int neg = S < 0;
    unsigned __int128 a = neg ? (unsigned __int128)0 - (unsigned __int128)S : (unsigned __int128)S;
    int n = 0;                                   /* bit length of |S| */
    for (unsigned __int128 t = a; t != 0; t >>= 1) n++;
    int drop = n - 53;                           /* bits below a 53-bit significand */
    if (n - 1 + k < -1022) drop = -1074 - k;     /* subnormal result */
    double r;
    if (drop <= 0) {
        r = ldexp((double)a, k);                 /* a < 2^53: exact */
    } else if (drop >= 128) {
        r = 0.0;                                 /* |S| < 2^127 <= half of the last kept bit */
    } else {
        unsigned __int128 q = a >> drop;
        unsigned __int128 rem = a - (q << drop);
        unsigned __int128 half = (unsigned __int128)1 << (drop - 1);
        if (rem > half || (rem == half && (q & 1))) q += 1;
        r = ldexp((double)q, k + drop);          /* q <= 2^53: exact, or infinity */
    }
    return neg ? -r : r;
}

/* the same with S given as its two 64-bit halves (for the tests) */
double oracle_round_scaled_parts(int64_t hi, uint64_t lo, int k)
{
    __int128 S = (__int128)(((unsigned __int128)(uint64_t)hi << 64) | lo);
    return oracle_round_scaled(S, k);
}

/* The emulated product on column-major operands; only the rows in rows_sel
 * (NULL = all) of C are computed and written. Optionally returns the level
 * sums G_d (int64, [s][nsel][N] row-major per level) for slice-level checks. */
int oracle_ozaki_gemm(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
                      const double *B, int64_t ldb, double beta, double *C, int64_t ldc, int s,
                      const int *rows_sel, int nrows_sel, int nthreads, int64_t *levels_out)
{
    if (s < 1 || s > 8) return -1;
    int *e_row = (int *)malloc(sizeof(int) * (size_t)(M + 1));
    int *f_col = (int *)malloc(sizeof(int) * (size_t)(N + 1));
    /* slices of B, stored [u][l][j] (j fastest) */
    signed char *SB = (signed char *)malloc((size_t)s * (size_t)K * (size_t)N + 1);
    if (!e_row || !f_col || !SB) { free(e_row); free(f_col); free(SB); return -1; }
    oracle_ozaki_exponents(M, N, K, A, lda, B, ldb, e_row, f_col);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; j++) {
        int sl[8];
        for (int64_t l = 0; l < K; l++) {
            if (f_col[j] == OZ_NONFINITE) memset(sl, 0, sizeof(sl));   /* never used: C column is NaN */
            else oracle_ozaki_split(ldexp(B[l + j * ldb], -f_col[j]), s, sl);
            for (int u = 0; u < s; u++) SB[((size_t)u * K + l) * N + j] = (signed char)sl[u];
        }
    }
    int nsel = rows_sel ? nrows_sel : (int)M;
#pragma omp parallel
    {
        signed char *SA = (signed char *)malloc((size_t)s * (size_t)K + 1);
        int64_t *G = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s + 2) * (size_t)N);
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < nsel; q++) {
            int64_t i = rows_sel ? rows_sel[q] : q;
            int sl[8];
            for (int64_t l = 0; l < K; l++) {
                if (e_row[i] == OZ_NONFINITE) memset(sl, 0, sizeof(sl));   /* never used: C row is NaN */
                else oracle_ozaki_split(ldexp(A[i + l * lda], -e_row[i]), s, sl);
                for (int t = 0; t < s; t++) SA[(size_t)t * K + l] = (signed char)sl[t];
            }
            memset(G, 0, sizeof(int64_t) * (size_t)(s + 2) * (size_t)N);
            for (int t = 1; t <= s; t++)
                for (int u = 1; u + t <= s + 1; u++) {
                    int64_t *g = G + (size_t)(t + u) * N;
                    for (int64_t l = 0; l < K; l++) {
                        int64_t a = SA[(size_t)(t - 1) * K + l];
                        if (a == 0) continue;
                        const signed char *b = SB + ((size_t)(u - 1) * K + l) * N;
                        for (int64_t j = 0; j < N; j++) g[j] += a * (int64_t)b[j];
                    }
                }
            for (int64_t j = 0; j < N; j++) {
                if (e_row[i] == OZ_NONFINITE || f_col[j] == OZ_NONFINITE) {
                    C[i + j * ldc] = NAN;
                    continue;
                }
                __int128 S = 0;
                for (int d = 2; d <= s + 1; d++) S += (__int128)G[(size_t)d * N + j] << (7 * (s + 1 - d));
                double v = alpha * oracle_round_scaled(S, e_row[i] + f_col[j] - 7 * (s + 1));
                if (beta != 0.0) v = v + beta * C[i + j * ldc];
                C[i + j * ldc] = v;
            }
            if (levels_out)
                for (int d = 2; d <= s + 1; d++)
                    memcpy(levels_out + ((size_t)(d - 2) * nsel + q) * N, G + (size_t)d * N,
                           sizeof(int64_t) * (size_t)N);
        }
        free(SA); free(G);
    }
    free(e_row); free(f_col); free(SB);
    return 0;
}
