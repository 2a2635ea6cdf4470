// stackgen.cu -- stack generation: the index join of op(A)'s block columns with
// op(B)'s block rows, the result pattern of C, and the product (stack) list.
//
// Paper, Sec. II: the local multiplication is a set of pairwise block products
// C_ij += A_ik B_kj; Traversal fixes their order ("loops over A matrix
// row-blocks and then, for each row-block, over B matrix column-blocks"),
// Generation organises them in batches, and the Scheduler assigns all batches
// of one A row-block to one thread "to avoid data-race conditions".
//
// GB300 design: one CTA per C block row (the GPU analogue of the paper's
// per-row-block thread assignment). The CTA joins op(A)'s row i with op(B)'s
// rows in shared memory (a dense marker over a window of C block columns),
// so no global sort is needed for the pattern: pass 1 counts C blocks,
// elements and products per row; prefix sums turn the counts into offsets;
// pass 2 writes C's index and the product list grouped by C block, each C
// block's products in ascending k. Every C block then has exactly one owner in
// the multiply kernels -- no atomics on C and a deterministic summation order.
#include <algorithm>

#include "internal.cuh"
#include "stackgen.cuh"

namespace dbcsr {

namespace {

constexpr int SG_NT = 512;
constexpr int SG_WIN = 4096;               // C block columns per shared-memory window
constexpr int SG_PER = SG_WIN / SG_NT;     // window entries per thread
constexpr int OLD_FLAG = 1 << 30;

__device__ __forceinline__ int view_pos(const OpView& v, int e) { return v.pos ? v.pos[e] : e; }

// Mark, for window [j0, j0+W), the number of products hitting each C column
// of row i; old C blocks (beta != 0) add OLD_FLAG.
__device__ void mark_window(const OpView& A, const OpView& B, const int* old_ptr, const int* old_col,
                            int i, int j0, int W, int* cnt) {
    for (int t = threadIdx.x; t < W; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
    const int a0 = A.ptr[i], a1 = A.ptr[i + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int p = a0 + warp; p < a1; p += nw) {
        int k = A.idx[p];
        int b0 = B.ptr[k], b1 = B.ptr[k + 1];
        for (int q = b0 + lane; q < b1; q += 32) {
            int j = B.idx[q] - j0;
            if (j >= 0 && j < W) atomicAdd(&cnt[j], 1);
        }
    }
    if (old_ptr) {
        for (int q = old_ptr[i] + threadIdx.x; q < old_ptr[i + 1]; q += blockDim.x) {
            int j = old_col[q] - j0;
            if (j >= 0 && j < W) atomicOr(&cnt[j], OLD_FLAG);
        }
    }
    __syncthreads();
}

template <class T>
__device__ T block_sum(T v, T* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T s = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += sh[q];
    __syncthreads();
    return s;
}

template <class T>
__device__ T block_excl(T v, T* total, T* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    T base = 0, tot = 0;
    for (int q = 0; q < nw; q++) {
        T s = sh[q];
        if (q < w) base += s;
        tot += s;
    }
    __syncthreads();
    *total = tot;
    return base + x - v;
}

__global__ void __launch_bounds__(SG_NT) k_sym_count(OpView A, OpView B, const int* old_ptr,
                                                     const int* old_col, const int* __restrict__ rsC,
                                                     const int* __restrict__ csC, int nbc,
                                                     int* __restrict__ row_nblk,
                                                     int64_t* __restrict__ row_nelem,
                                                     int64_t* __restrict__ row_nprod) {
    __shared__ int cnt[SG_WIN];
    __shared__ int64_t sh64[SG_NT / 32];
    const int i = blockIdx.x;
    const int m = rsC[i];
    int64_t nb = 0, ne = 0;
    for (int j0 = 0; j0 < nbc; j0 += SG_WIN) {
        int W = min(SG_WIN, nbc - j0);
        mark_window(A, B, old_ptr, old_col, i, j0, W, cnt);
        int64_t lb = 0, le = 0;
        for (int t = threadIdx.x; t < W; t += blockDim.x)
            if (cnt[t]) { lb++; le += (int64_t)m * csC[j0 + t]; }
        nb += block_sum<int64_t>(lb, sh64);
        ne += block_sum<int64_t>(le, sh64);
    }
    // products of row i: sum over op(A)'s row of op(B) row lengths
    int64_t lp = 0;
    for (int p = A.ptr[i] + threadIdx.x; p < A.ptr[i + 1]; p += blockDim.x) {
        int k = A.idx[p];
        lp += B.ptr[k + 1] - B.ptr[k];
    }
    int64_t np = block_sum<int64_t>(lp, sh64);
    if (threadIdx.x == 0) {
        row_nblk[i] = (int)nb;
        row_nelem[i] = ne;
        row_nprod[i] = np;
    }
}

__global__ void __launch_bounds__(SG_NT) k_sym_fill(
    OpView A, OpView B, const int* old_ptr, const int* old_col, const int* __restrict__ rsC,
    const int* __restrict__ csC, int nbc, const int* __restrict__ c_rowptr,
    const int64_t* __restrict__ row_ebase, const int64_t* __restrict__ row_pbase,
    int* __restrict__ c_col, int* __restrict__ c_row, int64_t* __restrict__ c_off,
    int* __restrict__ c_old, int64_t* __restrict__ c_pstart, int2* __restrict__ prod) {
    __shared__ int cnt[SG_WIN];
    __shared__ int slot[SG_WIN];
    __shared__ int bidx[SG_WIN];
    __shared__ int64_t sh64[SG_NT / 32];
    const int i = blockIdx.x;
    const int m = rsC[i];
    int64_t run_b = c_rowptr[i];
    int64_t run_e = row_ebase[i];
    int64_t run_p = 0;                       // row-local product offset
    const int64_t pbase = row_pbase[i];
    for (int j0 = 0; j0 < nbc; j0 += SG_WIN) {
        const int W = min(SG_WIN, nbc - j0);
        mark_window(A, B, old_ptr, old_col, i, j0, W, cnt);
        // per-thread chunk of SG_PER consecutive window entries
        const int t0 = threadIdx.x * SG_PER;
        int64_t sb = 0, se = 0, sp = 0;
        for (int q = 0; q < SG_PER; q++) {
            int t = t0 + q;
            if (t < W && cnt[t]) {
                sb++;
                se += (int64_t)m * csC[j0 + t];
                sp += cnt[t] & (OLD_FLAG - 1);
            }
        }
        int64_t tb, te, tp;
        int64_t xb = block_excl<int64_t>(sb, &tb, sh64);
        int64_t xe = block_excl<int64_t>(se, &te, sh64);
        int64_t xp = block_excl<int64_t>(sp, &tp, sh64);
        for (int q = 0; q < SG_PER; q++) {
            int t = t0 + q;
            if (t < W && cnt[t]) {
                int64_t b = run_b + xb;
                c_col[b] = j0 + t;
                c_row[b] = i;
                c_off[b] = run_e + xe;
                c_pstart[b] = pbase + run_p + xp;
                c_old[b] = -1;
                slot[t] = (int)(run_p + xp);
                bidx[t] = (int)b;
                xb++;
                xe += (int64_t)m * csC[j0 + t];
                xp += cnt[t] & (OLD_FLAG - 1);
            }
        }
        __syncthreads();
        if (old_ptr) {
            for (int q = old_ptr[i] + threadIdx.x; q < old_ptr[i + 1]; q += blockDim.x) {
                int j = old_col[q] - j0;
                if (j >= 0 && j < W) c_old[bidx[j]] = q;
            }
        }
        // products in k order: one op(A) entry at a time, its op(B) row in parallel
        // (distinct columns, so slot[] updates never collide)
        const int a0 = A.ptr[i], a1 = A.ptr[i + 1];
        for (int p = a0; p < a1; p++) {
            int k = A.idx[p];
            int apos = view_pos(A, p);
            int b0 = B.ptr[k], b1 = B.ptr[k + 1];
            for (int q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
                int j = B.idx[q] - j0;
                if (j >= 0 && j < W) {
                    int s = slot[j]++;
                    prod[pbase + s] = make_int2(apos, view_pos(B, q));
                }
            }
            __syncthreads();
        }
        run_b += tb;
        run_e += te;
        run_p += tp;
        __syncthreads();
    }
}

// CSC of a stored matrix: count per column, scan, then place each column's
// entries in ascending row order (stable: one thread per column walks the
// positions gathered by a sort).
__global__ void k_col_count(const int* __restrict__ col, int64_t nblks, int* __restrict__ cnt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nblks) atomicAdd(&cnt[col[e]], 1);
}

__global__ void k_iota_keys(const int* __restrict__ col, int64_t n, uint32_t* keys, uint32_t* vals) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) {
        keys[e] = (uint32_t)col[e];
        vals[e] = (uint32_t)e;
    }
}

__global__ void k_t_fill(const uint32_t* __restrict__ vals, const int* __restrict__ row_of, int64_t n,
                         int* __restrict__ tidx, int* __restrict__ tpos) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) {
        int p = (int)vals[e];
        tpos[e] = p;
        tidx[e] = row_of[p];
    }
}

// --------------------------------------------------------- canonical export
__global__ void k_prod_keys(int64_t nC, const int* __restrict__ c_row, const int* __restrict__ c_col,
                            const int64_t* __restrict__ c_pstart, const int2* __restrict__ prod,
                            const int* __restrict__ a_k_of, const int* __restrict__ size_rank,
                            const int* __restrict__ rsC, const int* __restrict__ csC,
                            const int* __restrict__ ksz, int nsizes, uint32_t* keys, uint32_t* vals,
                            int* kidx) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nC) return;
    int i = c_row[b], j = c_col[b];
    int mr = size_rank[rsC[i]], nr = size_rank[csC[j]];
    for (int64_t p = c_pstart[b]; p < c_pstart[b + 1]; p++) {
        int k = a_k_of[prod[p].x];
        int kr = size_rank[ksz[k]];
        keys[p] = (uint32_t)((mr * nsizes + nr) * nsizes + kr);
        vals[p] = (uint32_t)p;
        kidx[p] = k;
    }
}

__global__ void k_prod_cblk(int64_t nC, const int64_t* __restrict__ c_pstart, int* __restrict__ cb_of) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nC) return;
    for (int64_t p = c_pstart[b]; p < c_pstart[b + 1]; p++) cb_of[p] = (int)b;
}

__global__ void k_shape_hist(const uint32_t* __restrict__ keys, int64_t n, int* __restrict__ hist) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) atomicAdd(&hist[keys[e]], 1);
}

__global__ void k_stack_count(const int* __restrict__ hist, int nkeys, int cap, int* __restrict__ nst) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nkeys) nst[s] = (hist[s] + cap - 1) / cap;
}

__global__ void k_export(int64_t n, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                         const int* __restrict__ key_start, const int* __restrict__ stack_base, int cap,
                         const int* __restrict__ cb_of, const int* __restrict__ kidx,
                         const int* __restrict__ c_row, const int* __restrict__ c_col,
                         const int* __restrict__ rsC, const int* __restrict__ csC,
                         const int* __restrict__ ksz, int* __restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t key = keys[t];
    int p = (int)vals[t];
    int b = cb_of[p];
    int i = c_row[b], j = c_col[b], k = kidx[p];
    int sid = stack_base[key] + (int)((t - key_start[key]) / cap);
    int* o = out + 7 * t;
    o[0] = sid;
    o[1] = rsC[i];
    o[2] = csC[j];
    o[3] = ksz[k];
    o[4] = i;
    o[5] = j;
    o[6] = k;
}

__global__ void k_k_of(OpView A, int64_t nentries, int* __restrict__ k_of_pos) {
    // k_of_pos[stored position] = block column of that entry in op(A)
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nentries) k_of_pos[view_pos(A, (int)e)] = A.idx[e];
}

}  // namespace

int build_transpose_index(dbcsr_matrix_s* m) {
    if (m->t_valid) return DBCSR_OK;
    cudaStream_t st = ctx().stream;
    dfree(m->d_tptr, m->nbc + 1);
    dfree(m->d_tidx, m->nblks);
    dfree(m->d_tpos, m->nblks);
    DB_TRY(dalloc(&m->d_tptr, m->nbc + 1));
    DB_TRY(dalloc(&m->d_tidx, m->nblks ? m->nblks : 1));
    DB_TRY(dalloc(&m->d_tpos, m->nblks ? m->nblks : 1));
    DBuf<int> cnt;
    DB_TRY(cnt.alloc(m->nbc + 1));
    DB_CUDA(cudaMemsetAsync(cnt.p, 0, (m->nbc + 1) * sizeof(int), st));
    if (m->nblks > 0) {
        unsigned g = (unsigned)cdiv(m->nblks, 256);
        k_col_count<<<g, 256, 0, st>>>(m->d_col, m->nblks, cnt.p);
        DB_KCHECK();
    }
    DB_TRY(scan_i32(cnt.p, m->d_tptr, m->nbc + 1, nullptr));
    if (m->nblks > 0) {
        DBuf<uint32_t> keys, vals;
        DB_TRY(keys.alloc(m->nblks));
        DB_TRY(vals.alloc(m->nblks));
        unsigned g = (unsigned)cdiv(m->nblks, 256);
        k_iota_keys<<<g, 256, 0, st>>>(m->d_col, m->nblks, keys.p, vals.p);
        DB_KCHECK();
        int bits = 1;
        while ((1LL << bits) < (int64_t)m->nbc + 1) bits++;
        // storage is row-sorted, so a stable sort by column yields (column, row) order
        DB_TRY(radix_sort_u32(keys.p, vals.p, m->nblks, bits));
        k_t_fill<<<g, 256, 0, st>>>(vals.p, m->d_row_of, m->nblks, m->d_tidx, m->d_tpos);
        DB_KCHECK();
    }
    m->t_valid = true;
    return DBCSR_OK;
}

OpView make_view(dbcsr_matrix_s* m, bool trans) {
    OpView v;
    v.off = m->d_off;
    v.data = m->d_data;
    v.trans = trans ? 1 : 0;
    if (!trans) {
        v.ptr = m->d_rowptr;
        v.idx = m->d_col;
        v.pos = nullptr;
        v.rs = m->d_rs;
        v.cs = m->d_cs;
        v.nrows = m->nbr;
        v.ncols = m->nbc;
        v.nentries = m->nblks;
    } else {
        v.ptr = m->d_tptr;
        v.idx = m->d_tidx;
        v.pos = m->d_tpos;
        v.rs = m->d_cs;
        v.cs = m->d_rs;
        v.nrows = m->nbc;
        v.ncols = m->nbr;
        v.nentries = m->nblks;
    }
    return v;
}

void StackPlan::reset() {
    dfree(c_rowptr, (size_t)nbr + 1);
    dfree(c_col, (size_t)(nC ? nC : 1));
    dfree(c_row, (size_t)(nC ? nC : 1));
    dfree(c_off, (size_t)nC + 1);
    dfree(c_old, (size_t)(nC ? nC : 1));
    dfree(c_pstart, (size_t)nC + 1);
    dfree(prod, (size_t)(nprod ? nprod : 1));
    nC = nelem = nprod = 0;
}

// Build C's pattern and the product list for op(A)*op(B) (+ old C if given).
int build_stacks(const OpView& A, const OpView& B, const dbcsr_matrix_s* oldC, const int* d_rsC,
                 const int* d_csC, StackPlan& P) {
    cudaStream_t st = ctx().stream;
    P.reset();
    P.nbr = A.nrows;
    P.nbc = B.ncols;
    P.aentries = A.nentries;
    const int nbr = P.nbr, nbc = P.nbc;
    const int* old_ptr = oldC ? oldC->d_rowptr : nullptr;
    const int* old_col = oldC ? oldC->d_col : nullptr;
    DB_TRY(dalloc(&P.c_rowptr, (size_t)nbr + 1));
    if (nbr == 0) {
        DB_CUDA(cudaMemsetAsync(P.c_rowptr, 0, sizeof(int), st));
        DB_TRY(dalloc(&P.c_pstart, 1));
        DB_CUDA(cudaMemsetAsync(P.c_pstart, 0, sizeof(int64_t), st));
        return DBCSR_OK;
    }
    DBuf<int> row_nblk;
    DBuf<int64_t> row_nelem, row_nprod, tot;
    DB_TRY(row_nblk.alloc(nbr + 1));
    DB_TRY(row_nelem.alloc(nbr + 1));
    DB_TRY(row_nprod.alloc(nbr + 1));
    DB_TRY(tot.alloc(4));
    k_sym_count<<<nbr, SG_NT, 0, st>>>(A, B, old_ptr, old_col, d_rsC, d_csC, nbc, row_nblk.p,
                                        row_nelem.p, row_nprod.p);
    DB_KCHECK();
    DB_TRY(scan_i32(row_nblk.p, P.c_rowptr, nbr, tot.p + 0));
    DB_TRY(scan_i64(row_nelem.p, row_nelem.p, nbr, tot.p + 1));
    DB_TRY(scan_i64(row_nprod.p, row_nprod.p, nbr, tot.p + 2));
    int64_t h_tot[4];
    DB_CUDA(cudaMemcpyAsync(h_tot, tot.p, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    if (h_tot[0] >= INT32_MAX || h_tot[2] >= INT32_MAX)
        return fail(DBCSR_ERR_OVERFLOW, "multiply: result has too many blocks or products");
    P.nC = h_tot[0];
    P.nelem = h_tot[1];
    P.nprod = h_tot[2];
    int nCi = (int)P.nC;
    DB_CUDA(cudaMemcpyAsync(P.c_rowptr + nbr, &nCi, sizeof(int), cudaMemcpyHostToDevice, st));
    const size_t nc1 = P.nC ? P.nC : 1;
    DB_TRY(dalloc(&P.c_col, nc1));
    DB_TRY(dalloc(&P.c_row, nc1));
    DB_TRY(dalloc(&P.c_off, (size_t)P.nC + 1));
    DB_TRY(dalloc(&P.c_old, nc1));
    DB_TRY(dalloc(&P.c_pstart, (size_t)P.nC + 1));
    DB_TRY(dalloc(&P.prod, (size_t)(P.nprod ? P.nprod : 1)));
    DB_CUDA(cudaMemcpyAsync(P.c_pstart + P.nC, &h_tot[2], sizeof(int64_t), cudaMemcpyHostToDevice, st));
    DB_CUDA(cudaMemcpyAsync(P.c_off + P.nC, &h_tot[1], sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (P.nC > 0) {
        k_sym_fill<<<nbr, SG_NT, 0, st>>>(A, B, old_ptr, old_col, d_rsC, d_csC, nbc, P.c_rowptr,
                                           row_nelem.p, row_nprod.p, P.c_col, P.c_row, P.c_off, P.c_old,
                                           P.c_pstart, P.prod);
        DB_KCHECK();
    }
    // the host values above were copied from stack memory: finish before returning
    DB_CUDA(cudaStreamSynchronize(st));
    return DBCSR_OK;
}

// Canonical stack list (see dbcsr_get_stacks) from a built plan.
int export_stacks(const OpView& A, const StackPlan& P, const int* d_rsC, const int* d_csC,
                  const std::vector<int>& h_sizes_all, int stack_cap, int* h_out, int64_t* n_stacks,
                  int64_t* n_shapes) {
    cudaStream_t st = ctx().stream;
    const int64_t n = P.nprod;
    if (stack_cap <= 0) stack_cap = 30000;
    // distinct sizes -> rank (lexicographic shape order)
    std::vector<int> sz = h_sizes_all;
    std::sort(sz.begin(), sz.end());
    sz.erase(std::unique(sz.begin(), sz.end()), sz.end());
    int maxsz = sz.empty() ? 0 : sz.back();
    std::vector<int> rank(maxsz + 1, 0);
    for (size_t q = 0; q < sz.size(); q++) rank[sz[q]] = (int)q;
    const int ns = (int)sz.size();
    const int nkeys = ns * ns * ns;
    if (n == 0) {
        *n_stacks = 0;
        *n_shapes = 0;
        return DBCSR_OK;
    }
    if (n >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "get_stacks: too many products");
    DBuf<int> d_rank, a_k_of, kidx, cb_of, hist, nst, key_start, stack_base;
    DBuf<uint32_t> keys, vals;
    DBuf<int> d_out;
    DB_TRY(d_rank.alloc(maxsz + 1));
    DB_CUDA(cudaMemcpyAsync(d_rank.p, rank.data(), (maxsz + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    // k of every stored A position
    const int64_t nA = P.aentries;
    DB_TRY(a_k_of.alloc(nA ? nA : 1));
    if (nA) {
        k_k_of<<<(unsigned)cdiv(nA, 256), 256, 0, st>>>(A, nA, a_k_of.p);
        DB_KCHECK();
    }
    DB_TRY(keys.alloc(n));
    DB_TRY(vals.alloc(n));
    DB_TRY(kidx.alloc(n));
    DB_TRY(cb_of.alloc(n));
    unsigned gC = (unsigned)cdiv(P.nC, 128);
    k_prod_keys<<<gC, 128, 0, st>>>(P.nC, P.c_row, P.c_col, P.c_pstart, P.prod, a_k_of.p, d_rank.p, d_rsC,
                                    d_csC, A.cs, ns, keys.p, vals.p, kidx.p);
    DB_KCHECK();
    k_prod_cblk<<<gC, 128, 0, st>>>(P.nC, P.c_pstart, cb_of.p);
    DB_KCHECK();
    int bits = 1;
    while ((1LL << bits) < nkeys) bits++;
    DB_TRY(radix_sort_u32(keys.p, vals.p, n, bits));
    DB_TRY(hist.alloc(nkeys + 1));
    DB_TRY(nst.alloc(nkeys + 1));
    DB_TRY(key_start.alloc(nkeys + 1));
    DB_TRY(stack_base.alloc(nkeys + 1));
    DB_CUDA(cudaMemsetAsync(hist.p, 0, (nkeys + 1) * sizeof(int), st));
    unsigned gP = (unsigned)cdiv(n, 256);
    k_shape_hist<<<gP, 256, 0, st>>>(keys.p, n, hist.p);
    DB_KCHECK();
    k_stack_count<<<(unsigned)cdiv(nkeys + 1, 256), 256, 0, st>>>(hist.p, nkeys + 1, stack_cap, nst.p);
    DB_KCHECK();
    DBuf<int64_t> tot;
    DB_TRY(tot.alloc(2));
    DB_TRY(scan_i32(hist.p, key_start.p, nkeys + 1, nullptr));
    DB_TRY(scan_i32(nst.p, stack_base.p, nkeys + 1, tot.p));
    DB_TRY(d_out.alloc(7 * n));
    k_export<<<gP, 256, 0, st>>>(n, keys.p, vals.p, key_start.p, stack_base.p, stack_cap, cb_of.p, kidx.p,
                                 P.c_row, P.c_col, d_rsC, d_csC, A.cs, d_out.p);
    DB_KCHECK();
    int64_t h_tot = 0;
    std::vector<int> h_hist(nkeys + 1);
    DB_CUDA(cudaMemcpyAsync(&h_tot, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaMemcpyAsync(h_hist.data(), hist.p, (nkeys + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (h_out) DB_CUDA(cudaMemcpyAsync(h_out, d_out.p, 7 * n * sizeof(int), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    *n_stacks = h_tot;
    int64_t shapes = 0;
    for (int s = 0; s <= nkeys; s++) shapes += h_hist[s] > 0;
    *n_shapes = shapes;
    return DBCSR_OK;
}

}  // namespace dbcsr
