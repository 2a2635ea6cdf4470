// dense.cu -- the densified path of the paper's Sec. III.
//
// "When the input matrices are dense the blocks are coalesced into larger,
// dense blocks"; the batch size becomes 1, the product is one large GEMM, and
// at the end C is "undensified", split back following the original block
// sizes. With one GPU (P = 1 rank, t = 1 stream) Eq. (1)-(2) give one block
// of M x K for A and K x N for B: the whole matrices.
//
// Kernels here:
//   k_densify    stored blocks -> dense column-major op(M), transposing
//                through a shared-memory tile when op = T (coalesced both ways)
//   k_undensify  dense column-major C -> C's blocks (CSR order)
//   k_dgemm_dmma FP64 GEMM on the FP64 tensor-core instruction
//                (mma.sync m8n8k4 .f64); tiles of 64x64, k-steps of 16.
// The FP64 pipe (~1 TFLOP/s on GB300) bounds the GEMM; the copies are
// HBM-bound and small next to it.
#include "internal.cuh"
#include "dense.cuh"

namespace dbcsr {

namespace {

// One CTA per stored block, 32x32 tiles. Stored block (i,j) of size m x n.
// trans = 0: dense[(ro[i]+r) + (co[j]+c)*ld] = blk[r + c*m]
// trans = 1: dense[(co[j]+c) + (ro[i]+r)*ld] = blk[r + c*m]   (op = transpose)
__global__ void __launch_bounds__(256) k_densify(int64_t nblks, const int* __restrict__ row_of,
                                                 const int* __restrict__ col,
                                                 const int64_t* __restrict__ off,
                                                 const double* __restrict__ data,
                                                 const int* __restrict__ rs, const int* __restrict__ cs,
                                                 const int64_t* __restrict__ roff,
                                                 const int64_t* __restrict__ coff, int trans,
                                                 double* __restrict__ dense, int64_t ld, int lo, int hi,
                                                 int64_t base) {
    // only blocks whose op() block row lies in [lo, hi); op() element rows shift by -base
    __shared__ double tile[32][33];
    for (int64_t b = blockIdx.x; b < nblks; b += gridDim.x) {
        const int i = row_of[b], j = col[b];
        const int oprow = trans ? j : i;
        if (oprow < lo || oprow >= hi) continue;
        const int m = rs[i], n = cs[j];
        const double* blk = data + off[b];
        const int64_t r0 = roff[i] - (trans ? 0 : base), c0 = coff[j] - (trans ? base : 0);
        for (int tr = 0; tr < m; tr += 32)
            for (int tc = 0; tc < n; tc += 32) {
                const int x = threadIdx.x & 31, y = threadIdx.x >> 5;   // 32 x 8
                if (!trans) {
                    for (int yy = y; yy < 32; yy += 8) {
                        int r = tr + x, c = tc + yy;
                        if (r < m && c < n) dense[(r0 + r) + (c0 + c) * ld] = blk[r + (int64_t)c * m];
                    }
                } else {
                    for (int yy = y; yy < 32; yy += 8) {
                        int r = tr + x, c = tc + yy;
                        tile[yy][x] = (r < m && c < n) ? blk[r + (int64_t)c * m] : 0.0;
                    }
                    __syncthreads();
                    for (int yy = y; yy < 32; yy += 8) {
                        int c = tc + x, r = tr + yy;   // write along c (dense row of op)
                        if (r < m && c < n) dense[(c0 + c) + (r0 + r) * ld] = tile[x][yy];
                    }
                    __syncthreads();
                }
            }
    }
}

__global__ void __launch_bounds__(256) k_undensify(int64_t nblks, const int* __restrict__ row_of,
                                                   const int* __restrict__ col,
                                                   const int64_t* __restrict__ off, double* __restrict__ data,
                                                   const int* __restrict__ rs, const int* __restrict__ cs,
                                                   const int64_t* __restrict__ roff,
                                                   const int64_t* __restrict__ coff,
                                                   const double* __restrict__ dense, int64_t ld, int64_t base) {
    // dense row of element row r: r - base
    for (int64_t b = blockIdx.x; b < nblks; b += gridDim.x) {
        const int i = row_of[b], j = col[b];
        const int m = rs[i], n = cs[j];
        double* blk = data + off[b];
        const int64_t r0 = roff[i] - base, c0 = coff[j];
        const int mn = m * n;
        for (int e = threadIdx.x; e < mn; e += blockDim.x) {
            int r = e % m, c = e / m;
            blk[e] = dense[(r0 + r) + (c0 + c) * ld];
        }
    }
}

// ----------------------------------------------------------- FP64 DMMA GEMM
// C (M x N, ldc) = alpha * A (M x K, lda) * B (K x N, ldb) + beta * C, all
// column-major. 128 threads = 2x2 warps, each warp a 32x32 tile of 4x4
// m8n8 fragments; CTA tile 64x64, BK = 16, double-buffered shared memory.
constexpr int DG_BM = 64, DG_BN = 64, DG_BK = 16;

__device__ __forceinline__ void dmma_8x8x4(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(128) k_dgemm_dmma(int64_t M, int64_t N, int64_t K, double alpha,
                                                    const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb, double beta,
                                                    double* __restrict__ C, int64_t ldc) {
    __shared__ double As[2][DG_BK][DG_BM + 1];
    __shared__ double Bs[2][DG_BK][DG_BN + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
    const int64_t m0 = (int64_t)blockIdx.x * DG_BM, n0 = (int64_t)blockIdx.y * DG_BN;
    double acc[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b][0] = acc[a][b][1] = 0.0;

    // global -> registers: A tile 64 x 16 (8 per thread), B tile 16 x 64 (8 per thread)
    double ra[8], rb[8];
    auto gload = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < 8; q++) {
            int e = tid + 128 * q;          // 0..1023
            int r = e & 63, kk = e >> 6;    // A: r fastest (coalesced)
            int64_t gr = m0 + r, gk = k0 + kk;
            ra[q] = (gr < M && gk < K) ? __ldg(A + gr + gk * lda) : 0.0;
            int kb = e & 15, nb = e >> 4;   // B: k fastest
            int64_t gkb = k0 + kb, gn = n0 + nb;
            rb[q] = (gkb < K && gn < N) ? __ldg(B + gkb + gn * ldb) : 0.0;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 8; q++) {
            int e = tid + 128 * q;
            As[buf][e >> 6][e & 63] = ra[q];
            Bs[buf][e & 15][e >> 4] = rb[q];
        }
    };
    const int64_t nk = (K + DG_BK - 1) / DG_BK;
    if (nk > 0) {
        gload(0);
        sstore(0);
    }
    __syncthreads();
    for (int64_t t = 0; t < nk; t++) {
        const int buf = (int)(t & 1);
        if (t + 1 < nk) gload((t + 1) * DG_BK);
#pragma unroll
        for (int ks = 0; ks < DG_BK; ks += 4) {
            double af[4], bf[4];
#pragma unroll
            for (int a = 0; a < 4; a++) af[a] = As[buf][ks + (lane & 3)][wm + a * 8 + (lane >> 2)];
#pragma unroll
            for (int b = 0; b < 4; b++) bf[b] = Bs[buf][ks + (lane & 3)][wn + b * 8 + (lane >> 2)];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) dmma_8x8x4(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
        }
        if (t + 1 < nk) sstore(buf ^ 1);
        __syncthreads();
    }
    // epilogue: element (row = lane>>2, col = 2*(lane&3) + {0,1}) of each fragment
    const BlasUpd bu(alpha, beta);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                int64_t r = m0 + wm + a * 8 + (lane >> 2);
                int64_t c = n0 + wn + b * 8 + 2 * (lane & 3) + h;
                if (r < M && c < N) {
                    C[r + c * ldc] = bu.old ? bu.update(acc[a][b][h], C[r + c * ldc]) : bu.scale(acc[a][b][h]);
                }
            }
}

}  // namespace

int densify(const dbcsr_matrix_s* m, bool trans, double* dense, int64_t ld, bool zero_first) {
    cudaStream_t st = ctx().stream;
    const int64_t rows = trans ? m->h_coff[m->nbc] : m->h_roff[m->nbr];
    const int64_t cols = trans ? m->h_roff[m->nbr] : m->h_coff[m->nbc];
    if (zero_first && rows * cols > 0)
        DB_CUDA(cudaMemsetAsync(dense, 0, sizeof(double) * (size_t)(ld * (cols - 1) + rows), st));
    if (m->nblks == 0) return DBCSR_OK;
    int grid = (int)std::min<int64_t>(m->nblks, (int64_t)ctx().num_sms * 16);
    k_densify<<<grid, 256, 0, st>>>(m->nblks, m->d_row_of, m->d_col, m->d_off, m->d_data, m->d_rs, m->d_cs,
                                    m->d_roff, m->d_coff, trans ? 1 : 0, dense, ld, 0, INT32_MAX, 0);
    DB_KCHECK();
    return DBCSR_OK;
}

int densify_rows(const dbcsr_matrix_s* m, bool trans, int lo, int hi, double* dense, int64_t ld, int64_t at) {
    cudaStream_t st = ctx().stream;
    const std::vector<int64_t>& ro = trans ? m->h_coff : m->h_roff;
    const int64_t base = ro[lo] - at;   // element row ro[lo] lands on dense row `at`
    if (m->nblks == 0) return DBCSR_OK;
    int grid = (int)std::min<int64_t>(m->nblks, (int64_t)ctx().num_sms * 16);
    k_densify<<<grid, 256, 0, st>>>(m->nblks, m->d_row_of, m->d_col, m->d_off, m->d_data, m->d_rs, m->d_cs,
                                    m->d_roff, m->d_coff, trans ? 1 : 0, dense, ld, lo, hi, base);
    DB_KCHECK();
    return DBCSR_OK;
}

int undensify_blocks(int64_t b0, int64_t b1, const int* row_of, const int* col, const int64_t* off, double* data,
                     const dbcsr_matrix_s* shape, const double* dense, int64_t ld, int64_t base) {
    if (b1 <= b0) return DBCSR_OK;
    cudaStream_t st = ctx().stream;
    int grid = (int)std::min<int64_t>(b1 - b0, (int64_t)ctx().num_sms * 16);
    k_undensify<<<grid, 256, 0, st>>>(b1 - b0, row_of + b0, col + b0, off + b0, data, shape->d_rs, shape->d_cs,
                                      shape->d_roff, shape->d_coff, dense, ld, base);
    DB_KCHECK();
    return DBCSR_OK;
}

int undensify(dbcsr_matrix_s* m, const double* dense, int64_t ld) {
    if (m->nblks == 0) return DBCSR_OK;
    cudaStream_t st = ctx().stream;
    int grid = (int)std::min<int64_t>(m->nblks, (int64_t)ctx().num_sms * 16);
    k_undensify<<<grid, 256, 0, st>>>(m->nblks, m->d_row_of, m->d_col, m->d_off, m->d_data, m->d_rs, m->d_cs,
                                      m->d_roff, m->d_coff, dense, ld, 0);
    DB_KCHECK();
    return DBCSR_OK;
}

int dgemm_fp64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
               int64_t ldb, double beta, double* C, int64_t ldc) {
    if (M <= 0 || N <= 0) return DBCSR_OK;
    dim3 grid((unsigned)cdiv(M, DG_BM), (unsigned)cdiv(N, DG_BN));
    if (grid.y > 65535) return fail(DBCSR_ERR_OVERFLOW, "dgemm: N too large for the grid");
    k_dgemm_dmma<<<grid, 128, 0, ctx().stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    DB_KCHECK();
    return DBCSR_OK;
}

}  // namespace dbcsr
