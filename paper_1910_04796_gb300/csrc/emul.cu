// emul.cu -- emulated-FP64 dense product with 7-bit integer slices
// (Ozaki, Ogita, Oishi & Rump 2012, integer form) on the tensor cores.
//
//   1. exponents: e_i = frexp exponent of max_l |A(i,l)|, f_j likewise for
//      the columns of B, so |A(i,l)| 2^-e_i < 1 and |B(l,j)| 2^-f_j < 1; a
//      row or column holding a NaN or an infinity gets a marker instead and
//      its C elements come out NaN;
//   2. slices: sigma_t = the t-th 7-bit group of floor(|x| 2^(7s)) with the
//      sign of x -- the same integers as s rounds of "truncate x 2^(7t),
//      subtract", extracted here from the FP64 bit pattern with integer
//      operations (exact, no FP64 arithmetic); stored as bf16 (exact);
//   3. level sums G_d = sum_{t+u=d} S^A_t S^B_u for d = 2 .. s+1 on the
//      tensor cores, exactly (tc_ozaki.cu);
//   4. recombination: the exact 128-bit S = sum_d G_d 2^(7(s+1-d)), and
//      S 2^(e_i+f_j-7(s+1)) rounded once to FP64 (subnormal results too);
//      C = alpha * that + beta C.
// Steps 1, 2 and 4 are HBM-bound elementwise kernels; step 3 carries the work.
#include <cuda_bf16.h>

#include <mutex>

#include "emul.cuh"
#include "emul_common.cuh"
#include "smm_emul.cuh"
#include "tc_gemm.cuh"

namespace dbcsr {

namespace {

constexpr int OZ_KSEG_BLOCKS = 256;   // 16384: s * 16384 * 127^2 < 2^31 for s <= 8
constexpr int OZ_CHUNK_BLOCKS = 16;   // 1024: 1024 * 127^2 < 2^24, exact in fp32

// max |A(i,l)| over l for column-major A: bit patterns of non-negative
// doubles order like the values, so an unsigned max is a max of magnitudes.
__global__ void k_rowmax_bits(int64_t M, int64_t K, const double* __restrict__ A, int64_t lda, int64_t kchunk,
                              unsigned long long* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int64_t l0 = blockIdx.y * kchunk, l1 = min(K, l0 + kchunk);
    unsigned long long mx = 0;
    for (int64_t l = l0; l < l1; l++) {
        unsigned long long b = (unsigned long long)__double_as_longlong(A[i + l * lda]) & 0x7fffffffffffffffull;
        mx = b > mx ? b : mx;
    }
    if (mx) atomicMax(&out[i], mx);
}

// max |B(l,j)| over l for column-major B: one CTA per column
__global__ void k_colmax_bits(int64_t K, const double* __restrict__ B, int64_t ldb,
                              unsigned long long* __restrict__ out) {
    const int64_t j = blockIdx.x;
    unsigned long long mx = 0;
    for (int64_t l = threadIdx.x; l < K; l += blockDim.x) {
        unsigned long long b = (unsigned long long)__double_as_longlong(B[l + j * ldb]) & 0x7fffffffffffffffull;
        mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    __shared__ unsigned long long sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) mx = sh[w] > mx ? sh[w] : mx;
        out[j] = mx;
    }
}

__global__ void k_exponents(int64_t n, const unsigned long long* __restrict__ bits, int* __restrict__ e) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    e[i] = emul::exponent_of_bits(bits[i]);
}

using emul::fixed_point;
using emul::slice_bf16;

// A (column-major M x K) -> SA[t][i][l] (row-major, ldk), zero for l >= K.
// 32 (rows) x 64 (k) tiles through shared memory so that both sides coalesce.
__global__ void __launch_bounds__(256) k_slice_rows(int64_t M, int64_t K, int64_t ldk, const double* __restrict__ A,
                                                    int64_t lda, const int* __restrict__ e, int s,
                                                    __nv_bfloat16* __restrict__ SA) {
    __shared__ long long q[32][65];
    const int64_t i0 = blockIdx.y * 32, l0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int ll = ty; ll < 64; ll += 8) {
        const int64_t i = i0 + tx, l = l0 + ll;
        long long v = 0;
        if (i < M && l < K) v = fixed_point(A[i + l * lda], e[i], s);
        q[tx][ll] = v;
    }
    __syncthreads();
    // write: each thread two consecutive k of one row, for every slice
    for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
        const int r = idx >> 5, cp = (idx & 31) * 2;
        const int64_t i = i0 + r;
        if (i >= M) continue;
        for (int t = 1; t <= s; t++) {
            __nv_bfloat162 pr;
            pr.x = slice_bf16(q[r][cp], t, s);
            pr.y = slice_bf16(q[r][cp + 1], t, s);
            *reinterpret_cast<__nv_bfloat162*>(SA + ((int64_t)(t - 1) * M + i) * ldk + l0 + cp) = pr;
        }
    }
}

// B (column-major K x N) -> SB[u][j][l] (ldk), zero for l >= K.
__global__ void k_slice_cols(int64_t N, int64_t K, int64_t ldk, const double* __restrict__ B, int64_t ldb,
                             const int* __restrict__ f, int s, __nv_bfloat16* __restrict__ SB) {
    const int64_t j = blockIdx.y;
    const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 2;
    if (l >= ldk) return;
    long long q0 = (l < K) ? fixed_point(B[l + j * ldb], f[j], s) : 0;
    long long q1 = (l + 1 < K) ? fixed_point(B[l + 1 + j * ldb], f[j], s) : 0;
    for (int u = 1; u <= s; u++) {
        __nv_bfloat162 pr;
        pr.x = slice_bf16(q0, u, s);
        pr.y = slice_bf16(q1, u, s);
        *reinterpret_cast<__nv_bfloat162*>(SB + ((int64_t)(u - 1) * N + j) * ldk + l) = pr;
    }
}

// C = alpha * (sum_{d=s+1..2} G_d 2^(-7d)) 2^(e_i+f_j) + beta * C
__global__ void k_recombine(int64_t M, int64_t N, int s, int ksegs, const double* __restrict__ ws, int64_t stride,
                            const int* __restrict__ e, const int* __restrict__ f, double alpha, double beta,
                            double* __restrict__ C, int64_t ldc) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int64_t i = idx % M, j = idx / M;
    __int128 S = 0;   // exact sum of the level sums, each shifted to its weight
    for (int d = 2; d <= s + 1; d++) {
        long long g = 0;   // FP64 workspace entries are exact integers below 2^53
        for (int k = 0; k < ksegs; k++) g += (long long)ws[((int64_t)(d - 2) * ksegs + k) * stride + idx];
        S += (__int128)g << (7 * (s + 1 - d));
    }
    const double x = emul::recombined(S, e[i] + f[j], 7 * (s + 1));
    const BlasUpd bu(alpha, beta);
    C[i + j * ldc] = bu.old ? bu.update(x, C[i + j * ldc]) : bu.scale(x);
}

// Recombination from int32 row-major level sums ws[d-2][kseg][i][j] (row
// stride ldws) into column-major C, through a 32 x 32 shared-memory tile so
// that both the reads and the writes are coalesced. Same arithmetic and order
// as k_recombine.
// S (the slice count) is a template parameter: the level weights become
// constant shifts. The levels are joined as U 2^(7 (S - NU)) + V, U over the
// first NU = min(4, S) levels and V over the rest, each an int64 Horner sum
// (|U|, |V| < 2^64 while every level sum stays below 2^40, i.e. fewer than
// 2^9 K segments of 16 384), then one 128-bit step and one rounding.
// Output of the recombination: a column-major C (ldc), or, with `base`, the
// storage of a fully occupied block matrix (blocks in CSR order, each
// column-major), where element (i, j) lives at C[base[i] + stride[i] * j]
// (base[i] = roff(i's block row) * N + i's row within the block, stride[i] =
// that block row's size). Old values are read from the same place.
struct OzOut {
    double* C;
    int64_t ldc;
    const int64_t* base;
    const int* stride;
    __device__ __forceinline__ int64_t at(int64_t i, int64_t j) const {
        return base ? base[i] + (int64_t)stride[i] * j : i + j * ldc;
    }
};

template <int S>
__global__ void __launch_bounds__(256) k_recombine_rm(int64_t M, int64_t N, int ksegs, const int* __restrict__ ws,
                                                      int64_t ldws, const int* __restrict__ e,
                                                      const int* __restrict__ f, double alpha, double beta,
                                                      OzOut out) {
    constexpr int NU = S < 4 ? S : 4;
    __shared__ double tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    const int64_t lstride = M * ldws;
    const BlasUpd bu(alpha, beta);
    // the old C of this thread's four output elements first: its latency hides
    // behind the level sums
    int64_t addr[4];
    double cold[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int64_t i = i0 + tx, j = j0 + ty + 8 * c;
        addr[c] = (i < M && j < N) ? out.at(i, j) : -1;
        cold[c] = (bu.old && addr[c] >= 0) ? out.C[addr[c]] : 0.0;
    }
    // level sums of the thread's four elements (rows ty + 8 c, column tx), first
    // K segment: all loads issued before the arithmetic
    int v[4][S];
    bool in[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int64_t i = i0 + ty + 8 * c, j = j0 + tx;
        in[c] = i < M && j < N;
        const int* w = ws + (in[c] ? i * ldws + j : 0);
#pragma unroll
        for (int d = 0; d < S; d++) v[c][d] = in[c] ? w[(int64_t)d * ksegs * lstride] : 0;
    }
    const int fj = (j0 + tx < N) ? f[j0 + tx] : 0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int* w = ws + (in[c] ? (i0 + ty + 8 * c) * ldws + j0 + tx : 0);
        long long U = 0, V = 0;
#pragma unroll
        for (int d = 0; d < S; d++) {
            long long g = v[c][d];   // exact: further K segments summed in int64
            for (int k = 1; k < ksegs; k++) g += in[c] ? w[((int64_t)d * ksegs + k) * lstride] : 0;
            if (d < NU) U = U * 128 + g;
            else V = V * 128 + g;
        }
        const __int128 Sx = (__int128)U * ((__int128)1 << (7 * (S - NU))) + V;
        const int64_t i = i0 + ty + 8 * c;
        tile[ty + 8 * c][tx] = in[c] ? emul::recombined(Sx, e[i] + fj, 7 * (S + 1)) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 4; c++)
        if (addr[c] >= 0) {
            const double x = tile[tx][ty + 8 * c];
            out.C[addr[c]] = bu.old ? bu.update(x, cold[c]) : bu.scale(x);
        }
}

// element-row layout of a fully occupied block matrix (see OzOut)
__global__ void k_full_rows(int nbr, const int* __restrict__ rs, const int64_t* __restrict__ roff, int64_t N,
                            int64_t* __restrict__ base, int* __restrict__ stride) {
    const int bi = blockIdx.x;
    if (bi >= nbr) return;
    const int m = rs[bi];
    const int64_t r0 = roff[bi];
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        base[r0 + r] = r0 * N + r;
        stride[r0 + r] = m;
    }
}

// Slices of every stored block of one operand, written straight into the
// dense K-major slice layout S[(t-1) * rows + x][l] (row stride ldk): x is
// the op() line (row of op(A) / column of op(B)), l the inner index. A warp
// per block; a line's items (two consecutive l with 4-byte stores when the
// block's first l, its width and ldk are even, else single l) go to a group
// of lanes -- the item count rounded up to a power of two -- so that a warp
// covers 32 / group lines at once. A block (at most a few KB) stays in L1
// while its lines are read, so the strided reads cost little.
__global__ void k_slice_blocks(SliceGeom G, const int* __restrict__ ex, int s, int64_t rows, int64_t ldk,
                               __nv_bfloat16* __restrict__ S) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t plane = rows * ldk;
    for (int64_t b = w0; b < G.nblks; b += nw) {
        int X, L, xs, ls;
        int64_t xbase;
        geom_block(G, b, X, L, xs, ls, xbase);
        const int64_t lbase = G.x_is_row ? G.coff[G.col[b]] : G.roff[G.row_of[b]];
        const double* d = G.data + G.off[b];
        const bool pairs = ((lbase | L | ldk) & 1) == 0;
        const int items = pairs ? L >> 1 : L;   // per line
        int grp = 1;                             // lanes per line
        while (grp < items && grp < 32) grp <<= 1;
        const int sub = lane & (grp - 1), xr = lane / grp, lines = 32 / grp;
        for (int x = xr; x < X; x += lines) {
            const int e = ex[xbase + x];
            __nv_bfloat16* o = S + (xbase + x) * ldk + lbase;
            const double* dx = d + (int64_t)x * xs;
            for (int it = sub; it < items; it += grp) {
                if (pairs) {
                    const int l = 2 * it;
                    const long long q0 = fixed_point(dx[(int64_t)l * ls], e, s);
                    const long long q1 = fixed_point(dx[(int64_t)(l + 1) * ls], e, s);
                    for (int t = 1; t <= s; t++)
                        *reinterpret_cast<__nv_bfloat162*>(o + (int64_t)(t - 1) * plane + l) =
                            __halves2bfloat162(slice_bf16(q0, t, s), slice_bf16(q1, t, s));
                } else {
                    const long long q = fixed_point(dx[(int64_t)it * ls], e, s);
                    for (int t = 1; t <= s; t++) o[(int64_t)(t - 1) * plane + it] = slice_bf16(q, t, s);
                }
            }
        }
    }
}

// Slices of a fully occupied matrix whose block rows and block columns each
// have a single size, straight into the K-major slice layout. A warp takes one
// op() line x and a run of 64 consecutive l (two per lane), so every slice row
// segment is written as whole 128-byte lines; consecutive warps take
// consecutive lines of the same run, which read the same blocks (L1 hits).
// The element's block is found arithmetically: block (r, c) of the CSR-ordered
// full matrix starts at (r * nbc + c) * X * L.
struct UniGeom {
    const double* data;
    int X, L;          // block extent along x and along l
    int64_t nbc;       // stored block columns
    int x_is_row;      // x runs over stored rows (else stored columns)
    int64_t nlines;    // op() lines
    int64_t K;         // inner length
};

__device__ __forceinline__ double uni_elem(const UniGeom& G, unsigned bx, unsigned xw, unsigned l) {
    const unsigned bl = l / (unsigned)G.L, lw = l - bl * (unsigned)G.L;
    const int64_t blk = G.x_is_row ? (int64_t)bx * G.nbc + bl : (int64_t)bl * G.nbc + bx;
    const int64_t in_blk = G.x_is_row ? (int64_t)xw + (int64_t)lw * G.X : (int64_t)lw + (int64_t)xw * G.L;
    return G.data[blk * G.X * G.L + in_blk];
}

// TF32 operand straight from the blocks (fully occupied, one block size per
// dimension): line x of op(X) rounded to TF32 into out[x * ldk + l], zero for
// K <= l < ldk
__global__ void __launch_bounds__(256) k_tf32_uniform(UniGeom G, int64_t ldk, float* __restrict__ out) {
    const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= ldk) return;
    for (int64_t x = blockIdx.y; x < G.nlines; x += gridDim.y) {
        float v = 0.0f;
        if (l < G.K) {
            const unsigned bx = (unsigned)(x / G.X), xw = (unsigned)(x - (int64_t)bx * G.X);
            v = to_tf32(uni_elem(G, bx, xw, (unsigned)l));
        }
        out[x * ldk + l] = v;
    }
}

__global__ void __launch_bounds__(256) k_slice_uniform(UniGeom G, const int* __restrict__ ex, int s, int64_t ldk,
                                                       __nv_bfloat16* __restrict__ S) {
    const int lane = threadIdx.x & 31;
    const int64_t nruns = (G.K + 63) / 64;
    const int64_t plane = G.nlines * ldk;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < G.nlines * nruns; w += nw) {
        const int64_t x = w % G.nlines, run = w / G.nlines;
        const int64_t l = run * 64 + 2 * lane;
        if (l >= G.K) continue;
        const int e = ex[x];
        const unsigned bx = (unsigned)(x / G.X), xw = (unsigned)(x - (int64_t)bx * G.X);
        const long long q0 = fixed_point(uni_elem(G, bx, xw, (unsigned)l), e, s);
        // l + 1 = K is K padding: zero (ldk >= K is a multiple of 64, so it is inside the row)
        const long long q1 = l + 1 < G.K ? fixed_point(uni_elem(G, bx, xw, (unsigned)l + 1u), e, s) : 0;
        __nv_bfloat16* o = S + x * ldk + l;
        for (int t = 1; t <= s; t++)
            *reinterpret_cast<__nv_bfloat162*>(o + (int64_t)(t - 1) * plane) =
                __halves2bfloat162(slice_bf16(q0, t, s), slice_bf16(q1, t, s));
    }
}

__global__ void k_scale_c(int64_t M, int64_t N, double beta, double* __restrict__ C, int64_t ldc) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int64_t i = idx % M, j = idx / M;
    C[i + j * ldc] = beta != 0.0 ? __dmul_rn(beta, C[i + j * ldc]) : 0.0;
}

}  // namespace

int oz_exponents(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B, int64_t ldb,
                 int* e, int* f) {
    cudaStream_t st = ctx().stream;
    DBuf<unsigned long long> rb, cb;
    DB_TRY(rb.alloc(M ? M : 1));
    DB_TRY(cb.alloc(N ? N : 1));
    DB_CUDA(cudaMemsetAsync(rb.p, 0, sizeof(unsigned long long) * (M ? M : 1), st));
    if (M > 0 && K > 0) {
        const int64_t kchunk = 256;
        dim3 g((unsigned)cdiv(M, 256), (unsigned)cdiv(K, kchunk));
        if (g.y > 65535) return fail(DBCSR_ERR_OVERFLOW, "emulated gemm: K too large");
        k_rowmax_bits<<<g, 256, 0, st>>>(M, K, A, lda, kchunk, rb.p);
        DB_KCHECK();
    }
    if (N > 0) {
        k_colmax_bits<<<(unsigned)N, 256, 0, st>>>(K, B, ldb, cb.p);
        DB_KCHECK();
    }
    if (M > 0) {
        k_exponents<<<(unsigned)cdiv(M, 256), 256, 0, st>>>(M, rb.p, e);
        DB_KCHECK();
    }
    if (N > 0) {
        k_exponents<<<(unsigned)cdiv(N, 256), 256, 0, st>>>(N, cb.p, f);
        DB_KCHECK();
    }
    return DBCSR_OK;
}

// the slice GEMMs and the recombination into `out` (steps 3 and 4); the
// recombination, the first access to `out`, waits for out_ready when given
int oz_run(int64_t M, int64_t N, int64_t K, int64_t ldk, int s, const __nv_bfloat16* SA_p,
           const __nv_bfloat16* SB_p, const int* e_p, const int* f_p, double alpha, double beta, const OzOut& out,
           double* main_flops, int kernel, cudaEvent_t out_ready = nullptr);

int dgemm_ozaki(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
                int64_t ldb, double beta, double* C, int64_t ldc, int s, double* main_flops, int kernel) {
    cudaStream_t st = ctx().stream;
    if (M == 0 || N == 0) return DBCSR_OK;
    if (K == 0) {
        k_scale_c<<<(unsigned)cdiv(M * N, 256), 256, 0, st>>>(M, N, beta, C, ldc);
        DB_KCHECK();
        return DBCSR_OK;
    }
    if (M >= INT32_MAX || N >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "emulated gemm: dimension too large");
    const int64_t ldk = cdiv(K, 64) * 64;
    DBuf<int> e, f;
    DB_TRY(e.alloc(M));
    DB_TRY(f.alloc(N));
    DB_TRY(oz_exponents(M, N, K, A, lda, B, ldb, e.p, f.p));
    DBuf<__nv_bfloat16> SA, SB;
    DB_TRY(SA.alloc((size_t)s * M * ldk));
    DB_TRY(SB.alloc((size_t)s * N * ldk));
    {
        dim3 g((unsigned)(ldk / 64), (unsigned)cdiv(M, 32));
        if (g.y > 65535) return fail(DBCSR_ERR_OVERFLOW, "emulated gemm: M too large for the slicing grid");
        k_slice_rows<<<g, 256, 0, st>>>(M, K, ldk, A, lda, e.p, s, SA.p);
        DB_KCHECK();
        dim3 g2((unsigned)cdiv(ldk / 2, 256), (unsigned)N);
        if (N > 2147483647LL) return fail(DBCSR_ERR_OVERFLOW, "emulated gemm: N too large");
        k_slice_cols<<<g2, 256, 0, st>>>(N, K, ldk, B, ldb, f.p, s, SB.p);
        DB_KCHECK();
    }
    return oz_run(M, N, K, ldk, s, SA.p, SB.p, e.p, f.p, alpha, beta, OzOut{C, ldc, nullptr, nullptr}, main_flops,
                  kernel);
}

int oz_run(int64_t M, int64_t N, int64_t K, int64_t ldk, int s, const __nv_bfloat16* SA_p,
           const __nv_bfloat16* SB_p, const int* e_p, const int* f_p, double alpha, double beta, const OzOut& out,
           double* main_flops, int kernel, cudaEvent_t out_ready) {
    cudaStream_t st = ctx().stream;
    struct { const __nv_bfloat16* p; } SA{SA_p}, SB{SB_p};
    struct { const int* p; } e{e_p}, f{f_p};
    double* C = out.C;
    const int64_t ldc = out.ldc;
    // 128 x 256 tiles when the output is wide enough (fewer bytes moved per
    // flop), else 128 x 128 tiles; kernel 4: 256 x 256 tiles on CTA pairs
    // where both output dimensions reach 256. Measured on GB300 under its
    // power cap, the pairs need 5 % fewer cycles but more energy per flop
    // (the B halves read across the pair), so their clock settles 11 % lower
    // and they finish 7 % later: one CTA per tile is the default.
    const bool pair = kernel == 4 && M >= 256 && N >= 256 && tc2sm_usable();
    const bool wide = pair || (N >= 256 && tc256_usable());
    const int tn = wide ? 256 : 128;
    CUtensorMap tmA, tmB;
    DB_TRY(make_slice_tmap(&tmA, SA.p, ldk, M, s, 128, 2));
    DB_TRY(make_slice_tmap(&tmB, SB.p, ldk, N, s, pair ? 128 : tn, 2));
    OzParams p{};
    p.chunk_blocks = OZ_CHUNK_BLOCKS;
    p.elem_bytes = 2;
    p.M = (int)M;
    p.N = (int)N;
    p.kblocks = (int)(ldk / 64);
    p.s = s;
    p.kseg_blocks = OZ_KSEG_BLOCKS;
    p.ksegs = (int)cdiv(p.kblocks, OZ_KSEG_BLOCKS);
    p.tiles_m = (int)cdiv(M, 128);
    p.tiles_n = (int)cdiv(N, tn);
    p.units = (int64_t)p.tiles_m * p.tiles_n * p.ksegs * s;
    if (p.units >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "emulated gemm: too many work units");
    p.ws_stride = M * N;
    p.err = ctx().d_flags;
    p.wait_ns = ctx().wait_ns;
    DB_CUDA(cudaMemsetAsync(p.err, 0, sizeof(int), st));
    int h_err = 0;
    if (wide) {
        p.ldws = cdiv(N, 256) * 256;
        DBuf<int> wsi;
        DB_TRY(wsi.alloc((size_t)s * p.ksegs * M * p.ldws));
        p.ws_i32 = wsi.p;
        timer_kernel_begin();
        DB_TRY(pair ? oz_gemm2sm_launch(tmA, tmB, p) : oz_gemm256_launch(tmA, tmB, p));
        timer_kernel_end();
        DB_CUDA(cudaMemcpyAsync(&h_err, p.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        dim3 g((unsigned)cdiv(N, 32), (unsigned)cdiv(M, 32));
        if (g.y > 65535) return fail(DBCSR_ERR_OVERFLOW, "emulated gemm: M too large for the recombination grid");
        if (p.ksegs >= 512) return fail(DBCSR_ERR_OVERFLOW, "emulated gemm: K too large for exact level sums");
        if (out_ready) DB_CUDA(cudaStreamWaitEvent(st, out_ready, 0));
        switch (s) {
#define DB_RC(S_) case S_: k_recombine_rm<S_><<<g, 256, 0, st>>>(M, N, p.ksegs, wsi.p, p.ldws, e.p, f.p, alpha, beta, out); break
            DB_RC(1); DB_RC(2); DB_RC(3); DB_RC(4); DB_RC(5); DB_RC(6); DB_RC(7);
            default: DB_RC(8);
#undef DB_RC
        }
        DB_KCHECK();
    } else {
        if (out.base) return fail(DBCSR_ERR_STATE, "emulated gemm: block-layout output needs the 256-wide kernel");
        DBuf<double> ws;
        DB_TRY(ws.alloc((size_t)s * p.ksegs * M * N));
        p.ws = ws.p;
        timer_kernel_begin();
        DB_TRY(oz_gemm_launch(tmA, tmB, p));
        timer_kernel_end();
        DB_CUDA(cudaMemcpyAsync(&h_err, p.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (out_ready) DB_CUDA(cudaStreamWaitEvent(st, out_ready, 0));
        k_recombine<<<(unsigned)cdiv(M * N, 256), 256, 0, st>>>(M, N, s, p.ksegs, ws.p, p.ws_stride, e.p, f.p,
                                                               alpha, beta, C, ldc);
        DB_KCHECK();
    }
    DB_CUDA(cudaStreamSynchronize(st));
    if (h_err) return fail(DBCSR_ERR_TIMEOUT, "emulated gemm: a tensor-core pipeline wait timed out");
    // algorithmic slice-GEMM flops: one M x N x K product per slice pair (unpadded)
    if (main_flops) *main_flops = 2.0 * (double)M * (double)N * (double)K * (double)(s * (s + 1) / 2);
    return DBCSR_OK;
}

bool ozaki_blocks_ok(int64_t N) { return N >= 256 && (tc256_usable() || tc2sm_usable()); }

int dgemm_ozaki_blocks(dbcsr_matrix_s* A, bool ta, dbcsr_matrix_s* B, bool tb, dbcsr_matrix_s* C, double alpha,
                       double beta, int s, double* main_flops, int kernel) {
    cudaStream_t st = ctx().stream;
    const int64_t M = C->h_roff[C->nbr], N = C->h_coff[C->nbc];
    const int64_t K = ta ? A->h_roff[A->nbr] : A->h_coff[A->nbc];
    if (M == 0 || N == 0 || K == 0) return fail(DBCSR_ERR_STATE, "emulated block gemm: empty operand");
    if (M >= INT32_MAX || N >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "emulated gemm: dimension too large");
    const int64_t ldk = cdiv(K, 64) * 64;
    DBuf<int> e, f;
    // operands still uploading: each is awaited where it is first read, so the
    // later uploads overlap the work on the earlier operands (C's overlaps the
    // slice GEMMs; the recombination waits for it)
    DB_TRY(await_data(A));
    DB_TRY(line_exponents(A, !ta, M, e));
    DB_TRY(await_data(B));
    DB_TRY(line_exponents(B, tb, N, f));
    DBuf<__nv_bfloat16> SA, SB;
    DB_TRY(SA.alloc((size_t)s * M * ldk));
    DB_TRY(SB.alloc((size_t)s * N * ldk));
    if (ldk > K) {   // the K padding of every slice row reads as zero
        DB_CUDA(cudaMemset2DAsync(SA.p + K, ldk * sizeof(__nv_bfloat16), 0, (ldk - K) * sizeof(__nv_bfloat16),
                                  (size_t)s * M, st));
        DB_CUDA(cudaMemset2DAsync(SB.p + K, ldk * sizeof(__nv_bfloat16), 0, (ldk - K) * sizeof(__nv_bfloat16),
                                  (size_t)s * N, st));
    }
    const int sgrid = ctx().num_sms * 16;
    // one block size per dimension: whole-line runs (k_slice_uniform); else block by block
    auto uniform = [](const std::vector<int>& v) {
        for (int x : v)
            if (x != v[0]) return false;
        return !v.empty();
    };
    auto slice = [&](dbcsr_matrix_s* X, bool x_is_row, int64_t lines, const int* ex, __nv_bfloat16* out) -> int {
        if (uniform(X->h_rs) && uniform(X->h_cs)) {
            const UniGeom G{X->d_data, x_is_row ? X->h_rs[0] : X->h_cs[0], x_is_row ? X->h_cs[0] : X->h_rs[0],
                            (int64_t)X->nbc, x_is_row ? 1 : 0, lines, K};
            const int64_t warps = lines * cdiv(K, 64);
            k_slice_uniform<<<(int)std::min<int64_t>(cdiv(warps, 8), sgrid), 256, 0, st>>>(G, ex, s, ldk, out);
        } else {
            k_slice_blocks<<<(int)std::min<int64_t>(cdiv(X->nblks, 8), sgrid), 256, 0, st>>>(slice_geom(X, x_is_row),
                                                                                          ex, s, lines, ldk, out);
        }
        DB_KCHECK();
        return DBCSR_OK;
    };
    DB_TRY(slice(A, !ta, M, e.p, SA.p));
    DB_TRY(slice(B, tb, N, f.p, SB.p));
    DBuf<int64_t> base;
    DBuf<int> stride;
    DB_TRY(base.alloc(M));
    DB_TRY(stride.alloc(M));
    k_full_rows<<<C->nbr, 128, 0, st>>>(C->nbr, C->d_rs, C->d_roff, N, base.p, stride.p);
    DB_KCHECK();
    // oz_run orders the recombination, C's first access, after C's upload; on
    // failure C stays pending and its next use waits again
    DB_TRY(oz_run(M, N, K, ldk, s, SA.p, SB.p, e.p, f.p, alpha, beta, OzOut{C->d_data, 0, base.p, stride.p},
                  main_flops, kernel, C->pending ? C->ready : nullptr));
    C->pending = false;
    return DBCSR_OK;
}

static bool uniform_sizes(const std::vector<int>& v) {
    for (int x : v)
        if (x != v[0]) return false;
    return !v.empty();
}

bool tf32_blocks_ok(const dbcsr_matrix_s* A, const dbcsr_matrix_s* B, int64_t N) {
    return N >= 256 && tc256_usable() && uniform_sizes(A->h_rs) && uniform_sizes(A->h_cs) &&
           uniform_sizes(B->h_rs) && uniform_sizes(B->h_cs);
}

// The TF32 dense product of fully occupied operands without dense copies:
// the TF32 operands are rounded straight from the blocks, and the 128 x 256
// tile GEMM writes alpha * acc + beta * C into C's block storage (Sec. III's
// densification, fused as on the emulated path).
int dgemm_tf32_blocks(dbcsr_matrix_s* A, bool ta, dbcsr_matrix_s* B, bool tb, dbcsr_matrix_s* C, double alpha,
                      double beta, double* main_flops) {
    cudaStream_t st = ctx().stream;
    const int64_t M = C->h_roff[C->nbr], N = C->h_coff[C->nbc];
    const int64_t K = ta ? A->h_roff[A->nbr] : A->h_coff[A->nbc];
    if (M == 0 || N == 0 || K == 0) return fail(DBCSR_ERR_STATE, "tf32 block gemm: empty operand");
    if (M >= INT32_MAX || N >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "tf32 gemm: dimension too large");
    const int64_t ldk = cdiv(K, 32) * 32;
    DBuf<float> AT, BT;
    DB_TRY(AT.alloc((size_t)M * ldk));
    DB_TRY(BT.alloc((size_t)N * ldk));
    auto convert = [&](dbcsr_matrix_s* X, bool x_is_row, int64_t lines, float* out) -> int {
        DB_TRY(await_data(X));   // an upload still in flight: wait here, after the earlier operand's work
        const UniGeom G{X->d_data, x_is_row ? X->h_rs[0] : X->h_cs[0], x_is_row ? X->h_cs[0] : X->h_rs[0],
                        (int64_t)X->nbc, x_is_row ? 1 : 0, lines, K};
        dim3 g((unsigned)cdiv(ldk, 256), (unsigned)std::min<int64_t>(lines, 65535));
        k_tf32_uniform<<<g, 256, 0, st>>>(G, ldk, out);
        DB_KCHECK();
        return DBCSR_OK;
    };
    DB_TRY(convert(A, !ta, M, AT.p));
    DB_TRY(convert(B, tb, N, BT.p));
    DBuf<int64_t> base;
    DBuf<int> stride;
    DB_TRY(base.alloc(M));
    DB_TRY(stride.alloc(M));
    k_full_rows<<<C->nbr, 128, 0, st>>>(C->nbr, C->d_rs, C->d_roff, N, base.p, stride.p);
    DB_KCHECK();
    CUtensorMap tmA, tmB;
    DB_TRY(make_slice_tmap(&tmA, AT.p, ldk, M, 1, 128, 4));
    DB_TRY(make_slice_tmap(&tmB, BT.p, ldk, N, 1, 256, 4));
    OzParams p{};
    p.M = (int)M;
    p.N = (int)N;
    p.kblocks = (int)(ldk / 32);
    p.s = 1;                       // one "level": d = 2, one operand pair
    p.ksegs = 1;
    p.kseg_blocks = p.kblocks;
    p.chunk_blocks = p.kblocks;    // the whole K accumulates in TMEM
    p.elem_bytes = 4;
    p.tiles_m = (int)cdiv(M, 128);
    p.tiles_n = (int)cdiv(N, 128);
    p.units = (int64_t)p.tiles_m * p.tiles_n;
    p.C = C->d_data;
    p.cbase = base.p;
    p.cstride = stride.p;
    p.alpha = alpha;
    p.beta = beta;
    p.err = ctx().d_flags;
    p.wait_ns = ctx().wait_ns;
    DB_TRY(await_data(C));         // the GEMM's epilogue is C's first access
    DB_CUDA(cudaMemsetAsync(p.err, 0, sizeof(int), st));
    timer_kernel_begin();
    DB_TRY(tf32_gemm256_launch(tmA, tmB, p));
    timer_kernel_end();
    int h_err = 0;
    DB_CUDA(cudaMemcpyAsync(&h_err, p.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    if (h_err) return fail(DBCSR_ERR_TIMEOUT, "tf32 gemm: a tensor-core pipeline wait timed out");
    if (main_flops) *main_flops = 2.0 * (double)M * (double)N * (double)K;   // algorithmic, unpadded
    return DBCSR_OK;
}

int dgemm_emulated(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double beta, double* C, int64_t ldc, const dbcsr_opts& o, double* main_flops) {
    if (o.precision == DBCSR_PREC_OZAKI) {
        const int s = o.ozaki_slices > 0 ? o.ozaki_slices : 7;
        if (s > 8) return fail(DBCSR_ERR_ARG, "ozaki_slices must be 1..8");
        return dgemm_ozaki(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, main_flops, o.kernel);
    }
    if (o.precision == DBCSR_PREC_TF32) return dgemm_tf32(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, main_flops);
    return fail(DBCSR_ERR_ARG, "unknown precision");
}


}  // namespace dbcsr

// ---------------------------------------------------------------------------
// Allocation-free variant of the emulated-FP64 GEMM.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// entirely owned by another allocator (a framework that reserved the HBM up
// front), and code paths that must not perform the device-wide
// synchronisation that cudaMalloc / cudaFree may imply. For them the scratch
// of this operation (exponents, slices, level sums, error flag) lives in the
// file-scope array below, of a fixed maximum size, which every GPU that loads
// this library holds until the process exits. Every call shares it and it
// keeps the previous call's contents, so whatever must start at zero is
// cleared on the stream at the start of each call; calls whose work overlaps
// on the GPU (different streams, or threads) race on it.
// ---------------------------------------------------------------------------
namespace dbcsr {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(128) << 20;   // 128 MiB
constexpr uint64_t NOALLOC_WAIT_NS = 4000000000ull;            // each pipeline wait gives up after 4 s
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
int g_noalloc_sms[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
int noalloc_scratch(unsigned char** ptr, int* sms) {
    int dev = 0;
    DB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(DBCSR_ERR_STATE, "no-alloc gemm: device ordinal too large");
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        DB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        int n = 0;
        DB_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        g_noalloc_sms[dev] = n;
        g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *ptr = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return DBCSR_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte layout of the scratch for one call; returns the total.
size_t noalloc_layout(int64_t M, int64_t N, int64_t ldk, int s, int ksegs, size_t off[7]) {
    size_t o = 0;
    off[0] = o; o += align256(sizeof(int));                                   // error flag
    off[1] = o; o += align256(sizeof(unsigned long long) * (size_t)M);         // row max bits
    off[2] = o; o += align256(sizeof(unsigned long long) * (size_t)N);         // column max bits
    off[3] = o; o += align256(sizeof(int) * (size_t)M);                        // e
    off[4] = o; o += align256(sizeof(int) * (size_t)N);                        // f
    off[5] = o; o += align256(2 * (size_t)s * (size_t)(M + N) * (size_t)ldk);   // slices of A then B
    off[6] = o; o += align256(8 * (size_t)s * (size_t)ksegs * (size_t)M * (size_t)N);  // level sums
    return o;
}

}  // namespace

int dgemm_ozaki_noalloc(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
                        int64_t ldb, double beta, double* C, int64_t ldc, int s, cudaStream_t st) {
    if (s == 0) s = 7;
    if (s < 1 || s > 8) return fail(DBCSR_ERR_ARG, "no-alloc gemm: slices must be 1..8");
    if (M < 0 || N < 0 || K < 0) return fail(DBCSR_ERR_ARG, "no-alloc gemm: negative size");
    if ((M > 0 && lda < M) || (K > 0 && ldb < K) || (M > 0 && ldc < M))
        return fail(DBCSR_ERR_ARG, "no-alloc gemm: leading dimension smaller than the matrix");
    if (M == 0 || N == 0) return DBCSR_OK;
    if (!A || !B || !C) return fail(DBCSR_ERR_ARG, "no-alloc gemm: NULL matrix pointer");
    if (K == 0) {
        k_scale_c<<<(unsigned)cdiv(M * N, 256), 256, 0, st>>>(M, N, beta, C, ldc);
        DB_KCHECK();
        return DBCSR_OK;
    }
    const int64_t ldk = cdiv(K, 64) * 64;
    const int kblocks = (int)(ldk / 64);
    const int ksegs = (int)cdiv(kblocks, OZ_KSEG_BLOCKS);
    size_t off[7];
    if (M > (int64_t)1 << 24 || N > (int64_t)1 << 24 || K > (int64_t)1 << 30)
        return fail(DBCSR_ERR_OVERFLOW, "no-alloc gemm: a dimension exceeds the fixed scratch");
    const size_t need = noalloc_layout(M, N, ldk, s, ksegs, off);
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(DBCSR_ERR_OVERFLOW, "no-alloc gemm: needs " + std::to_string(need) +
                                            " bytes of scratch, the fixed maximum is " +
                                            std::to_string(NOALLOC_SCRATCH_BYTES) +
                                            " (about M = N = K = 1024 with 7 slices)");
    unsigned char* base = nullptr;
    int sms = 0;
    DB_TRY(noalloc_scratch(&base, &sms));
    int* err = reinterpret_cast<int*>(base + off[0]);
    unsigned long long* rb = reinterpret_cast<unsigned long long*>(base + off[1]);
    unsigned long long* cb = reinterpret_cast<unsigned long long*>(base + off[2]);
    int* e = reinterpret_cast<int*>(base + off[3]);
    int* f = reinterpret_cast<int*>(base + off[4]);
    __nv_bfloat16* SA = reinterpret_cast<__nv_bfloat16*>(base + off[5]);
    __nv_bfloat16* SB = SA + (size_t)s * M * ldk;
    double* ws = reinterpret_cast<double*>(base + off[6]);
    // the shared scratch keeps the last call's contents: clear what starts at zero
    DB_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    DB_CUDA(cudaMemsetAsync(rb, 0, sizeof(unsigned long long) * M, st));
    {
        const int64_t kchunk = 256;
        dim3 g((unsigned)cdiv(M, 256), (unsigned)cdiv(K, kchunk));
        if (g.y > 65535) return fail(DBCSR_ERR_OVERFLOW, "no-alloc gemm: K too large");
        k_rowmax_bits<<<g, 256, 0, st>>>(M, K, A, lda, kchunk, rb);
        DB_KCHECK();
        k_colmax_bits<<<(unsigned)N, 256, 0, st>>>(K, B, ldb, cb);
        DB_KCHECK();
        k_exponents<<<(unsigned)cdiv(M, 256), 256, 0, st>>>(M, rb, e);
        DB_KCHECK();
        k_exponents<<<(unsigned)cdiv(N, 256), 256, 0, st>>>(N, cb, f);
        DB_KCHECK();
        dim3 g1((unsigned)(ldk / 64), (unsigned)cdiv(M, 32));
        if (g1.y > 65535) return fail(DBCSR_ERR_OVERFLOW, "no-alloc gemm: M too large for the slicing grid");
        k_slice_rows<<<g1, 256, 0, st>>>(M, K, ldk, A, lda, e, s, SA);
        DB_KCHECK();
        dim3 g2((unsigned)cdiv(ldk / 2, 256), (unsigned)N);
        k_slice_cols<<<g2, 256, 0, st>>>(N, K, ldk, B, ldb, f, s, SB);
        DB_KCHECK();
    }
    CUtensorMap tmA, tmB;
    DB_TRY(make_slice_tmap(&tmA, SA, ldk, M, s, 128, 2));
    DB_TRY(make_slice_tmap(&tmB, SB, ldk, N, s, 128, 2));
    OzParams p{};
    p.chunk_blocks = OZ_CHUNK_BLOCKS;
    p.elem_bytes = 2;
    p.M = (int)M;
    p.N = (int)N;
    p.kblocks = kblocks;
    p.s = s;
    p.kseg_blocks = OZ_KSEG_BLOCKS;
    p.ksegs = ksegs;
    p.tiles_m = (int)cdiv(M, 128);
    p.tiles_n = (int)cdiv(N, 128);
    p.units = (int64_t)p.tiles_m * p.tiles_n * ksegs * s;
    p.ws = ws;
    p.ws_stride = M * N;
    p.err = err;
    p.wait_ns = NOALLOC_WAIT_NS;
    DB_TRY(oz_gemm_launch_on(tmA, tmB, p, st, sms));
    k_recombine<<<(unsigned)cdiv(M * N, 256), 256, 0, st>>>(M, N, s, ksegs, ws, p.ws_stride, e, f, alpha, beta, C,
                                                           ldc);
    DB_KCHECK();
    int h_err = 0;
    DB_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    if (h_err) return fail(DBCSR_ERR_TIMEOUT, "no-alloc gemm: a tensor-core pipeline wait timed out");
    return DBCSR_OK;
}

}  // namespace dbcsr

extern "C" int dbcsr_dgemm_emulated_noalloc(int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                                            int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                                            int64_t ldc, int slices, void* stream) {
    dbcsr::set_error("");
    return dbcsr::dgemm_ozaki_noalloc(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, slices,
                                      static_cast<cudaStream_t>(stream));
}
