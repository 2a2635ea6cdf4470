// tf32.cu -- the TF32 variant of the dense product: inputs rounded to TF32
// (FP64 -> FP32 round-to-nearest-even, then FP32 -> TF32 round-to-nearest
// with ties away, cvt.rna.tf32.f32), products and sums in FP32 on the tensor
// cores (tcgen05 kind::tf32), result written to the FP64 C as
// alpha * acc + beta * C. Its error against the FP64 result is reported, not
// bounded (the paper's library "accepts single precision", Sec. II).
#include "internal.cuh"
#include "tc_gemm.cuh"

namespace dbcsr {

namespace {


// A (column-major M x K) -> AT[i][l] (row-major, ldk), zero for l >= K
__global__ void __launch_bounds__(256) k_tf32_rows(int64_t M, int64_t K, int64_t ldk, const double* __restrict__ A,
                                                   int64_t lda, float* __restrict__ AT) {
    __shared__ float t[32][33];
    const int64_t i0 = blockIdx.y * 32, l0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int ll = ty; ll < 32; ll += 8) {
        const int64_t i = i0 + tx, l = l0 + ll;
        t[tx][ll] = (i < M && l < K) ? to_tf32(A[i + l * lda]) : 0.0f;
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
        const int64_t i = i0 + rr;
        if (i < M) AT[i * ldk + l0 + tx] = t[rr][tx];
    }
}

// B (column-major K x N) -> BT[j][l] (ldk), zero for l >= K
__global__ void k_tf32_cols(int64_t N, int64_t K, int64_t ldk, const double* __restrict__ B, int64_t ldb,
                            float* __restrict__ BT) {
    const int64_t j = blockIdx.y;
    const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= ldk) return;
    BT[j * ldk + l] = (l < K) ? to_tf32(B[l + j * ldb]) : 0.0f;
}

}  // namespace

int dgemm_tf32(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
               int64_t ldb, double beta, double* C, int64_t ldc, double* main_flops) {
    cudaStream_t st = ctx().stream;
    if (M == 0 || N == 0) return DBCSR_OK;
    if (M >= INT32_MAX || N >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "tf32 gemm: dimension too large");
    const int64_t ldk = cdiv(std::max<int64_t>(K, 1), 32) * 32;
    DBuf<float> AT, BT;
    DB_TRY(AT.alloc((size_t)M * ldk));
    DB_TRY(BT.alloc((size_t)N * ldk));
    dim3 g1((unsigned)(ldk / 32), (unsigned)cdiv(M, 32));
    if (g1.y > 65535) return fail(DBCSR_ERR_OVERFLOW, "tf32 gemm: M too large for the conversion grid");
    k_tf32_rows<<<g1, 256, 0, st>>>(M, K, ldk, A, lda, AT.p);
    DB_KCHECK();
    dim3 g2((unsigned)cdiv(ldk, 256), (unsigned)N);
    k_tf32_cols<<<g2, 256, 0, st>>>(N, K, ldk, B, ldb, BT.p);
    DB_KCHECK();
    CUtensorMap tmA, tmB;
    DB_TRY(make_slice_tmap(&tmA, AT.p, ldk, M, 1, 128, 4));
    const bool wide = N >= 256 && tc256_usable();
    DB_TRY(make_slice_tmap(&tmB, BT.p, ldk, N, 1, wide ? 256 : 128, 4));
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
    p.C = C;
    p.ldc = ldc;
    p.alpha = alpha;
    p.beta = beta;
    p.err = ctx().d_flags;
    p.wait_ns = ctx().wait_ns;
    DB_CUDA(cudaMemsetAsync(p.err, 0, sizeof(int), st));
    timer_kernel_begin();
    if (wide) DB_TRY(tf32_gemm256_launch(tmA, tmB, p));
    else DB_TRY(tf32_gemm_launch(tmA, tmB, p));
    timer_kernel_end();
    int h_err = 0;
    DB_CUDA(cudaMemcpyAsync(&h_err, p.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    if (h_err) return fail(DBCSR_ERR_TIMEOUT, "tf32 gemm: a tensor-core pipeline wait timed out");
    if (main_flops) *main_flops = 2.0 * (double)M * (double)N * (double)K;   // algorithmic, unpadded
    return DBCSR_OK;
}

}  // namespace dbcsr
