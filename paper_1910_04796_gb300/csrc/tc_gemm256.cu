// tc_gemm256.cu -- the tensor-core GEMM of the emulated paths with 128 x 256
// output tiles (one tcgen05.mma of M = 128, N = 256, K = 16 per step).
//
// Same work decomposition and arithmetic as k_tc_gemm in tc_ozaki.cu (see its
// header): integer-slice GEMMs with exact fp32 stretches of 1024 K flushed to
// int32, or the TF32 GEMM. A 256-wide tile reads each A tile once for twice
// the output: 85 instead of 64 flops per byte moved into shared memory, and
// proportionally less L2 and DRAM traffic per flop. Both 256-column fp32
// accumulator buffers fill TMEM (512 columns), so the exact int32 level sums
// live in registers of the epilogue warps instead:
//   warpgroup 0 (warps 0-3): warp 0 TMA producer, warp 1 TMEM allocator and
//                MMA issuer; shrinks to 56 registers per thread (setmaxnreg)
//   warpgroups 1-2 (warps 4-11): epilogue, warp w reads TMEM lane quadrant
//                w % 4 and columns 128 * ((w - 4) / 4) .. +127; grows to 224
//                registers per thread and holds 128 int32 sums per thread.
// Register budget: launched with 384 threads x 168 registers = 64 512;
// 128 x 56 + 256 x 224 = 64 512. The host checks the compiled register count
// before launching (a larger split would make setmaxnreg.inc wait forever).
// Every mbarrier wait is bounded as in k_tc_gemm (pipeline waits by
// OzParams::wait_ns, clean-up waits by a fixed 4 s).
#include <cuda.h>

#include "internal.cuh"
#include "sm100_ptx.cuh"
#include "tc_gemm.cuh"

namespace dbcsr {

namespace {

constexpr int W_TM = 128, W_TN = 256, W_ROW_BYTES = 128;
constexpr int W_STAGE_A = W_TM * W_ROW_BYTES;    // 16 KB
constexpr int W_STAGE_B = W_TN * W_ROW_BYTES;    // 32 KB
constexpr int W_STAGES = 4;
constexpr int W_THREADS = 384;
constexpr int W_EPI_WARPS = 8;
constexpr int W_LAUNCH_REGS = 168;               // 65536 / 384, rounded down to a multiple of 8
constexpr int W_REGS_CTRL = 56, W_REGS_EPI = 224;
static_assert(128 * W_REGS_CTRL + 256 * W_REGS_EPI <= W_THREADS * W_LAUNCH_REGS, "register split exceeds launch");
constexpr int W_SMEM = W_STAGES * (W_STAGE_A + W_STAGE_B) + 1024 + 256;
constexpr uint64_t W_DRAIN_NS = 4000000000ull;   // clean-up waits before the CTA exits
constexpr int W_GROUP_M = 16;

template <int MODE>
struct WTraits;
template <>
struct WTraits<0> {   // bf16 slices
    static constexpr uint32_t IDESC = ptx::idesc_f32acc(1, W_TM, W_TN);
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
        ptx::mma_f16_ss(d, a, b, IDESC, acc);
    }
};
template <>
struct WTraits<1> {   // tf32
    static constexpr uint32_t IDESC = ptx::idesc_f32acc(2, W_TM, W_TN);
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
        ptx::mma_tf32_ss(d, a, b, IDESC, acc);
    }
};

// 32-bit unit decoding (units < 2^31, checked on the host): a 64-bit division
// would be a subroutine call with the 128 live sums of the epilogue around it
__device__ __forceinline__ void w_unit(int u, const OzParams& p, int tiles_n, int& tm, int& tn, int& kseg,
                                       int& li) {
    const int tiles = p.tiles_m * tiles_n;
    const int x = u % tiles, r = u / tiles;
    kseg = r % p.ksegs;
    li = r / p.ksegs;
    const int per_group = W_GROUP_M * tiles_n;
    const int g = x / per_group;
    const int first_m = g * W_GROUP_M;
    const int gm = min(W_GROUP_M, p.tiles_m - first_m);
    const int xi = x - g * per_group;
    tm = first_m + xi % gm;
    tn = xi / gm;
}

template <int MODE>
__global__ void __launch_bounds__(W_THREADS, 1)
    k_tc_gemm256(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams p) {
    using Tr = WTraits<MODE>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + W_STAGES * W_STAGE_A;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + W_STAGES * W_STAGE_B);
    uint64_t* empty = full + W_STAGES;
    uint64_t* tfull = empty + W_STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_n = (p.N + W_TN - 1) / W_TN;
    if (threadIdx.x == 0) {
        for (int s = 0; s < W_STAGES; s++) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            ptx::mbar_init(&tfull[b], 1);
            ptx::mbar_init(&tempty[b], W_EPI_WARPS);
        }
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_holder, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const int kelems = W_ROW_BYTES / p.elem_bytes;
    auto on_timeout = [&]() {
        atomicExch(p.err, 1);
        *abort_flag = 1;
    };

    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(W_REGS_CTRL));
        if (warp == 0 && lane == 0) {
            // ------------------------------------------------------ TMA producer
            int64_t it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < (int)p.units && ok; u += gridDim.x) {
                int tm, tn, kseg, li;
                w_unit(u, p, tiles_n, tm, tn, kseg, li);
                const int d = li + 2;
                const int kb0 = kseg * p.kseg_blocks, kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
                for (int t = 1; t < d && ok; t++)
                    for (int kb = kb0; kb < kb1; kb++, it++) {
                        const int st = (int)(it % W_STAGES);
                        const uint32_t ph = (uint32_t)((it / W_STAGES) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, p.wait_ns)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::mbar_arrive_expect_tx(&full[st], W_STAGE_A + W_STAGE_B);
                        ptx::tma_load_3d(sA + st * W_STAGE_A, &tmA, &full[st], kb * kelems, tm * W_TM, t - 1);
                        ptx::tma_load_3d(sB + st * W_STAGE_B, &tmB, &full[st], kb * kelems, tn * W_TN, d - t - 1);
                    }
            }
            const int64_t first = it > W_STAGES ? it - W_STAGES : 0;
            for (int64_t q = first; q < it; q++)
                if (!ptx::mbar_wait_bounded(&full[q % W_STAGES], (uint32_t)((q / W_STAGES) & 1), W_DRAIN_NS)) {
                    on_timeout();
                    break;
                }
        } else if (warp == 1 && lane == 0) {
            // ------------------------------------------------------- MMA issuer
            int64_t it = 0, ci = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < (int)p.units && ok; u += gridDim.x) {
                int tm, tn, kseg, li;
                w_unit(u, p, tiles_n, tm, tn, kseg, li);
                const int d = li + 2;
                const int kb0 = kseg * p.kseg_blocks, kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
                for (int t = 1; t < d && ok; t++)
                    for (int c = kb0; c < kb1 && ok; c += p.chunk_blocks, ci++) {
                        const int buf = (int)(ci & 1);
                        const uint32_t aph = (uint32_t)((ci >> 1) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded(&tempty[buf], aph ^ 1u, p.wait_ns)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t dt = tmem + (uint32_t)(buf * W_TN);
                        const int ce = min(c + p.chunk_blocks, kb1);
                        for (int kb = c; kb < ce; kb++, it++) {
                            const int st = (int)(it % W_STAGES);
                            const uint32_t ph = (uint32_t)((it / W_STAGES) & 1);
                            if (*abort_flag || !ptx::mbar_wait_bounded(&full[st], ph, p.wait_ns)) {
                                if (!*abort_flag) on_timeout();
                                ok = false;
                                break;
                            }
                            ptx::tc_fence_after();
                            const uint64_t ad = ptx::smem_desc_sw128(sA + st * W_STAGE_A);
                            const uint64_t bd = ptx::smem_desc_sw128(sB + st * W_STAGE_B);
#pragma unroll
                            for (int kk = 0; kk < 4; kk++)
                                Tr::mma(dt, ad + (uint64_t)((kk * 32) >> 4), bd + (uint64_t)((kk * 32) >> 4),
                                        (kb > c || kk > 0) ? 1u : 0u);
                            ptx::mma_commit(&empty[st]);
                        }
                        if (ok) ptx::mma_commit(&tfull[buf]);
                    }
            }
            ptx::mma_commit(drain);
            if (!ptx::mbar_wait_bounded(drain, 0, W_DRAIN_NS)) on_timeout();
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(W_REGS_EPI));
        // --------------------------------------------------------- epilogue
        const BlasUpd bu(p.alpha, p.beta);
        const int q = warp & 3;
        const int half = (warp - 4) >> 2;
        const int row = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 128);
        int64_t ci = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < (int)p.units && ok; u += gridDim.x) {
            int tm, tn, kseg, li;
            w_unit(u, p, tiles_n, tm, tn, kseg, li);
            const int d = li + 2;
            const int kb0 = kseg * p.kseg_blocks, kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
            const int nchunks = (d - 1) * ((kb1 - kb0 + p.chunk_blocks - 1) / p.chunk_blocks);
            const int64_t i = (int64_t)tm * W_TM + row;
            const int64_t j0 = (int64_t)tn * W_TN + half * 128;
            // TF32: this thread's output row (column-major C, or C's block storage)
            double* crow = nullptr;
            int64_t cst = 0;
            if (MODE == 1 && i < p.M) {
                crow = p.cbase ? p.C + p.cbase[i] : p.C + i;
                cst = p.cbase ? (int64_t)p.cstride[i] : p.ldc;
            }
            int acc[128];
            if (MODE == 0) {
#pragma unroll
                for (int c = 0; c < 128; c++) acc[c] = 0;
            }
            for (int ch = 0; ch < nchunks; ch++, ci++) {
                const int buf = (int)(ci & 1);
                const uint32_t aph = (uint32_t)((ci >> 1) & 1);
                if (*abort_flag || !ptx::mbar_wait_bounded(&tfull[buf], aph, p.wait_ns)) {
                    if (!*abort_flag) on_timeout();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                if (MODE == 0) {
                    // 16 columns at a time: the 128 sums plus one 16-register staging set fit the budget
#pragma unroll
                    for (int g = 0; g < 8; g++) {
                        uint32_t r[16];
                        ptx::tmem_ld_32x32b_x16(tl + (uint32_t)(buf * W_TN + g * 16), r);
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int c = 0; c < 16; c++) acc[g * 16 + c] += __float2int_rn(__uint_as_float(r[c]));
                    }
                }
#pragma unroll 1
                for (int g = 0; g < (MODE == 0 ? 0 : 4); g++) {
                    uint32_t r[32];
                    ptx::tmem_ld_32x32b_x32(tl + (uint32_t)(buf * W_TN + g * 32), r);
                    ptx::tmem_wait_ld();
                    if (i < p.M) {
#pragma unroll
                        for (int c = 0; c < 32; c++) {
                            const int64_t j = j0 + g * 32 + c;
                            if (j < p.N) {
                                double* cp = crow + j * cst;
                                const double x = (double)__uint_as_float(r[c]);
                                *cp = bu.old ? bu.update(x, *cp) : bu.scale(x);
                            }
                        }
                    }
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[buf]);
            }
            if (!ok) break;
            if (MODE == 0 && i < p.M) {
                // row-major int32 level sums: 128 consecutive columns of row i,
                // 16-byte stores at immediate offsets from one base address
                int* out = p.ws_i32 + (((int64_t)li * p.ksegs + kseg) * p.M + i) * p.ldws + j0;
#pragma unroll
                for (int c = 0; c < 128; c += 4)
                    *reinterpret_cast<int4*>(out + c) = make_int4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem, 512);
}

template <int MODE>
int launch256(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p, cudaStream_t st, int num_sms) {
    OzParams q = p;
    const int tiles_n = (int)cdiv(p.N, W_TN);
    q.units = (int64_t)p.tiles_m * tiles_n * p.ksegs * p.s;
    if (q.units <= 0) return DBCSR_OK;
    auto kern = k_tc_gemm256<MODE>;
    cudaFuncAttributes fa;
    DB_CUDA(cudaFuncGetAttributes(&fa, kern));
    if (fa.numRegs != W_LAUNCH_REGS)   // the setmaxnreg split assumes exactly this launch budget
        return fail(DBCSR_ERR_STATE, "256-wide tensor-core GEMM built with " + std::to_string(fa.numRegs) +
                                         " registers per thread, expected " + std::to_string(W_LAUNCH_REGS));
    DB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, W_SMEM));
    const int grid = (int)std::min<int64_t>(q.units, num_sms);
    kern<<<grid, W_THREADS, W_SMEM, st>>>(tmA, tmB, q);
    DB_KCHECK();
    return DBCSR_OK;
}

}  // namespace

bool tc256_usable() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_tc_gemm256<0>) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaFuncAttributes fb;
    if (cudaFuncGetAttributes(&fb, k_tc_gemm256<1>) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return fa.numRegs == W_LAUNCH_REGS && fb.numRegs == W_LAUNCH_REGS;
}

int oz_gemm256_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p) {
    return launch256<0>(tmA, tmB, p, ctx().stream, ctx().num_sms);
}

int tf32_gemm256_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p) {
    return launch256<1>(tmA, tmB, p, ctx().stream, ctx().num_sms);
}

}  // namespace dbcsr
