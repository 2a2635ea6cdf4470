// tc_ozaki.cu -- integer-slice GEMMs of the emulated-FP64 product on the
// 5th-generation tensor cores (tcgen05, kind::f16 with bf16 operands).
//
// The emulation (Ozaki, Ogita, Oishi & Rump 2012, integer form) needs exact
// products of 7-bit integer slices: G_d = sum_{t+u=d} S^A_t * S^B_u. Slices
// are integers in [-127, 127], exactly representable in bf16; a bf16 MMA
// with fp32 accumulation is exact while every partial sum stays below 2^24,
// i.e. for up to 1040 products of two slices. The kernel therefore lets the
// tensor core accumulate 1024-long stretches of K in TMEM (fp32, exact), and
// the epilogue warps convert each stretch to int32 and add it to a register
// accumulator (exact while s * K_segment * 127^2 < 2^31: K segments of 16384).
// One work unit = one 128 x TN output tile, one level d, one K segment; its
// exact integer level sum is written as FP64 (exact below 2^53) to a
// workspace that the recombination kernel reads.
//
// Warp roles (one CTA per SM, persistent over work units):
//   warp 0      TMA producer: A-slice and B-slice tiles (128 x 64 bf16,
//               128-byte swizzle) into a ring of shared-memory stages
//   warp 1      TMEM allocator; lane 0 issues tcgen05.mma (4 x K=16 per stage)
//               into one of two TMEM accumulators and commits to mbarriers
//   warps 2..   epilogue: tcgen05.ld, fp32 -> int32, accumulate, release
// Every mbarrier wait is bounded (4 s on the global timer); on a timeout the
// kernel records an error flag, unwinds all roles, drains its TMA loads and
// MMAs, frees TMEM and returns -- the host reports DBCSR_ERR_TIMEOUT.
#include <cuda.h>

#include "internal.cuh"
#include "sm100_ptx.cuh"
#include "tc_gemm.cuh"

namespace dbcsr {

namespace {

constexpr int OZ_TM = 128;
constexpr int OZ_TK = 64;             // bf16 elements per 128-byte swizzle row
constexpr int OZ_CHUNK = 16;          // k-blocks (x64) per exact fp32 stretch: 1024
constexpr uint64_t OZ_WAIT_NS = 4000000000ull;
constexpr int OZ_GROUP_M = 16;        // tile rasterisation group (L2 reuse)

template <int TN>
struct OzCfg {
    static constexpr int STAGE_A = OZ_TM * OZ_TK * 2;
    static constexpr int STAGE_B = TN * OZ_TK * 2;
    static constexpr int STAGES = (TN == 256) ? 4 : 6;
    static constexpr int EPI_WARPS = 4 * (TN / 128);
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    // fp32 accumulators (two buffers of TN columns) + int32 level sums (TN columns)
    static constexpr int TMEM_COLS = (3 * TN <= 512) ? 512 : 1024;
    static constexpr int ACC_COL = 2 * TN;
    static constexpr int SMEM = STAGES * (STAGE_A + STAGE_B) + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr uint32_t IDESC = ptx::idesc_f32acc(1 /*bf16*/, OZ_TM, TN);
};

__device__ __forceinline__ void unit_coords(int64_t u, const OzParams& p, int& tm, int& tn, int& kseg, int& li) {
    const int64_t tiles = (int64_t)p.tiles_m * p.tiles_n;
    int64_t x = u % tiles;
    int64_t r = u / tiles;
    kseg = (int)(r % p.ksegs);
    li = (int)(r / p.ksegs);
    // grouped rasterisation: OZ_GROUP_M tile rows advance together
    const int64_t per_group = (int64_t)OZ_GROUP_M * p.tiles_n;
    const int64_t g = x / per_group;
    const int first_m = (int)(g * OZ_GROUP_M);
    const int gm = min(OZ_GROUP_M, p.tiles_m - first_m);
    const int64_t xi = x - g * per_group;
    tm = first_m + (int)(xi % gm);
    tn = (int)(xi / gm);
}

template <int TN>
__global__ void __launch_bounds__(OzCfg<TN>::THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams p) {
    using Cfg = OzCfg<TN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + Cfg::STAGES * Cfg::STAGE_A;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + Cfg::STAGES * Cfg::STAGE_B);
    uint64_t* empty = full + Cfg::STAGES;
    uint64_t* tfull = empty + Cfg::STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; s++) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            ptx::mbar_init(&tfull[b], 1);
            ptx::mbar_init(&tempty[b], Cfg::EPI_WARPS);
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
        ptx::tmem_alloc(tmem_holder, Cfg::TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    auto on_timeout = [&]() {
        atomicExch(p.err, 1);
        *abort_flag = 1;
    };

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            int64_t it = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
                int tm, tn, kseg, li;
                unit_coords(u, p, tm, tn, kseg, li);
                const int d = li + 2;
                const int kb0 = kseg * p.kseg_blocks;
                const int kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
                for (int t = 1; t < d && ok; t++) {
                    for (int kb = kb0; kb < kb1; kb++, it++) {
                        const int st = (int)(it % Cfg::STAGES);
                        const uint32_t ph = (uint32_t)((it / Cfg::STAGES) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, OZ_WAIT_NS)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::mbar_arrive_expect_tx(&full[st], Cfg::STAGE_A + Cfg::STAGE_B);
                        ptx::tma_load_3d(sA + st * Cfg::STAGE_A, &tmA, &full[st], kb * OZ_TK, tm * OZ_TM, t - 1);
                        ptx::tma_load_3d(sB + st * Cfg::STAGE_B, &tmB, &full[st], kb * OZ_TK, tn * TN, d - t - 1);
                    }
                }
            }
            // drain: the last issued stages must have landed before the CTA exits
            const int64_t first = it > Cfg::STAGES ? it - Cfg::STAGES : 0;
            for (int64_t q = first; q < it; q++) {
                if (!ptx::mbar_wait_bounded(&full[q % Cfg::STAGES], (uint32_t)((q / Cfg::STAGES) & 1),
                                            OZ_WAIT_NS)) {
                    on_timeout();
                    break;
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int64_t it = 0, ci = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
                int tm, tn, kseg, li;
                unit_coords(u, p, tm, tn, kseg, li);
                const int d = li + 2;
                const int kb0 = kseg * p.kseg_blocks;
                const int kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
                for (int t = 1; t < d && ok; t++) {
                    for (int c = kb0; c < kb1 && ok; c += OZ_CHUNK, ci++) {
                        const int buf = (int)(ci & 1);
                        const uint32_t aph = (uint32_t)((ci >> 1) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded(&tempty[buf], aph ^ 1u, OZ_WAIT_NS)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t dt = tmem + (uint32_t)(buf * TN);
                        const int ce = min(c + OZ_CHUNK, kb1);
                        for (int kb = c; kb < ce; kb++, it++) {
                            const int st = (int)(it % Cfg::STAGES);
                            const uint32_t ph = (uint32_t)((it / Cfg::STAGES) & 1);
                            if (*abort_flag || !ptx::mbar_wait_bounded(&full[st], ph, OZ_WAIT_NS)) {
                                if (!*abort_flag) on_timeout();
                                ok = false;
                                break;
                            }
                            ptx::tc_fence_after();
                            const uint64_t ad = ptx::smem_desc_sw128(sA + st * Cfg::STAGE_A);
                            const uint64_t bd = ptx::smem_desc_sw128(sB + st * Cfg::STAGE_B);
#pragma unroll
                            for (int kk = 0; kk < OZ_TK / 16; kk++) {
                                // advance 16 bf16 = 32 bytes along K inside the swizzled row
                                ptx::mma_f16_ss(dt, ad + (uint64_t)((kk * 32) >> 4), bd + (uint64_t)((kk * 32) >> 4),
                                                Cfg::IDESC, (kb > c || kk > 0) ? 1u : 0u);
                            }
                            ptx::mma_commit(&empty[st]);
                        }
                        if (ok) ptx::mma_commit(&tfull[buf]);
                    }
                }
            }
            // every issued MMA must be complete before TMEM is released
            ptx::mma_commit(drain);
            if (!ptx::mbar_wait_bounded(drain, 0, OZ_WAIT_NS)) on_timeout();
        }
    } else {
        // --------------------------------------------------------- epilogue
        // The exact int32 level sum of the unit lives in TMEM columns
        // [ACC_COL, ACC_COL + TN); each 1024-long fp32 stretch is added to it.
        const int ew = warp - 2;                  // 0 .. EPI_WARPS-1
        const int q = warp & 3;                   // TMEM lane quadrant this warp may access
        const int half = ew / 4;                  // 128-column half of the tile
        const int row = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 128);
        int64_t ci = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
            int tm, tn, kseg, li;
            unit_coords(u, p, tm, tn, kseg, li);
            const int d = li + 2;
            const int kb0 = kseg * p.kseg_blocks;
            const int kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
            const int nchunks = (d - 1) * ((kb1 - kb0 + OZ_CHUNK - 1) / OZ_CHUNK);
            for (int ch = 0; ch < nchunks; ch++, ci++) {
                const int buf = (int)(ci & 1);
                const uint32_t aph = (uint32_t)((ci >> 1) & 1);
                if (*abort_flag || !ptx::mbar_wait_bounded(&tfull[buf], aph, OZ_WAIT_NS)) {
                    if (!*abort_flag) on_timeout();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
#pragma unroll 1
                for (int g = 0; g < 4; g++) {
                    uint32_t r[32], a[32];
                    ptx::tmem_ld_32x32b_x32(tl + (uint32_t)(buf * TN + g * 32), r);
                    if (ch > 0) ptx::tmem_ld_32x32b_x32(tl + (uint32_t)(Cfg::ACC_COL + g * 32), a);
                    ptx::tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 32; c++) {
                        const int v = __float2int_rn(__uint_as_float(r[c]));
                        a[c] = (ch > 0) ? (uint32_t)((int)a[c] + v) : (uint32_t)v;
                    }
                    ptx::tmem_st_32x32b_x32(tl + (uint32_t)(Cfg::ACC_COL + g * 32), a);
                }
                ptx::tmem_wait_st();
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[buf]);
            }
            if (!ok) break;
            const int64_t i = (int64_t)tm * OZ_TM + row;
            double* out = p.ws + ((int64_t)li * p.ksegs + kseg) * p.ws_stride + i;
            const int64_t j0 = (int64_t)tn * TN + half * 128;
            out += j0 * p.M;
#pragma unroll 1
            for (int g = 0; g < 4; g++) {
                uint32_t a[32];
                ptx::tmem_ld_32x32b_x32(tl + (uint32_t)(Cfg::ACC_COL + g * 32), a);
                ptx::tmem_wait_ld();
                if (i < p.M) {
#pragma unroll
                    for (int c = 0; c < 32; c++) {
                        if (j0 + g * 32 + c < p.N) out[(int64_t)(g * 32 + c) * p.M] = (double)(int)a[c];
                    }
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda
// symbol needed at link time).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int get_encoder(EncodeTiledFn* fn) {
    static EncodeTiledFn cached = nullptr;
    if (!cached) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        DB_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
        if (!f || q != cudaDriverEntryPointSuccess)
            return fail(DBCSR_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        cached = reinterpret_cast<EncodeTiledFn>(f);
    }
    *fn = cached;
    return DBCSR_OK;
}

}  // namespace

// 3-D tensor map over [slices][rows][ldk] bf16 (ldk a multiple of 64),
// box 64 x box_rows x 1, 128-byte swizzle, zero fill out of bounds.
int make_slice_tmap(CUtensorMap* map, const void* base, int64_t ldk, int64_t rows, int slices, int box_rows,
                    int elem_bytes) {
    EncodeTiledFn enc;
    DB_TRY(get_encoder(&enc));
    cuuint64_t dims[3] = {(cuuint64_t)ldk, (cuuint64_t)rows, (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)(ldk * elem_bytes), (cuuint64_t)(ldk * rows * elem_bytes)};
    cuuint32_t box[3] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(DBCSR_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return DBCSR_OK;
}

int oz_gemm_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p, int tn) {
    if (p.units <= 0) return DBCSR_OK;
    cudaStream_t st = ctx().stream;
    const int grid = (int)std::min<int64_t>(p.units, ctx().num_sms);
    if (tn == 256) {
        using Cfg = OzCfg<256>;
        DB_CUDA(cudaFuncSetAttribute(k_oz_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
        k_oz_gemm<256><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(tmA, tmB, p);
    } else {
        using Cfg = OzCfg<128>;
        DB_CUDA(cudaFuncSetAttribute(k_oz_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
        k_oz_gemm<128><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(tmA, tmB, p);
    }
    DB_KCHECK();
    return DBCSR_OK;
}

}  // namespace dbcsr

namespace dbcsr {

// The same launch on an explicit stream and SM count, for callers that do not
// go through the library context.
int oz_gemm_launch_on(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p, cudaStream_t st,
                      int num_sms) {
    if (p.units <= 0) return DBCSR_OK;
    using Cfg = OzCfg<128>;
    const int grid = (int)std::min<int64_t>(p.units, num_sms);
    DB_CUDA(cudaFuncSetAttribute(k_oz_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
    k_oz_gemm<128><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(tmA, tmB, p);
    DB_KCHECK();
    return DBCSR_OK;
}

}  // namespace dbcsr
