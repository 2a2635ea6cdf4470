// tc_ozaki.cu -- tensor-core (tcgen05) GEMMs of the emulated paths.
//
// MODE_SLICES: integer-slice GEMMs of the emulated-FP64 product (Ozaki,
// Ogita, Oishi & Rump 2012, integer form): G_d = sum_{t+u=d} S^A_t * S^B_u.
// Slices are integers in [-127, 127], exactly representable in bf16; a bf16
// MMA (kind::f16) with fp32 accumulation is exact while every partial sum
// stays below 2^24, i.e. for up to 1040 products of two slices. The tensor
// core therefore accumulates 1024-long stretches of K in TMEM (fp32, exact)
// and the epilogue warps convert each stretch to int32 and add it to an int32
// sum that also lives in TMEM (exact while s * K_segment * 127^2 < 2^31: K
// segments of 16384). One work unit = one 128 x 128 output tile, one level d,
// one K segment; its exact integer level sum is written as FP64 (exact below
// 2^53) to a workspace that the recombination kernel reads.
//
// MODE_TF32: the TF32 variant -- operands are fp32 values already rounded to
// TF32, kind::tf32 MMAs accumulate the whole K in fp32, and the epilogue
// writes C = alpha * acc + beta * C (FP64 C) directly.
//
// Warp roles (one CTA per SM, persistent over work units):
//   warp 0      TMA producer: 128 x (128 bytes) tiles of A and B, 128-byte
//               swizzle, into a ring of shared-memory stages
//   warp 1      TMEM allocator; lane 0 issues tcgen05.mma (4 per stage) into
//               one of two TMEM accumulators and commits to mbarriers
//   warps 2..5  epilogue: tcgen05.ld, convert, accumulate / store
// Every mbarrier wait of the pipeline is bounded (OzParams::wait_ns on the
// global timer, 4 s unless a caller set another limit); on a timeout the
// kernel records an error flag, unwinds all roles, drains its TMA loads and
// MMAs (those clean-up waits always allow 4 s), frees TMEM and returns -- the
// host reports DBCSR_ERR_TIMEOUT. Each CTA loads its own A and B tiles.
#include <cuda.h>

#include "internal.cuh"
#include "sm100_ptx.cuh"
#include "tc_gemm.cuh"

namespace dbcsr {

namespace {

constexpr int MODE_SLICES = 0;
constexpr int MODE_TF32 = 1;

constexpr int TC_TM = 128;
constexpr int TC_TN = 128;
constexpr int TC_ROW_BYTES = 128;     // one 128-byte swizzle row of K per tile row
constexpr uint64_t TC_DRAIN_NS = 4000000000ull;   // clean-up waits before the CTA exits
constexpr int TC_GROUP_M = 16;        // tile rasterisation group (L2 reuse)

struct TcCfg {
    static constexpr int STAGE_A = TC_TM * TC_ROW_BYTES;
    static constexpr int STAGE_B = TC_TN * TC_ROW_BYTES;
    static constexpr int STAGES = 6;
    static constexpr int EPI_WARPS = 4;
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    // fp32 accumulators (two buffers of TC_TN columns) + int32 level sums
    static constexpr int TMEM_COLS = 512;
    static constexpr int ACC_COL = 2 * TC_TN;
    static constexpr int SMEM = STAGES * (STAGE_A + STAGE_B) + 1024 /*align*/ + 256 /*barriers*/;
};

template <int MODE>
struct ModeTraits;
template <>
struct ModeTraits<MODE_SLICES> {
    static constexpr uint32_t IDESC = ptx::idesc_f32acc(1 /*bf16*/, TC_TM, TC_TN);
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
        ptx::mma_f16_ss(d, a, b, IDESC, acc);
    }
};
template <>
struct ModeTraits<MODE_TF32> {
    static constexpr uint32_t IDESC = ptx::idesc_f32acc(2 /*tf32*/, TC_TM, TC_TN);
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
        ptx::mma_tf32_ss(d, a, b, IDESC, acc);
    }
};

// Work unit u -> (tile row, tile column, K segment, level): level-major, and
// within a level the tiles in groups of TC_GROUP_M tile rows.
__device__ __forceinline__ void unit_coords(int64_t u, const OzParams& p, int& tm, int& tn, int& kseg, int& li) {
    const int tiles_mc = p.tiles_m;
    const int64_t tiles = (int64_t)tiles_mc * p.tiles_n;
    int64_t x = u % tiles;
    int64_t r = u / tiles;
    kseg = (int)(r % p.ksegs);
    li = (int)(r / p.ksegs);
    // grouped rasterisation: TC_GROUP_M tile rows advance together
    const int64_t per_group = (int64_t)TC_GROUP_M * p.tiles_n;
    const int64_t g = x / per_group;
    const int first_m = (int)(g * TC_GROUP_M);
    const int gm = min(TC_GROUP_M, tiles_mc - first_m);
    const int64_t xi = x - g * per_group;
    tm = first_m + (int)(xi % gm);
    tn = (int)(xi / gm);
}

template <int MODE>
__global__ void __launch_bounds__(TcCfg::THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams p) {
    using Cfg = TcCfg;
    using Tr = ModeTraits<MODE>;
    const int64_t cl_id = blockIdx.x, n_cl = gridDim.x;
    const uint64_t wait_ns = p.wait_ns;
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
    const int kelems = TC_ROW_BYTES / p.elem_bytes;   // K elements per k-block

    auto on_timeout = [&]() {
        atomicExch(p.err, 1);
        *abort_flag = 1;
    };

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            int64_t it = 0;
            bool ok = true;
            for (int64_t u = cl_id; u < p.units && ok; u += n_cl) {
                int tm, tn, kseg, li;
                unit_coords(u, p, tm, tn, kseg, li);
                const int d = li + 2;
                const int kb0 = kseg * p.kseg_blocks;
                const int kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
                for (int t = 1; t < d && ok; t++) {
                    for (int kb = kb0; kb < kb1; kb++, it++) {
                        const int st = (int)(it % Cfg::STAGES);
                        const uint32_t ph = (uint32_t)((it / Cfg::STAGES) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, wait_ns)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::mbar_arrive_expect_tx(&full[st], Cfg::STAGE_A + Cfg::STAGE_B);
                        ptx::tma_load_3d(sA + st * Cfg::STAGE_A, &tmA, &full[st], kb * kelems, tm * TC_TM, t - 1);
                        ptx::tma_load_3d(sB + st * Cfg::STAGE_B, &tmB, &full[st], kb * kelems, tn * TC_TN, d - t - 1);
                    }
                }
            }
            // drain: the last issued stages must have landed before the CTA exits
            const int64_t first = it > Cfg::STAGES ? it - Cfg::STAGES : 0;
            for (int64_t q = first; q < it; q++) {
                if (!ptx::mbar_wait_bounded(&full[q % Cfg::STAGES], (uint32_t)((q / Cfg::STAGES) & 1),
                                            TC_DRAIN_NS)) {
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
            for (int64_t u = cl_id; u < p.units && ok; u += n_cl) {
                int tm, tn, kseg, li;
                unit_coords(u, p, tm, tn, kseg, li);
                const int d = li + 2;
                const int kb0 = kseg * p.kseg_blocks;
                const int kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
                for (int t = 1; t < d && ok; t++) {
                    for (int c = kb0; c < kb1 && ok; c += p.chunk_blocks, ci++) {
                        const int buf = (int)(ci & 1);
                        const uint32_t aph = (uint32_t)((ci >> 1) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded(&tempty[buf], aph ^ 1u, wait_ns)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t dt = tmem + (uint32_t)(buf * TC_TN);
                        const int ce = min(c + p.chunk_blocks, kb1);
                        for (int kb = c; kb < ce; kb++, it++) {
                            const int st = (int)(it % Cfg::STAGES);
                            const uint32_t ph = (uint32_t)((it / Cfg::STAGES) & 1);
                            if (*abort_flag || !ptx::mbar_wait_bounded(&full[st], ph, wait_ns)) {
                                if (!*abort_flag) on_timeout();
                                ok = false;
                                break;
                            }
                            ptx::tc_fence_after();
                            const uint64_t ad = ptx::smem_desc_sw128(sA + st * Cfg::STAGE_A);
                            const uint64_t bd = ptx::smem_desc_sw128(sB + st * Cfg::STAGE_B);
#pragma unroll
                            for (int kk = 0; kk < 4; kk++) {
                                // each MMA takes 32 bytes of K (16 bf16 / 8 tf32) of the swizzled row
                                Tr::mma(dt, ad + (uint64_t)((kk * 32) >> 4), bd + (uint64_t)((kk * 32) >> 4),
                                        (kb > c || kk > 0) ? 1u : 0u);
                            }
                            ptx::mma_commit(&empty[st]);
                        }
                        if (ok) ptx::mma_commit(&tfull[buf]);
                    }
                }
            }
            // every issued MMA must be complete before TMEM is released
            ptx::mma_commit(drain);
            if (!ptx::mbar_wait_bounded(drain, 0, TC_DRAIN_NS)) on_timeout();
        }
    } else {
        // --------------------------------------------------------- epilogue
        const BlasUpd bu(p.alpha, p.beta);
        const int q = warp & 3;                   // TMEM lane quadrant this warp may access
        const int row = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        int64_t ci = 0;
        bool ok = true;
        for (int64_t u = cl_id; u < p.units && ok; u += n_cl) {
            int tm, tn, kseg, li;
            unit_coords(u, p, tm, tn, kseg, li);
            const int d = li + 2;
            const int kb0 = kseg * p.kseg_blocks;
            const int kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
            const int nchunks = (d - 1) * ((kb1 - kb0 + p.chunk_blocks - 1) / p.chunk_blocks);
            const int64_t i = (int64_t)tm * TC_TM + row;
            const int64_t j0 = (int64_t)tn * TC_TN;
            for (int ch = 0; ch < nchunks; ch++, ci++) {
                const int buf = (int)(ci & 1);
                const uint32_t aph = (uint32_t)((ci >> 1) & 1);
                if (*abort_flag || !ptx::mbar_wait_bounded(&tfull[buf], aph, wait_ns)) {
                    if (!*abort_flag) on_timeout();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                if (MODE == MODE_SLICES) {
                    // add this exact fp32 stretch to the int32 level sum in TMEM
#pragma unroll 1
                    for (int g = 0; g < 4; g++) {
                        uint32_t r[32], a[32];
                        ptx::tmem_ld_32x32b_x32(tl + (uint32_t)(buf * TC_TN + g * 32), r);
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
                } else {
                    // whole K accumulated: C = alpha * acc + beta * C
#pragma unroll 1
                    for (int g = 0; g < 4; g++) {
                        uint32_t r[32];
                        ptx::tmem_ld_32x32b_x32(tl + (uint32_t)(buf * TC_TN + g * 32), r);
                        ptx::tmem_wait_ld();
                        if (i < p.M) {
#pragma unroll
                            for (int c = 0; c < 32; c++) {
                                const int64_t j = j0 + g * 32 + c;
                                if (j < p.N) {
                                    double* cp = p.C + i + j * p.ldc;
                                    const double x = (double)__uint_as_float(r[c]);
                                    *cp = bu.old ? bu.update(x, *cp) : bu.scale(x);
                                }
                            }
                        }
                    }
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[buf]);
            }
            if (!ok) break;
            if (MODE == MODE_SLICES) {
                double* out = p.ws + ((int64_t)li * p.ksegs + kseg) * p.ws_stride + i + j0 * p.M;
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

template <int MODE>
int launch_mode(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p, cudaStream_t st, int num_sms) {
    OzParams q = p;
    q.units = (int64_t)p.tiles_m * p.tiles_n * p.ksegs * p.s;
    if (q.units <= 0) return DBCSR_OK;
    const int grid = (int)std::min<int64_t>(q.units, num_sms);
    auto kern = k_tc_gemm<MODE>;
    DB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg::SMEM));
    kern<<<grid, TcCfg::THREADS, TcCfg::SMEM, st>>>(tmA, tmB, q);
    DB_KCHECK();
    return DBCSR_OK;
}

}  // namespace

// 3-D tensor map over [slices][rows][ldk] elements (ldk * elem_bytes a
// multiple of 128), box (128 bytes of K) x box_rows x 1, 128-byte swizzle,
// zero fill out of bounds.
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

int oz_gemm_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p) {
    return launch_mode<MODE_SLICES>(tmA, tmB, p, ctx().stream, ctx().num_sms);
}

int oz_gemm_launch_on(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p, cudaStream_t st,
                      int num_sms) {
    return launch_mode<MODE_SLICES>(tmA, tmB, p, st, num_sms);
}

int tf32_gemm_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p) {
    return launch_mode<MODE_TF32>(tmA, tmB, p, ctx().stream, ctx().num_sms);
}

}  // namespace dbcsr
