// tc_gemm2sm.cu -- the slice GEMM of the emulated-FP64 path on CTA pairs:
// 256 x 256 output tiles, one tile per pair of CTAs (a cluster of two), with
// tcgen05 MMAs of M = 256, N = 256, K = 16 (.cta_group::2).
//
// Same work decomposition and arithmetic as k_tc_gemm256 (see tc_gemm256.cu
// and tc_ozaki.cu): one work unit is one output tile, one level d and one K
// segment; the exact fp32 stretches of 1024 K are flushed into int32 level
// sums held in the epilogue warps' registers and written once per unit.
//
// What the pair changes: CTA r (r = 0, 1) loads rows r*128 .. r*128+127 of the
// tile's A panel and of its B panel into its own shared memory (each CTA loads
// its own halves: no copy is shared between CTAs). The even CTA issues every
// MMA; the tensor cores read A's two halves (M) and B's two halves (N) from
// the same shared-memory offsets of both CTAs and write rows r*128 .. of the
// fp32 accumulator into CTA r's tensor memory. Per tile, 256 + 256 operand
// rows feed 256 x 256 outputs instead of 128 + 256 rows feeding 128 x 256:
// a third less operand traffic from L2 per flop.
//
// Signals between the two CTAs (cluster addresses from mapa):
//   - both CTAs' TMA loads of a stage complete on the even CTA's `full`
//     barrier (the even producer expects the bytes of both);
//   - the MMA issuer commits each consumed stage to the `empty` barriers and
//     each finished accumulator to the `tfull` barriers of both CTAs;
//   - all sixteen epilogue warps of the pair arrive on the even CTA's `tempty`.
// Before the pair's final cluster barrier the even CTA waits until its last
// stages have landed and its MMAs are complete, and the odd CTA waits until
// its last stages have been consumed (which implies that they landed); when
// a wait gives up, each of these waits still allows 4 s, far longer than any
// copy in flight takes, so no CTA leaves while a copy into it can land.
// Warps: 0 TMA producer, 1 TMEM allocator (both CTAs, collectively) and MMA
// issuer (even CTA), 2-3 idle, 4-11 epilogue; setmaxnreg split as in the
// 128 x 256 kernel. Every pipeline wait is bounded (OzParams::wait_ns).
#include <cuda.h>

#include "internal.cuh"
#include "sm100_ptx.cuh"
#include "tc_gemm.cuh"

namespace dbcsr {

namespace {

constexpr int P_TM = 256, P_TN = 256, P_HALF = 128, P_ROW_BYTES = 128;
constexpr int P_STAGE_A = P_HALF * P_ROW_BYTES;   // 16 KB: this CTA's 128 rows of A
constexpr int P_STAGE_B = P_HALF * P_ROW_BYTES;   // 16 KB: this CTA's 128 rows of B
constexpr int P_STAGE = P_STAGE_A + P_STAGE_B;
constexpr int P_STAGES = 6;
constexpr int P_THREADS = 384;
constexpr int P_EPI_WARPS = 8;                    // per CTA
constexpr int P_LAUNCH_REGS = 168;
constexpr int P_REGS_CTRL = 56, P_REGS_EPI = 224;
static_assert(128 * P_REGS_CTRL + 256 * P_REGS_EPI <= P_THREADS * P_LAUNCH_REGS, "register split exceeds launch");
constexpr int P_SMEM = P_STAGES * P_STAGE + 1024 + 256;
constexpr uint64_t P_DRAIN_NS = 4000000000ull;
constexpr int P_GROUP_M = 8;                      // tile rows (of 256) that advance together
constexpr uint32_t P_IDESC = ptx::idesc_f32acc(1 /*bf16*/, P_TM, P_TN);

__device__ __forceinline__ void p_unit(int u, const OzParams& p, int tiles_m2, int tiles_n, int& tm2, int& tn,
                                       int& kseg, int& li) {
    const int tiles = tiles_m2 * tiles_n;
    const int x = u % tiles, r = u / tiles;
    kseg = r % p.ksegs;
    li = r / p.ksegs;
    const int per_group = P_GROUP_M * tiles_n;
    const int g = x / per_group;
    const int first_m = g * P_GROUP_M;
    const int gm = min(P_GROUP_M, tiles_m2 - first_m);
    const int xi = x - g * per_group;
    tm2 = first_m + xi % gm;
    tn = xi / gm;
}

__global__ void __launch_bounds__(P_THREADS, 1)
    k_tc_gemm2sm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + P_STAGES * P_STAGE_A;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + P_STAGES * P_STAGE_B);
    uint64_t* empty = full + P_STAGES;
    uint64_t* tfull = empty + P_STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = ptx::cluster_ctarank();
    const bool lead = rank == 0;
    const int cl_id = (int)(blockIdx.x >> 1), n_cl = (int)(gridDim.x >> 1);
    const int tiles_m2 = (p.M + P_TM - 1) / P_TM, tiles_n = (p.N + P_TN - 1) / P_TN;
    const uint64_t wait_ns = p.wait_ns;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P_STAGES; s++) {
            ptx::mbar_init(&full[s], 1);    // even CTA: its producer's arrive.expect_tx (bytes of both CTAs)
            ptx::mbar_init(&empty[s], 1);   // one commit of the MMA issuer
        }
        for (int b = 0; b < 2; b++) {
            ptx::mbar_init(&tfull[b], 1);
            ptx::mbar_init(&tempty[b], 2 * P_EPI_WARPS);
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
        ptx::tmem_alloc_pair(tmem_holder, 512);
        ptx::tmem_relinquish_pair();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::cluster_sync();   // the peer's barriers are initialised before any arrival on them
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const int kelems = P_ROW_BYTES / p.elem_bytes;
    auto on_timeout = [&]() {
        atomicExch(p.err, 1);
        *abort_flag = 1;
    };

    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(P_REGS_CTRL));
        if (warp == 0 && lane == 0) {
            // -------------------------------------------- TMA producer (both CTAs)
            int64_t it = 0;
            bool ok = true;
            const uint32_t full_c = ptx::mapa_shared(full, 0);   // the even CTA's `full` barriers
            for (int u = cl_id; u < (int)p.units && ok; u += n_cl) {
                int tm2, tn, kseg, li;
                p_unit(u, p, tiles_m2, tiles_n, tm2, tn, kseg, li);
                const int d = li + 2;
                const int kb0 = kseg * p.kseg_blocks, kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
                for (int t = 1; t < d && ok; t++)
                    for (int kb = kb0; kb < kb1; kb++, it++) {
                        const int st = (int)(it % P_STAGES);
                        const uint32_t ph = (uint32_t)((it / P_STAGES) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded_cluster(&empty[st], ph ^ 1u, wait_ns)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        if (lead) ptx::mbar_arrive_expect_tx(&full[st], 2 * P_STAGE);
                        const uint32_t fb = full_c + (uint32_t)(st * 8);
                        ptx::tma_load_3d_pair(sA + st * P_STAGE_A, &tmA, fb, kb * kelems,
                                              tm2 * P_TM + (int)rank * P_HALF, t - 1);
                        ptx::tma_load_3d_pair(sB + st * P_STAGE_B, &tmB, fb, kb * kelems,
                                              tn * P_TN + (int)rank * P_HALF, d - t - 1);
                    }
            }
            // this CTA's last copies have landed before it may leave: the even
            // CTA sees its `full` phases complete, the odd one its stages consumed
            const int64_t first = it > P_STAGES ? it - P_STAGES : 0;
            for (int64_t q = first; q < it; q++) {
                const uint32_t ph = (uint32_t)((q / P_STAGES) & 1);
                const bool done = lead ? ptx::mbar_wait_bounded_cluster(&full[q % P_STAGES], ph, P_DRAIN_NS)
                                       : ptx::mbar_wait_bounded_cluster(&empty[q % P_STAGES], ph, P_DRAIN_NS);
                if (!done) {
                    on_timeout();
                    break;
                }
            }
        } else if (warp == 1 && lane == 0 && lead) {
            // ------------------------------------------ MMA issuer (even CTA)
            int64_t it = 0, ci = 0;
            bool ok = true;
            const uint32_t empty0 = ptx::mapa_shared(empty, 0), empty1 = ptx::mapa_shared(empty, 1);
            const uint32_t tfull0 = ptx::mapa_shared(tfull, 0), tfull1 = ptx::mapa_shared(tfull, 1);
            for (int u = cl_id; u < (int)p.units && ok; u += n_cl) {
                int tm2, tn, kseg, li;
                p_unit(u, p, tiles_m2, tiles_n, tm2, tn, kseg, li);
                const int d = li + 2;
                const int kb0 = kseg * p.kseg_blocks, kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
                for (int t = 1; t < d && ok; t++)
                    for (int c = kb0; c < kb1 && ok; c += p.chunk_blocks, ci++) {
                        const int buf = (int)(ci & 1);
                        const uint32_t aph = (uint32_t)((ci >> 1) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded_cluster(&tempty[buf], aph ^ 1u, wait_ns)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t dt = tmem + (uint32_t)(buf * P_TN);
                        const int ce = min(c + p.chunk_blocks, kb1);
                        for (int kb = c; kb < ce; kb++, it++) {
                            const int st = (int)(it % P_STAGES);
                            const uint32_t ph = (uint32_t)((it / P_STAGES) & 1);
                            if (*abort_flag || !ptx::mbar_wait_bounded_cluster(&full[st], ph, wait_ns)) {
                                if (!*abort_flag) on_timeout();
                                ok = false;
                                break;
                            }
                            ptx::tc_fence_after();
                            const uint64_t ad = ptx::smem_desc_sw128(sA + st * P_STAGE_A);
                            const uint64_t bd = ptx::smem_desc_sw128(sB + st * P_STAGE_B);
#pragma unroll
                            for (int kk = 0; kk < 4; kk++)
                                ptx::mma_f16_ss_pair(dt, ad + (uint64_t)((kk * 32) >> 4),
                                                     bd + (uint64_t)((kk * 32) >> 4), P_IDESC,
                                                     (kb > c || kk > 0) ? 1u : 0u);
                            // the stage is free in both CTAs once these MMAs have read it
                            ptx::mma_commit_pair(empty0 + (uint32_t)(st * 8));
                            ptx::mma_commit_pair(empty1 + (uint32_t)(st * 8));
                        }
                        if (ok) {
                            ptx::mma_commit_pair(tfull0 + (uint32_t)(buf * 8));
                            ptx::mma_commit_pair(tfull1 + (uint32_t)(buf * 8));
                        }
                    }
            }
            // every issued MMA is complete before tensor memory is released
            ptx::mma_commit_pair(ptx::mapa_shared(drain, 0));
            if (!ptx::mbar_wait_bounded(drain, 0, P_DRAIN_NS)) on_timeout();
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(P_REGS_EPI));
        // ------------------------------------------------ epilogue (both CTAs)
        const int q = warp & 3;
        const int half = (warp - 4) >> 2;
        const int row = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 128);
        int64_t ci = 0;
        bool ok = true;
        const uint32_t tempty_c = ptx::mapa_shared(tempty, 0);
        for (int u = cl_id; u < (int)p.units && ok; u += n_cl) {
            int tm2, tn, kseg, li;
            p_unit(u, p, tiles_m2, tiles_n, tm2, tn, kseg, li);
            const int d = li + 2;
            const int kb0 = kseg * p.kseg_blocks, kb1 = min(kb0 + p.kseg_blocks, p.kblocks);
            const int nchunks = (d - 1) * ((kb1 - kb0 + p.chunk_blocks - 1) / p.chunk_blocks);
            const int64_t i = (int64_t)tm2 * P_TM + (int64_t)rank * P_HALF + row;
            const int64_t j0 = (int64_t)tn * P_TN + half * 128;
            int acc[128];
#pragma unroll
            for (int c = 0; c < 128; c++) acc[c] = 0;
            for (int ch = 0; ch < nchunks; ch++, ci++) {
                const int buf = (int)(ci & 1);
                const uint32_t aph = (uint32_t)((ci >> 1) & 1);
                if (*abort_flag || !ptx::mbar_wait_bounded_cluster(&tfull[buf], aph, wait_ns)) {
                    if (!*abort_flag) on_timeout();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                // 16 columns at a time: the 128 sums plus one 16-register staging set fit the budget
#pragma unroll
                for (int g = 0; g < 8; g++) {
                    uint32_t r[16];
                    ptx::tmem_ld_32x32b_x16(tl + (uint32_t)(buf * P_TN + g * 16), r);
                    ptx::tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 16; c++) acc[g * 16 + c] += __float2int_rn(__uint_as_float(r[c]));
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive_cluster(tempty_c + (uint32_t)(buf * 8));
            }
            if (!ok) break;
            if (i < p.M) {
                int* out = p.ws_i32 + (((int64_t)li * p.ksegs + kseg) * p.M + i) * p.ldws + j0;
#pragma unroll
                for (int c = 0; c < 128; c += 4)
                    *reinterpret_cast<int4*>(out + c) = make_int4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    // neither CTA leaves while the pair's MMAs may still write its tensor memory
    // or the other CTA may still arrive on its barriers
    ptx::cluster_sync();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc_pair(tmem, 512);
}

}  // namespace

bool tc2sm_usable() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_tc_gemm2sm) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return fa.numRegs == P_LAUNCH_REGS;
}

// ws_i32 rows of ldws >= cdiv(N, 256) * 256 columns; tmA, tmB boxes of 128 rows
int oz_gemm2sm_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p) {
    OzParams q = p;
    const int64_t tiles_m2 = cdiv(p.M, P_TM), tiles_n = cdiv(p.N, P_TN);
    q.units = tiles_m2 * tiles_n * p.ksegs * p.s;
    if (q.units <= 0) return DBCSR_OK;
    if (q.units >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "pair slice GEMM: too many work units");
    cudaFuncAttributes fa;
    DB_CUDA(cudaFuncGetAttributes(&fa, k_tc_gemm2sm));
    if (fa.numRegs != P_LAUNCH_REGS)   // the setmaxnreg split assumes exactly this launch budget
        return fail(DBCSR_ERR_STATE, "pair slice GEMM built with " + std::to_string(fa.numRegs) +
                                         " registers per thread, expected " + std::to_string(P_LAUNCH_REGS));
    DB_CUDA(cudaFuncSetAttribute(k_tc_gemm2sm, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(P_THREADS);
    cfg.dynamicSmemBytes = P_SMEM;
    cfg.stream = ctx().stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2);
    int active = 0;   // pairs resident at once (persistent: no more are launched)
    DB_CUDA(cudaOccupancyMaxActiveClusters(&active, k_tc_gemm2sm, &cfg));
    if (active < 1) return fail(DBCSR_ERR_CUDA, "pair slice GEMM: no pair of CTAs fits on this GPU");
    const int64_t pairs = std::min<int64_t>(q.units, active);
    cfg.gridDim = dim3((unsigned)(2 * pairs));
    DB_CUDA(cudaLaunchKernelEx(&cfg, k_tc_gemm2sm, tmA, tmB, q));
    DB_KCHECK();
    return DBCSR_OK;
}

}  // namespace dbcsr
