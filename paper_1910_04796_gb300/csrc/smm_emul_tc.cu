// smm_emul_tc.cu -- the stack path in emulated FP64 on the 5th-generation
// tensor cores (tcgen05): every block product's slice pairs are tensor-core
// MMAs into fp32 accumulators in tensor memory (TMEM).
//
// Arithmetic as in smm_emul.cu (integer-slice emulation after Ozaki, Ogita,
// Oishi & Rump 2012): with P_tu = sum over the C block's products of
// A_t * B_u (slices t of the A blocks, u of the B blocks, integers in
// [-127, 127]) and the level sums G_d = sum_{t+u=d} P_tu,
//   C(i,j) = alpha * round(sum_d G_d(i,j) 2^(7(s+1-d)) * 2^(e_i+f_j-7(s+1))) + beta * C_old(i,j),
// the 128-bit sum exact, rounded once -- the same value the oracle computes.
//
// Operand layout. Every block is padded to 32 x 32. The s slices of each
// stored block are written once, slice after slice, in the no-swizzle K-major
// operand layout of tcgen05: 8-row x 16-byte core matrices, core (r/8, k/8)
// at byte ((r/8) * 4 + k/8) * 128 of the slice (leading-dimension byte offset
// 128 between K neighbours, stride byte offset 512 between 8-row groups).
// Consecutive slices therefore form one taller operand, and one bulk copy
// brings all s slices of a block into shared memory. Per product two MMA
// groups, each K = 32 (two K = 16 instructions):
//   G1: rows A slices 1..4 (M = 128) x columns B slices 1..s (N = 32 s)
//   G2: rows A slices 5..8 (M = 128) x columns B slices 1..s-4 (N = 32 (s-4))
// so pair (t, u) owns the 32 x 32 accumulator block at TMEM lanes 32 (t-1)
// (mod 128) and columns 32 (u-1) (+ 32 s for G2); pairs with t + u > s + 1
// are computed and ignored. An fp32 accumulator is exact for 32 products
// (32 * 32 * 127^2 < 2^24): a C block's products run in chunks of 32.
//
// Warps: 0 bulk-copy producer (one lane), 1 TMEM owner and MMA issuer (one
// lane), 2-5 epilogue; epilogue warp w reads TMEM lane quadrant q = w % 4,
// i.e. A slice t = q + 1 of G1 and t = q + 5 of G2. Per chunk the epilogue
//   1. drains TMEM: level d's contribution of its slices, P_{t,d-t} (+ the
//      G2 term), converted exactly to int32, into a level block in shared
//      memory; then releases TMEM, so the next chunk's MMAs overlap the rest;
//   2. sums the level blocks of the four quadrants into per-thread int32
//      level sums (thread: row i = lane, columns 8 q .. 8 q + 7).
// After the C block's last chunk it recombines, rounds, scales and stores.
// int32 level sums are exact while products * s * 32 * 127^2 < 2^31 (checked
// on the host). Every wait is bounded (4 s): on expiry the kernel sets the
// error flag, the other roles see the abort flag, every role leaves its loop
// and TMEM is freed.
#include <cuda_bf16.h>

#include "emul_common.cuh"
#include "internal.cuh"
#include "sm100_ptx.cuh"
#include "smm_emul.cuh"

namespace dbcsr {

namespace {

constexpr int TC_THREADS = 192;
constexpr int TC_SLOT = 2048;                 // one 32 x 32 bf16 slice
constexpr int TC_SMEM_CAP = 232448;           // 227 KB of shared memory per CTA
constexpr int TC_SMEM_MIN = 120 * 1024;       // one CTA per SM: it allocates all 512 TMEM columns
constexpr int TC_CHUNK = 32;                  // products per exact fp32 stretch
constexpr uint64_t TC_WAIT_NS = 4000000000ull;

template <int S>
struct TcGeo {
    static constexpr int STAGE = 2 * S * TC_SLOT;                 // A then B slices of one product
    static constexpr int T1 = S < 4 ? S : 4;                      // A slices of G1 that exist
    static constexpr int N1 = 32 * S;
    static constexpr int N2 = S > 4 ? 32 * (S - 4) : 0;
    static constexpr int NBLK = T1 * S - T1 * (T1 - 1) / 2;       // level blocks of the staging area
    static constexpr int STG = NBLK * 4096;                       // 32 x 32 int32 each
    static constexpr int RESERVE = 1024 + 256;                    // alignment + barriers
    static constexpr int NST0 = (TC_SMEM_CAP - RESERVE - STG) / STAGE;
    static constexpr int NST = NST0 > 6 ? 6 : NST0;
    static constexpr int SMEM0 = NST * STAGE + STG + RESERVE;
    static constexpr int SMEM = SMEM0 < TC_SMEM_MIN ? TC_SMEM_MIN : SMEM0;
    static constexpr uint32_t IDESC1 = ptx::idesc_f32acc(1, 128, N1);
    static constexpr uint32_t IDESC2 = ptx::idesc_f32acc(1, 128, N2 > 0 ? N2 : 32);
    static_assert(N1 + N2 <= 512, "accumulators exceed TMEM");
    static_assert(NST >= 2, "at least two pipeline stages");
};

// staging block of quadrant w (A slice w + 1) for level d, w + 2 <= d <= S + 1
template <int S>
__host__ __device__ constexpr int lvl_blk(int w, int d) {
    return w * S - w * (w - 1) / 2 + (d - w - 2);
}

struct TcArgs {
    int64_t nC;
    const int* c_row;
    const int* c_col;
    const int64_t* c_off;
    const int* c_old;
    const int64_t* c_pstart;
    const int2* prod;
    const int* rsC;
    const int* csC;
    const int64_t* croff;
    const int64_t* ccoff;
    const int* e;               // exponents of C's element rows
    const int* f;               // exponents of C's element columns
    const uint8_t* SA;          // s slices (2 KB each) per stored A block
    const uint8_t* SB;
    double* Cd;
    const double* Cold;
    const int64_t* Cold_off;
    double alpha, beta;
    int* err;
};

// Slices of every stored block in the operand layout above, zero-padded to
// 32 x 32: warp per block, lane per 8-element chunk of a row.
__global__ void k_tc_slice(SliceGeom G, const int* __restrict__ ex, int s, uint8_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = w0; b < G.nblks; b += nw) {
        int X, L, xs, ls;
        int64_t xbase;
        geom_block(G, b, X, L, xs, ls, xbase);
        const double* d = G.data + G.off[b];
        __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out + b * (int64_t)s * TC_SLOT);
        for (int c = lane; c < 128; c += 32) {
            const int x = c >> 2, l8 = c & 3;
            long long q[8];
            const int e = x < X ? ex[xbase + x] : 0;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int l = l8 * 8 + k;
                q[k] = (x < X && l < L) ? emul::fixed_point(d[(int64_t)x * xs + (int64_t)l * ls], e, s) : 0;
            }
            const int pos = ((x >> 3) * 4 + l8) * 64 + (x & 7) * 8;
            for (int t = 1; t <= s; t++) {
                uint32_t w[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const __nv_bfloat162 pr = __halves2bfloat162(emul::slice_bf16(q[2 * k], t, s),
                                                                 emul::slice_bf16(q[2 * k + 1], t, s));
                    w[k] = *reinterpret_cast<const uint32_t*>(&pr);
                }
                *reinterpret_cast<uint4*>(o + (t - 1) * 1024 + pos) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

// all lanes of the warp agree: the wait succeeded and no role aborted
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    bool ok = !*abort_flag && ptx::mbar_wait_bounded(bar, parity, TC_WAIT_NS);
    return __all_sync(0xffffffffu, ok);
}

template <int S>
__global__ void __launch_bounds__(TC_THREADS, 1) k_smm_emul_tc(TcArgs a) {
    using G = TcGeo<S>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* stages = smem;
    uint8_t* stg = smem + G::NST * G::STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(stg + G::STG);
    uint64_t* empty = full + G::NST;
    uint64_t* tfull = empty + G::NST;   // MMA -> epilogue: a chunk's pair sums are in TMEM
    uint64_t* tempty = tfull + 1;       // epilogue -> MMA: TMEM drained
    uint64_t* sfull = tempty + 1;       // staging area written by all epilogue threads
    uint64_t* sfree = sfull + 1;        // staging area read by all epilogue threads
    uint64_t* drain = sfree + 1;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < G::NST; i++) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        ptx::mbar_init(tfull, 1);
        ptx::mbar_init(tempty, 128);
        ptx::mbar_init(sfull, 128);
        ptx::mbar_init(sfree, 128);
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_holder, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    auto on_timeout = [&]() {
        atomicExch(a.err, 1);
        *abort_flag = 1;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ bulk-copy producer
            int64_t it = 0;
            bool ok = true;
            for (int64_t cb = blockIdx.x; cb < a.nC && ok; cb += gridDim.x) {
                const int64_t p1 = a.c_pstart[cb + 1];
                for (int64_t p = a.c_pstart[cb]; p < p1; p++, it++) {
                    const int st = (int)(it % G::NST);
                    const uint32_t ph = (uint32_t)((it / G::NST) & 1);
                    if (*abort_flag || !ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, TC_WAIT_NS)) {
                        if (!*abort_flag) on_timeout();
                        ok = false;
                        break;
                    }
                    const int2 pr = a.prod[p];
                    uint8_t* sa = stages + st * G::STAGE;
                    ptx::mbar_arrive_expect_tx(&full[st], G::STAGE);
                    ptx::bulk_load(sa, a.SA + (int64_t)pr.x * (S * TC_SLOT), S * TC_SLOT, &full[st]);
                    ptx::bulk_load(sa + S * TC_SLOT, a.SB + (int64_t)pr.y * (S * TC_SLOT), S * TC_SLOT, &full[st]);
                }
            }
            // no copy may still be in flight when the CTA exits
            const int64_t first = it > G::NST ? it - G::NST : 0;
            for (int64_t q = first; q < it; q++)
                if (!ptx::mbar_wait_bounded(&full[q % G::NST], (uint32_t)((q / G::NST) & 1), TC_WAIT_NS)) {
                    on_timeout();
                    break;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------ MMA issuer
            int64_t it = 0, ci = 0;
            bool ok = true;
            for (int64_t cb = blockIdx.x; cb < a.nC && ok; cb += gridDim.x) {
                const int64_t p0 = a.c_pstart[cb], p1 = a.c_pstart[cb + 1];
                for (int64_t c0 = p0; c0 < p1 && ok; c0 += TC_CHUNK, ci++) {
                    if (*abort_flag || !ptx::mbar_wait_bounded(tempty, (uint32_t)((ci & 1) ^ 1), TC_WAIT_NS)) {
                        if (!*abort_flag) on_timeout();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int64_t c1 = c0 + TC_CHUNK < p1 ? c0 + TC_CHUNK : p1;
                    for (int64_t p = c0; p < c1; p++, it++) {
                        const int st = (int)(it % G::NST);
                        const uint32_t ph = (uint32_t)((it / G::NST) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded(&full[st], ph, TC_WAIT_NS)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint8_t* sa = stages + st * G::STAGE;
                        const uint64_t a1 = ptx::smem_desc_kmajor(sa, 128, 512);
                        const uint64_t a2 = ptx::smem_desc_kmajor(sa + 4 * TC_SLOT, 128, 512);
                        const uint64_t bd = ptx::smem_desc_kmajor(sa + S * TC_SLOT, 128, 512);
#pragma unroll
                        for (int ks = 0; ks < 2; ks++) {
                            // the second K = 16 step starts two core matrices (256 bytes) further
                            const uint32_t acc = (p > c0 || ks > 0) ? 1u : 0u;
                            ptx::mma_f16_ss(tmem, a1 + (uint64_t)(ks * 16), bd + (uint64_t)(ks * 16), G::IDESC1, acc);
                            if (G::N2 > 0)
                                ptx::mma_f16_ss(tmem + (uint32_t)G::N1, a2 + (uint64_t)(ks * 16),
                                                bd + (uint64_t)(ks * 16), G::IDESC2, acc);
                        }
                        ptx::mma_commit(&empty[st]);
                    }
                    if (ok) ptx::mma_commit(tfull);
                }
            }
            ptx::mma_commit(drain);
            if (!ptx::mbar_wait_bounded(drain, 0, TC_WAIT_NS)) on_timeout();
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        const int t1 = q + 1, t2 = q + 5;
        int64_t ci = 0;
        bool ok = true;
        for (int64_t cb = blockIdx.x; cb < a.nC && ok; cb += gridDim.x) {
            const int64_t p0 = a.c_pstart[cb], p1 = a.c_pstart[cb + 1];
            int lv[S][8];
#pragma unroll
            for (int d = 0; d < S; d++)
#pragma unroll
                for (int k = 0; k < 8; k++) lv[d][k] = 0;
            for (int64_t c0 = p0; c0 < p1; c0 += TC_CHUNK, ci++) {
                const uint32_t ph = (uint32_t)(ci & 1);
                if (!warp_wait(tfull, ph, abort_flag) || !warp_wait(sfree, ph ^ 1u, abort_flag)) {
                    if (!*abort_flag) on_timeout();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                // 1. drain: level d of slice t1 (and t2), exact fp32 integers -> int32
                if (t1 <= S) {
                    for (int d = t1 + 1; d <= S + 1; d++) {
                        const bool two = (G::N2 > 0) && (t2 <= S) && (d - t2 >= 1);
                        uint32_t r1[32], r2[32];
                        ptx::tmem_ld_32x32b_x32(tl + (uint32_t)((d - t1 - 1) * 32), r1);
                        if (two) ptx::tmem_ld_32x32b_x32(tl + (uint32_t)(G::N1 + (d - t2 - 1) * 32), r2);
                        ptx::tmem_wait_ld();
                        uint8_t* row = stg + lvl_blk<S>(q, d) * 4096 + lane * 128;
#pragma unroll
                        for (int c8 = 0; c8 < 8; c8++) {
                            int v[4];
#pragma unroll
                            for (int k = 0; k < 4; k++) {
                                v[k] = __float2int_rn(__uint_as_float(r1[c8 * 4 + k]));
                                if (two) v[k] += __float2int_rn(__uint_as_float(r2[c8 * 4 + k]));
                            }
                            // 16-byte chunks XOR-swizzled by row: conflict-free stores and loads
                            *reinterpret_cast<int4*>(row + ((c8 ^ (lane & 7)) << 4)) = make_int4(v[0], v[1], v[2], v[3]);
                        }
                    }
                }
                ptx::tc_fence_before();
                ptx::mbar_arrive(tempty);
                ptx::mbar_arrive(sfull);
                if (!warp_wait(sfull, ph, abort_flag)) {
                    if (!*abort_flag) on_timeout();
                    ok = false;
                    break;
                }
                // 2. level sums of row i = lane, columns 8 q .. 8 q + 7
#pragma unroll
                for (int d = 2; d <= S + 1; d++)
#pragma unroll
                    for (int w = 0; w < G::T1; w++)
                        if (w + 2 <= d) {
                            const uint8_t* row = stg + lvl_blk<S>(w, d) * 4096 + lane * 128;
                            const int4 x0 = *reinterpret_cast<const int4*>(row + (((2 * q) ^ (lane & 7)) << 4));
                            const int4 x1 = *reinterpret_cast<const int4*>(row + (((2 * q + 1) ^ (lane & 7)) << 4));
                            lv[d - 2][0] += x0.x;
                            lv[d - 2][1] += x0.y;
                            lv[d - 2][2] += x0.z;
                            lv[d - 2][3] += x0.w;
                            lv[d - 2][4] += x1.x;
                            lv[d - 2][5] += x1.y;
                            lv[d - 2][6] += x1.z;
                            lv[d - 2][7] += x1.w;
                        }
                ptx::mbar_arrive(sfree);
            }
            if (!ok) break;
            // 3. exact recombination, one rounding, alpha / beta, column-major C block
            const int br = a.c_row[cb], bc = a.c_col[cb];
            const int m = a.rsC[br], n = a.csC[bc];
            const int i = lane;
            if (i < m) {
                const int64_t cbase = a.ccoff[bc];
                const int ei = a.e[a.croff[br] + i];
                double* cout = a.Cd + a.c_off[cb];
                const int old = a.c_old ? a.c_old[cb] : -1;
                const double* cold = old >= 0 ? a.Cold + a.Cold_off[old] : nullptr;
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int j = 8 * q + k;
                    if (j < n) {
                        __int128 Sx = 0;
#pragma unroll
                        for (int d = 0; d < S; d++) Sx += (__int128)lv[d][k] << (7 * (S - 1 - d));
                        double v = __dmul_rn(a.alpha,
                                             emul::round_i128_scaled(Sx, ei + a.f[cbase + j] - 7 * (S + 1)));
                        const int64_t idx = (int64_t)j * m + i;
                        if (cold) v = __dadd_rn(v, __dmul_rn(a.beta, cold[idx]));
                        cout[idx] = v;
                    }
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem, 512);
}

template <int S>
int launch_tc(const TcArgs& a, int grid) {
    using G = TcGeo<S>;
    DB_CUDA(cudaFuncSetAttribute(k_smm_emul_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    k_smm_emul_tc<S><<<grid, TC_THREADS, G::SMEM, ctx().stream>>>(a);
    DB_KCHECK();
    return DBCSR_OK;
}

template <int S>
double issued_per_product() {
    using G = TcGeo<S>;
    return 2.0 * 128.0 * (double)(G::N1 + G::N2) * 32.0;
}

}  // namespace

bool smm_emul_tc_usable() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_smm_emul_tc<7>) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

int smm_emul_tc(const SmmArgs& g, dbcsr_matrix_s* A, bool ta, dbcsr_matrix_s* B, bool tb, dbcsr_matrix_s* C,
                const int* e, const int* f, int s, int64_t nprod, double* issued_flops) {
    cudaStream_t st = ctx().stream;
    DBuf<uint8_t> SA, SB;
    DB_TRY(SA.alloc((size_t)(A->nblks ? A->nblks : 1) * s * TC_SLOT));
    DB_TRY(SB.alloc((size_t)(B->nblks ? B->nblks : 1) * s * TC_SLOT));
    const int sgrid = ctx().num_sms * 16;
    if (A->nblks > 0) {
        k_tc_slice<<<(int)std::min<int64_t>(cdiv(A->nblks, 8), sgrid), 256, 0, st>>>(slice_geom(A, !ta), e, s, SA.p);
        DB_KCHECK();
    }
    if (B->nblks > 0) {
        k_tc_slice<<<(int)std::min<int64_t>(cdiv(B->nblks, 8), sgrid), 256, 0, st>>>(slice_geom(B, tb), f, s, SB.p);
        DB_KCHECK();
    }
    TcArgs a;
    a.nC = g.nC;
    a.c_row = g.c_row;
    a.c_col = g.c_col;
    a.c_off = g.c_off;
    a.c_old = g.c_old;
    a.c_pstart = g.c_pstart;
    a.prod = g.prod;
    a.rsC = g.rsC;
    a.csC = g.csC;
    a.croff = C->d_roff;
    a.ccoff = C->d_coff;
    a.e = e;
    a.f = f;
    a.SA = SA.p;
    a.SB = SB.p;
    a.Cd = g.Cd;
    a.Cold = g.Cold;
    a.Cold_off = g.Cold_off;
    a.alpha = g.alpha;
    a.beta = g.beta;
    a.err = ctx().d_flags;
    DB_CUDA(cudaMemsetAsync(a.err, 0, sizeof(int), st));
    const int grid = (int)std::min<int64_t>(g.nC, ctx().num_sms);
    int rc;
    double per = 0.0;
    timer_kernel_begin();
    switch (s) {
        case 1: rc = launch_tc<1>(a, grid); per = issued_per_product<1>(); break;
        case 2: rc = launch_tc<2>(a, grid); per = issued_per_product<2>(); break;
        case 3: rc = launch_tc<3>(a, grid); per = issued_per_product<3>(); break;
        case 4: rc = launch_tc<4>(a, grid); per = issued_per_product<4>(); break;
        case 5: rc = launch_tc<5>(a, grid); per = issued_per_product<5>(); break;
        case 6: rc = launch_tc<6>(a, grid); per = issued_per_product<6>(); break;
        case 7: rc = launch_tc<7>(a, grid); per = issued_per_product<7>(); break;
        default: rc = launch_tc<8>(a, grid); per = issued_per_product<8>(); break;
    }
    timer_kernel_end();
    if (rc) return rc;
    int h_err = 0;
    DB_CUDA(cudaMemcpyAsync(&h_err, a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    if (h_err) return fail(DBCSR_ERR_TIMEOUT, "emulated stack kernel: a tensor-core pipeline wait timed out");
    if (issued_flops) *issued_flops = per * (double)nprod;
    return DBCSR_OK;
}

}  // namespace dbcsr
