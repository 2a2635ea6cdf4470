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
// Consecutive slices therefore form one taller operand.
//
// One accumulator of M = 128 rows x N = 32 s columns per C block: lane
// quadrant q, column group u is slot (q, u). Per product, up to three operand
// segments of K = 32 (two K = 16 instructions each) accumulate into it:
//   segment 0: A slices 1, 2, 3, 4 as the quadrants x B slices 1..s
//   segment 1: A slices 0, 5, 6, 7 (0: zero slice) x B slices 0, 0, 0, 1, 2, ..
//   segment 2: A slices 0, 0, 0, 8                 x B slices 0, 0, 0, 0, 1, ..
// so slot (q, u) sums the pairs (q+1, u), (q+4, u-3) and (8, u-4) where they
// exist -- all of level q + 1 + u. Every pair t + u <= s + 1 lands in exactly
// one slot with u <= s - q, and each such slot holds one level. The slots fit
// in 256 TMEM columns, so the accumulator is double-buffered: the MMAs of the
// next chunk of products run while the previous chunk is drained. In shared
// memory A's slots are [1 2 3 4 | 0 5 6 7 | 0 0 0 8] and B's [0 0 0 (0) 1 .. s]
// (zero slices written once), so every segment's operand is one contiguous
// window. A C block's products run in chunks of 16 (10 with three segments):
// a slot then stays below 2^24 and converts to int32 exactly.
//
// Warps: 0 bulk-copy producer (one lane), 1 TMEM owner and MMA issuer (one
// lane), 2-5 drain, 6-13 finish. Every role reads its C blocks from a schedule
// in traversal order (product range, offsets, sizes in one record) and loads
// the next record ahead.
//   drain warp q (TMEM lane quadrant q = warp % 4, row i = lane): per chunk,
//     reads the slots (q, u), u = 1 .. s - q (all 32 columns), converts each
//     once to int32 and adds it into level q + 1 + u of the C block's level
//     sums in shared memory (int32 atomics: the four quadrants contribute to
//     the same levels); then releases the TMEM buffer.
//   finish warps: once a C block's level sums are complete, the 256 threads
//     take its m x n elements in column-major order (one to four each): read
//     and zero the element's level sums, hand the buffer back, recombine
//     exactly, round, scale and store -- while the drain warps fill the other
//     of the two level-sum buffers with the next C block.
// int32 level sums are exact while products * s * 32 * 127^2 < 2^31 (checked
// on the host). Every pipeline wait is bounded (TcArgs::wait_ns, 4 s unless a
// caller set another limit; the clean-up waits before exit always allow 4 s):
// on expiry the kernel sets the
// error flag, the other roles see the abort flag, every role leaves its loop
// and TMEM is freed.
#include <cuda_bf16.h>

#include "emul_common.cuh"
#include "internal.cuh"
#include "sm100_ptx.cuh"
#include "smm_emul.cuh"

namespace dbcsr {

namespace {

constexpr int TC_DRAIN = 4;                   // drain warps: one per TMEM lane quadrant
constexpr int TC_FIN = 8;                     // finish warps
constexpr int TC_THREADS = 64 + 32 * (TC_DRAIN + TC_FIN);   // producer warp, MMA warp, drain, finish
constexpr int TC_EL = 32 / TC_FIN;            // most C elements per finish thread (32 x 32 over 256 threads)
constexpr int TC_LROW = 33;                   // level-sum row stride in words: rows and columns conflict-free
constexpr int TC_SLOT = 2048;                 // one 32 x 32 bf16 slice
constexpr int TC_SMEM_CAP = 232448;           // 227 KB of shared memory per CTA
constexpr int TC_SMEM_MIN = 120 * 1024;       // one CTA per SM: it allocates all 512 TMEM columns
constexpr int TC_ACC_COLS = 256;              // TMEM columns of one accumulator buffer (two buffers)
constexpr uint64_t TC_DRAIN_NS = 4000000000ull;   // clean-up waits before the CTA exits
// C blocks are visited tile by tile: the CTAs working at the same time share
// the tile's A block rows and B block columns, which stay in L2
constexpr int TC_TILE = 32;

// Operand segments. Quadrant q of the M = 128 accumulator rows holds one A
// slice, column group u (32 columns) one B slice; every pair (t, u) that a
// level t + u <= s + 1 needs lands in a slot whose first pair has the same
// level, so each slot's fp32 sum belongs to one level:
//   segment 0: A slices 1, 2, 3, 4      x B slices u           (pairs (q+1, u))
//   segment 1: A slices -, 5, 6, 7      x B slices u - 3, u>=4 (pairs (q+4, u-3))
//   segment 2: A slices -, -, -, 8      x B slices u - 4, u>=5 (pairs (8, u-4))
// ("-": zero slice). In shared memory A's slots are [1 2 3 4 | 0 5 6 7 | 0 0 0 8]
// and B's [0 0 0 0 | 1 .. s] (zero prefix 3 for two segments), so each
// segment's operand is one contiguous window.
template <int S>
struct TcGeo {
    static constexpr int NSEG = S <= 4 ? 1 : (S <= 7 ? 2 : 3);
    static constexpr int A_SLOTS = 4 * NSEG;
    static constexpr int B_ZERO = NSEG == 1 ? 0 : (NSEG == 2 ? 3 : 4);
    static constexpr int B_SLOTS = B_ZERO + S;
    static constexpr int STAGE = (A_SLOTS + B_SLOTS) * TC_SLOT;
    static constexpr int N = 32 * S;                              // accumulator columns
    // products per exact fp32 stretch: a slot sums up to NSEG pairs of
    // CHUNK * 32 * 127^2 each, below 2^24
    static constexpr int CHUNK = NSEG <= 2 ? 16 : 10;
    static constexpr int LSBUF = S * 32 * TC_LROW;                // int32 level sums of one C block
    static constexpr int LS = 2 * LSBUF * 4;                      // two buffers, bytes
    static constexpr int RESERVE = 1024 + 256;                    // alignment + barriers
    static constexpr int NST0 = (TC_SMEM_CAP - RESERVE - LS) / STAGE;
    static constexpr int NST = NST0 > 6 ? 6 : NST0;
    static constexpr int SMEM0 = NST * STAGE + LS + RESERVE;
    static constexpr int SMEM = SMEM0 < TC_SMEM_MIN ? TC_SMEM_MIN : SMEM0;
    static constexpr uint32_t IDESC = ptx::idesc_f32acc(1, 128, N);
    // segments 1 and 2 hold needed pairs only in columns u = 4 .. S - 1 and
    // u = 5 (pairs (q+4, u-3) and (8, u-4) with t + u' <= S + 1): their MMAs
    // cover just those columns (N1, N2 at column 32 * 3 and 32 * 4) with B's
    // window starting at slice 1
    static constexpr int N1 = S >= 5 ? 32 * (S - 4) : 32;
    static constexpr int N2 = S >= 8 ? 32 * (S - 7) : 32;
    static constexpr uint32_t IDESC1 = ptx::idesc_f32acc(1, 128, N1);
    static constexpr uint32_t IDESC2 = ptx::idesc_f32acc(1, 128, N2);
    static_assert(N <= TC_ACC_COLS, "accumulator exceeds its TMEM buffer");
    static_assert(NSEG * CHUNK * 32 * 127 * 127 < (1 << 24), "fp32 stretch not exact");
    static_assert(NST >= 2, "at least two pipeline stages");
};

// One C block in traversal order: everything the three roles need, one record.
struct __align__(16) TcBlk {
    int64_t p0, p1;         // products [p0, p1)
    int64_t c_off;          // element offset of the new C block
    int64_t old_off;        // element offset of the old C block (beta != 0), -1: none
    int64_t rbase, cbase;   // first element row / column of the block
    int m, n;               // block sizes
    int64_t pad;
};
static_assert(sizeof(TcBlk) == 64, "schedule record is four 16-byte loads");

struct TcArgs {
    int64_t nC;
    const TcBlk* sched;
    const int2* prod;
    const int* e;               // exponents of C's element rows
    const int* f;               // exponents of C's element columns
    const uint8_t* SA;          // s slices (2 KB each) per stored A block
    const uint8_t* SB;
    double* Cd;
    const double* Cold;
    double alpha, beta;
    int* err;
    uint64_t wait_ns;           // limit of each pipeline wait (ns on the global timer)
};

// Slices of every stored block in the operand layout above, zero-padded to
// 32 x 32: warp per block, lane per 8-element chunk of a row; slice t in slot
// t - 1 (is_a is kept for the call sites: both operands use the same order).
__global__ void k_tc_slice(SliceGeom G, const int* __restrict__ ex, int s, int is_a, uint8_t* __restrict__ out) {
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
                const int slot = t - 1;
                *reinterpret_cast<uint4*>(o + slot * 1024 + pos) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

// traversal key of each C block: its tile, row-major over tiles
// (C blocks first .. first + n - 1 of the plan)
__global__ void k_tile_keys(int64_t n, int64_t first, const int* __restrict__ c_row, const int* __restrict__ c_col,
                            int tiles_c, uint32_t* __restrict__ key, uint32_t* __restrict__ idx) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t b = first + q;
    key[q] = (uint32_t)(c_row[b] / TC_TILE) * (uint32_t)tiles_c + (uint32_t)(c_col[b] / TC_TILE);
    idx[q] = (uint32_t)b;
}

__global__ void k_tc_sched(int64_t nC, const uint32_t* __restrict__ order, const int* __restrict__ c_row,
                           const int* __restrict__ c_col, const int64_t* __restrict__ c_pstart,
                           const int64_t* __restrict__ c_off, const int* __restrict__ c_old,
                           const int64_t* __restrict__ cold_off, const int* __restrict__ rsC,
                           const int* __restrict__ csC, const int64_t* __restrict__ croff,
                           const int64_t* __restrict__ ccoff, TcBlk* __restrict__ out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nC) return;
    const int64_t cb = order[q];
    const int br = c_row[cb], bc = c_col[cb];
    TcBlk b;
    b.p0 = c_pstart[cb];
    b.p1 = c_pstart[cb + 1];
    b.c_off = c_off[cb];
    const int old = c_old ? c_old[cb] : -1;
    b.old_off = old >= 0 ? cold_off[old] : -1;
    b.rbase = croff[br];
    b.cbase = ccoff[bc];
    b.m = rsC[br];
    b.n = csC[bc];
    b.pad = 0;
    out[q] = b;
}

// the product range of schedule entry q (a beyond-the-end q gives an empty range)
__device__ __forceinline__ longlong2 sched_range(const TcArgs& a, int64_t q) {
    if (q >= a.nC) return make_longlong2(0, 0);
    return *reinterpret_cast<const longlong2*>(a.sched + q);
}

// all lanes of the warp agree: the wait succeeded and no role aborted
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t wait_ns) {
    bool ok = !*abort_flag && ptx::mbar_wait_bounded(bar, parity, wait_ns);
    return __all_sync(0xffffffffu, ok);
}

template <int S>
__global__ void __launch_bounds__(TC_THREADS, 1) k_smm_emul_tc(TcArgs a) {
    using G = TcGeo<S>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* stages = smem;
    int* LS = reinterpret_cast<int*>(smem + G::NST * G::STAGE);   // [2][S][32][TC_LROW] level sums
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + G::NST * G::STAGE + G::LS);
    uint64_t* empty = full + G::NST;
    uint64_t* tfull = empty + G::NST;   // [2] MMA -> drain: a chunk's sums are in TMEM buffer b
    uint64_t* tempty = tfull + 2;       // [2] drain -> MMA: TMEM buffer b drained
    uint64_t* lfull = tempty + 2;       // [2] drain -> finish: a C block's level sums are complete
    uint64_t* lfree = lfull + 2;        // [2] finish -> drain: level sums read and zeroed
    uint64_t* drain = lfree + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < G::NST; i++) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; b++) {
            ptx::mbar_init(&tfull[b], 1);
            ptx::mbar_init(&tempty[b], 32 * TC_DRAIN);
            ptx::mbar_init(&lfull[b], 32 * TC_DRAIN);
            ptx::mbar_init(&lfree[b], 32 * TC_FIN);
        }
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    // zero slices of the operand windows (never written by the copies) and
    // level sums; the tensor cores read the stages through the async proxy
    for (int w = threadIdx.x; w < G::NST * G::STAGE / 16; w += blockDim.x)
        reinterpret_cast<uint4*>(stages)[w] = make_uint4(0u, 0u, 0u, 0u);
    for (int w = threadIdx.x; w < 2 * G::LSBUF; w += blockDim.x) LS[w] = 0;
    ptx::fence_proxy_async_shared();
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
            // a product's slices: A 1..4 to slots 0.., A 5..7 to slots 5.., A 8 to
            // slot 11; B 1..s to slots B_ZERO..
            int64_t it = 0;
            bool ok = true;
            longlong2 nxt = sched_range(a, blockIdx.x);
            for (int64_t seq = blockIdx.x; seq < a.nC && ok; seq += gridDim.x) {
                const longlong2 cur = nxt;
                nxt = sched_range(a, seq + gridDim.x);
                for (int64_t p = cur.x; p < cur.y; p++, it++) {
                    const int st = (int)(it % G::NST);
                    const uint32_t ph = (uint32_t)((it / G::NST) & 1);
                    const int2 pr = a.prod[p];
                    if (*abort_flag || !ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, a.wait_ns)) {
                        if (!*abort_flag) on_timeout();
                        ok = false;
                        break;
                    }
                    uint8_t* sa = stages + st * G::STAGE;
                    uint8_t* sb = sa + G::A_SLOTS * TC_SLOT;
                    const uint8_t* ga = a.SA + (int64_t)pr.x * (S * TC_SLOT);
                    ptx::mbar_arrive_expect_tx(&full[st], 2 * S * TC_SLOT);
                    ptx::bulk_load(sa, ga, (S < 4 ? S : 4) * TC_SLOT, &full[st]);
                    if constexpr (S > 4)
                        ptx::bulk_load(sa + 5 * TC_SLOT, ga + 4 * TC_SLOT, ((S < 7 ? S : 7) - 4) * TC_SLOT, &full[st]);
                    if constexpr (S > 7) ptx::bulk_load(sa + 11 * TC_SLOT, ga + 7 * TC_SLOT, TC_SLOT, &full[st]);
                    ptx::bulk_load(sb + G::B_ZERO * TC_SLOT, a.SB + (int64_t)pr.y * (S * TC_SLOT), S * TC_SLOT,
                                   &full[st]);
                }
            }
            // no copy may still be in flight when the CTA exits
            const int64_t first = it > G::NST ? it - G::NST : 0;
            for (int64_t q = first; q < it; q++)
                if (!ptx::mbar_wait_bounded(&full[q % G::NST], (uint32_t)((q / G::NST) & 1), TC_DRAIN_NS)) {
                    on_timeout();
                    break;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------ MMA issuer
            // chunk ci accumulates into TMEM buffer ci % 2 (columns 256 (ci % 2) ..)
            int64_t it = 0, ci = 0;
            bool ok = true;
            longlong2 nxt = sched_range(a, blockIdx.x);
            for (int64_t seq = blockIdx.x; seq < a.nC && ok; seq += gridDim.x) {
                const longlong2 cur = nxt;
                nxt = sched_range(a, seq + gridDim.x);
                for (int64_t c0 = cur.x; c0 < cur.y && ok; c0 += G::CHUNK, ci++) {
                    const int tb = (int)(ci & 1);
                    if (*abort_flag ||
                        !ptx::mbar_wait_bounded(&tempty[tb], (uint32_t)(((ci >> 1) & 1) ^ 1), a.wait_ns)) {
                        if (!*abort_flag) on_timeout();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(tb * TC_ACC_COLS);
                    const int64_t c1 = c0 + G::CHUNK < cur.y ? c0 + G::CHUNK : cur.y;
                    for (int64_t p = c0; p < c1; p++, it++) {
                        const int st = (int)(it % G::NST);
                        const uint32_t ph = (uint32_t)((it / G::NST) & 1);
                        if (*abort_flag || !ptx::mbar_wait_bounded(&full[st], ph, a.wait_ns)) {
                            if (!*abort_flag) on_timeout();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint8_t* sa = stages + st * G::STAGE;
                        const uint8_t* sb = sa + G::A_SLOTS * TC_SLOT;
#pragma unroll
                        for (int sg = 0; sg < G::NSEG; sg++) {
                            // segment sg >= 1 starts at accumulator column 32 * (sg + 2)
                            const uint32_t dcol = sg == 0 ? 0u : (uint32_t)(32 * (sg + 2));
                            const uint32_t idesc = sg == 0 ? G::IDESC : (sg == 1 ? G::IDESC1 : G::IDESC2);
                            const uint64_t ad = ptx::smem_desc_kmajor(sa + 4 * sg * TC_SLOT, 128, 512);
                            const uint64_t bd = ptx::smem_desc_kmajor(sb + G::B_ZERO * TC_SLOT, 128, 512);
#pragma unroll
                            for (int ks = 0; ks < 2; ks++) {
                                // the second K = 16 step starts two core matrices (256 bytes) further;
                                // segment 0 of a chunk's first product initialises every column
                                const uint32_t acc = (p > c0 || sg > 0 || ks > 0) ? 1u : 0u;
                                ptx::mma_f16_ss(d + dcol, ad + (uint64_t)(ks * 16), bd + (uint64_t)(ks * 16), idesc,
                                                acc);
                            }
                        }
                        ptx::mma_commit(&empty[st]);
                    }
                    if (ok) ptx::mma_commit(&tfull[tb]);
                }
            }
            ptx::mma_commit(drain);
            if (!ptx::mbar_wait_bounded(drain, 0, TC_DRAIN_NS)) on_timeout();
        }
    } else if (warp < 2 + TC_DRAIN) {
        // ------------------------------------------------------------- drain
        // warp q (TMEM lane quadrant q = warp % 4, row i = lane): per chunk, the
        // slots (q, u) for u = 1 .. s - q hold level q + 1 + u (every other slot
        // is beyond level s + 1); each is read, converted once to int32 (exact:
        // an integer below 2^24) and added into the C block's level sums in
        // shared memory (the quadrants meet there: shared-memory atomics); then
        // the TMEM buffer is released for the chunk after next.
        const int q = warp & 3;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        int64_t ci = 0, cbi = 0;
        bool ok = true;
        for (int64_t seq = blockIdx.x; seq < a.nC && ok; seq += gridDim.x, cbi++) {
            const longlong2 cur = sched_range(a, seq);
            const int buf = (int)(cbi & 1);
            if (!warp_wait(&lfree[buf], (uint32_t)(((cbi >> 1) & 1) ^ 1), abort_flag, a.wait_ns)) {
                if (!*abort_flag) on_timeout();
                ok = false;
                break;
            }
            int* ls = LS + buf * G::LSBUF + lane * TC_LROW;   // level 0, row lane
            for (int64_t c0 = cur.x; c0 < cur.y; c0 += G::CHUNK, ci++) {
                const int tb = (int)(ci & 1);
                if (!warp_wait(&tfull[tb], (uint32_t)((ci >> 1) & 1), abort_flag, a.wait_ns)) {
                    if (!*abort_flag) on_timeout();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                for (int u = 1; u <= S - q; u++) {
                    uint32_t x[32];
                    ptx::tmem_ld_32x32b_x32(tl + (uint32_t)(tb * TC_ACC_COLS + (u - 1) * 32), x);
                    ptx::tmem_wait_ld();
                    int* row = ls + (q + u - 1) * 32 * TC_LROW;   // level q + 1 + u, index from level 2
#pragma unroll
                    for (int c = 0; c < 32; c++) atomicAdd(row + c, __float2int_rn(__uint_as_float(x[c])));
                }
                ptx::tc_fence_before();
                ptx::mbar_arrive(&tempty[tb]);
            }
            if (!ok) break;
            ptx::mbar_arrive(&lfull[buf]);   // this C block's level sums are complete
        }
    } else {
        // ------------------------------------------------------------ finish
        // finish thread ft takes the C block's elements e = ft, ft + 256, ..
        // below m n (column-major: row e % m, column e / m, so consecutive
        // threads store consecutive addresses and a small block keeps few
        // threads busy for little time): it reads and zeroes the element's level
        // sums, hands the buffer back, recombines exactly, rounds once, applies
        // alpha / beta and stores -- while the drain warps accumulate the next
        // C block. Level sums outside m x n are never written (zero padding).
        const int ft = (warp - 2 - TC_DRAIN) * 32 + lane;
        constexpr int NFT = 32 * TC_FIN;
        const BlasUpd bu(a.alpha, a.beta);
        int64_t cbi = 0;
        bool ok = true;
        TcBlk nxt;
        if (blockIdx.x < a.nC) nxt = a.sched[blockIdx.x];
        for (int64_t seq = blockIdx.x; seq < a.nC && ok; seq += gridDim.x, cbi++) {
            const TcBlk cur = nxt;
            if (seq + gridDim.x < a.nC) nxt = a.sched[seq + gridDim.x];
            const int mn = cur.m * cur.n;
            // what the recombination needs, loaded before the wait
            int ri[TC_EL], cj[TC_EL], ex[TC_EL];
            double oldv[TC_EL];
#pragma unroll
            for (int k = 0; k < TC_EL; k++) {
                const int e = ft + NFT * k;
                const bool in = e < mn;
                ri[k] = in ? e % cur.m : 0;
                cj[k] = in ? e / cur.m : 0;
                ex[k] = in ? a.e[cur.rbase + ri[k]] + a.f[cur.cbase + cj[k]] : 0;
                oldv[k] = (in && cur.old_off >= 0) ? a.Cold[cur.old_off + e] : 0.0;
            }
            const int buf = (int)(cbi & 1);
            if (!warp_wait(&lfull[buf], (uint32_t)((cbi >> 1) & 1), abort_flag, a.wait_ns)) {
                if (!*abort_flag) on_timeout();
                ok = false;
                break;
            }
            int lv[S][TC_EL];
            int* lsb = LS + buf * G::LSBUF;
#pragma unroll
            for (int k = 0; k < TC_EL; k++) {
                int* ls = lsb + ri[k] * TC_LROW + cj[k];
                const bool in = ft + NFT * k < mn;
#pragma unroll
                for (int d = 0; d < S; d++) {
                    lv[d][k] = in ? ls[d * 32 * TC_LROW] : 0;
                    if (in) ls[d * 32 * TC_LROW] = 0;
                }
            }
            ptx::mbar_arrive(&lfree[buf]);
            // exact recombination, one rounding, alpha / beta, column-major C block.
            // sum_d G_d 2^(7(s-1-d)) (d from 0) = U 2^(7 (s - NU)) + V with U over the
            // first NU = min(4, s) levels and V over the rest: |U|, |V| < 2^53, so
            // both run in int64 and one 128-bit shift and add joins them.
            constexpr int NU = S < 4 ? S : 4;
            double* cout = a.Cd + cur.c_off;
#pragma unroll
            for (int k = 0; k < TC_EL; k++) {
                const int e = ft + NFT * k;
                if (e >= mn) break;
                long long U = 0, V = 0;
#pragma unroll
                for (int d = 0; d < NU; d++) U = U * 128 + lv[d][k];
#pragma unroll
                for (int d = NU; d < S; d++) V = V * 128 + lv[d][k];
                const __int128 Sx = (__int128)U * ((__int128)1 << (7 * (S - NU))) + V;
                const double x = emul::recombined(Sx, ex[k], 7 * (S + 1));
                cout[e] = cur.old_off >= 0 ? bu.update(x, oldv[k]) : bu.scale(x);
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
    const double cols = (double)G::N + (G::NSEG > 1 ? (double)G::N1 : 0.0) + (G::NSEG > 2 ? (double)G::N2 : 0.0);
    return 2.0 * 128.0 * cols * 32.0;
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
                const int* e, const int* f, int s, int64_t nprod, double* issued_flops, const CRanges* ranges) {
    cudaStream_t st = ctx().stream;
    DBuf<uint8_t> SA, SB;
    DB_TRY(SA.alloc((size_t)(A->nblks ? A->nblks : 1) * s * TC_SLOT));
    DB_TRY(SB.alloc((size_t)(B->nblks ? B->nblks : 1) * s * TC_SLOT));
    const int sgrid = ctx().num_sms * 16;
    if (A->nblks > 0) {
        k_tc_slice<<<(int)std::min<int64_t>(cdiv(A->nblks, 8), sgrid), 256, 0, st>>>(slice_geom(A, !ta), e, s, 1, SA.p);
        DB_KCHECK();
    }
    if (B->nblks > 0) {
        k_tc_slice<<<(int)std::min<int64_t>(cdiv(B->nblks, 8), sgrid), 256, 0, st>>>(slice_geom(B, tb), f, s, 0, SB.p);
        DB_KCHECK();
    }
    // the C blocks to compute (all, or the given ranges), in tile order
    // (stable: row-major within a tile, as the C blocks are stored)
    if (g.nC >= (int64_t)UINT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "emulated stack kernel: too many C blocks");
    const CRanges all{{0, g.nC}};
    const CRanges& rr = ranges ? *ranges : all;
    int64_t nsel = 0;
    for (const auto& r : rr) nsel += std::max<int64_t>(0, r.second - r.first);
    if (nsel == 0) return DBCSR_OK;
    DBuf<uint32_t> key, order;
    DB_TRY(key.alloc(nsel));
    DB_TRY(order.alloc(nsel));
    const int tiles_r = (int)cdiv(C->nbr, TC_TILE), tiles_c = (int)cdiv(C->nbc, TC_TILE);
    int64_t at = 0;
    for (const auto& r : rr) {
        const int64_t n = r.second - r.first;
        if (n <= 0) continue;
        k_tile_keys<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, r.first, g.c_row, g.c_col, tiles_c, key.p + at,
                                                            order.p + at);
        DB_KCHECK();
        at += n;
    }
    int bits = 0;
    while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)tiles_r * tiles_c) bits++;
    DB_TRY(radix_sort_u32(key.p, order.p, nsel, bits));
    DBuf<TcBlk> sched;
    DB_TRY(sched.alloc(nsel));
    k_tc_sched<<<(unsigned)cdiv(nsel, 256), 256, 0, st>>>(nsel, order.p, g.c_row, g.c_col, g.c_pstart, g.c_off,
                                                          g.c_old, g.Cold_off, g.rsC, g.csC, C->d_roff, C->d_coff,
                                                          sched.p);
    DB_KCHECK();
    TcArgs a;
    a.nC = nsel;
    a.sched = sched.p;
    a.prod = g.prod;
    a.e = e;
    a.f = f;
    a.SA = SA.p;
    a.SB = SB.p;
    a.Cd = g.Cd;
    a.Cold = g.Cold;
    a.alpha = g.alpha;
    a.beta = g.beta;
    a.err = ctx().d_flags;
    a.wait_ns = ctx().wait_ns;
    DB_CUDA(cudaMemsetAsync(a.err, 0, sizeof(int), st));
    const int grid = (int)std::min<int64_t>(nsel, ctx().num_sms);
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
