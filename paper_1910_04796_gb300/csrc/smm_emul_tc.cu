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
//   G2: rows A slices s, s-1, .., 5 (M = 128, padded) x columns B slices
//       1..s-4 (N = 32 (s-4)); A's slices are stored in the order
//       1, 2, 3, 4, s, s-1, .., 5 so that G2 is one operand and every lane
//       quadrant q holds the slices q + 1 and s - q, which balances the
//       epilogue's work over the quadrants
// so pair (t, u) owns a 32 x 32 accumulator block of TMEM (lane quadrant
// t - 1 or s - t, columns 32 (u-1), + 32 s for G2); pairs with t + u > s + 1
// are computed and ignored. A C block's products run in chunks of 16: an fp32
// accumulator then stays below 2^23 (16 * 32 * 127^2), so the G1 and G2 sums
// of a level are added exactly in fp32 before one conversion to int32.
//
// Warps: 0 bulk-copy producer (one lane), 1 TMEM owner and MMA issuer (one
// lane), 2-9 epilogue; epilogue warp w reads TMEM lane quadrant q = w % 4,
// i.e. A slice t = q + 1 of G1 and t = s - q of G2, two warps per quadrant
// splitting the columns. Every role reads its C blocks from a schedule in
// traversal order (product range, offsets, sizes in one record) and loads
// the next record ahead. Per chunk the epilogue
//   1. drains TMEM: level d's contribution of its slices, P_{t,d-t} (+ the
//      G2 term), converted exactly to int32, into a level block in shared
//      memory; then releases TMEM, so the next chunk's MMAs overlap the rest;
//   2. sums the level blocks of the four quadrants into per-thread int32
//      level sums (thread: row i = lane, four columns).
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

constexpr int TC_R = 2;                       // epilogue warps per TMEM lane quadrant
constexpr int TC_EPI = 4 * TC_R;              // epilogue warps
constexpr int TC_THREADS = 64 + 32 * TC_EPI;  // producer warp, MMA warp, epilogue
constexpr int TC_COLS = 32 / TC_R;            // accumulator columns an epilogue warp drains per block
constexpr int TC_EL = 8 / TC_R;               // C elements per epilogue thread
constexpr int TC_SLOT = 2048;                 // one 32 x 32 bf16 slice
constexpr int TC_SMEM_CAP = 232448;           // 227 KB of shared memory per CTA
constexpr int TC_SMEM_MIN = 120 * 1024;       // one CTA per SM: it allocates all 512 TMEM columns
constexpr int TC_CHUNK = 16;                  // products per exact fp32 stretch (16 * 32 * 127^2 < 2^23)
constexpr uint64_t TC_WAIT_NS = 4000000000ull;
// C blocks are visited tile by tile: the CTAs working at the same time share
// the tile's A block rows and B block columns, which stay in L2
constexpr int TC_TILE = 32;

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
};

// Slices of every stored block in the operand layout above, zero-padded to
// 32 x 32: warp per block, lane per 8-element chunk of a row.
// A (is_a) stores slice t in slot t - 1 for t <= 4 and 4 + s - t above; B in slot t - 1.
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
                const int slot = (is_a && t > 4) ? 4 + s - t : t - 1;
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
        ptx::mbar_init(tempty, 32 * TC_EPI);
        ptx::mbar_init(sfull, 32 * TC_EPI);
        ptx::mbar_init(sfree, 32 * TC_EPI);
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
            longlong2 nxt = sched_range(a, blockIdx.x);
            for (int64_t seq = blockIdx.x; seq < a.nC && ok; seq += gridDim.x) {
                const longlong2 cur = nxt;
                nxt = sched_range(a, seq + gridDim.x);
                for (int64_t p = cur.x; p < cur.y; p++, it++) {
                    const int st = (int)(it % G::NST);
                    const uint32_t ph = (uint32_t)((it / G::NST) & 1);
                    const int2 pr = a.prod[p];
                    if (*abort_flag || !ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, TC_WAIT_NS)) {
                        if (!*abort_flag) on_timeout();
                        ok = false;
                        break;
                    }
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
            longlong2 nxt = sched_range(a, blockIdx.x);
            for (int64_t seq = blockIdx.x; seq < a.nC && ok; seq += gridDim.x) {
                const longlong2 cur = nxt;
                nxt = sched_range(a, seq + gridDim.x);
                for (int64_t c0 = cur.x; c0 < cur.y && ok; c0 += TC_CHUNK, ci++) {
                    if (*abort_flag || !ptx::mbar_wait_bounded(tempty, (uint32_t)((ci & 1) ^ 1), TC_WAIT_NS)) {
                        if (!*abort_flag) on_timeout();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int64_t c1 = c0 + TC_CHUNK < cur.y ? c0 + TC_CHUNK : cur.y;
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
        // warp (q, r): TMEM lane quadrant q = warp % 4, columns 16 r .. 16 r + 15
        // of every 32-column accumulator block; in the sum and the final
        // stage thread (warp (q, r), lane) owns row i = lane, columns 4 ep .. 4 ep + 3
        const int q = warp & 3, r = (warp - 2) >> 2, ep = q * TC_R + r;
        const BlasUpd bu(a.alpha, a.beta);
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(r * TC_COLS);
        const int t1 = q + 1, t2 = S - q;                 // A slices of quadrant q in G1 and G2
        const bool has2 = (G::N2 > 0) && (t2 >= 5);
        const int sw = lane & 7;   // 16-byte chunks XOR-swizzled by row: conflict-free stores and loads
        const int i = lane;
        int64_t ci = 0;
        bool ok = true;
        TcBlk nxt;
        if (blockIdx.x < a.nC) nxt = a.sched[blockIdx.x];
        for (int64_t seq = blockIdx.x; seq < a.nC && ok; seq += gridDim.x) {
            const TcBlk cur = nxt;
            if (seq + gridDim.x < a.nC) nxt = a.sched[seq + gridDim.x];
            // what the final stage needs, loaded now: its latency hides behind the MMAs
            const bool row_ok = i < cur.m;
            const int ei = row_ok ? a.e[cur.rbase + i] : 0;
            int fj[TC_EL];
            double oldv[TC_EL];
#pragma unroll
            for (int k = 0; k < TC_EL; k++) {
                const int j = TC_EL * ep + k;
                fj[k] = j < cur.n ? a.f[cur.cbase + j] : 0;
                oldv[k] = (row_ok && j < cur.n && cur.old_off >= 0) ? a.Cold[cur.old_off + (int64_t)j * cur.m + i] : 0.0;
            }
            int lv[S][TC_EL];
#pragma unroll
            for (int d = 0; d < S; d++)
#pragma unroll
                for (int k = 0; k < TC_EL; k++) lv[d][k] = 0;
            for (int64_t c0 = cur.p0; c0 < cur.p1; c0 += TC_CHUNK, ci++) {
                const uint32_t ph = (uint32_t)(ci & 1);
                if (!warp_wait(tfull, ph, abort_flag) || !warp_wait(sfree, ph ^ 1u, abort_flag)) {
                    if (!*abort_flag) on_timeout();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                // 1. drain, two levels per TMEM round trip: level d of slice t1
                //    (G1, u = d - t1) plus slice t2 (G2, u = d - t2) where it exists;
                //    exact fp32 integers -> int32 level blocks
                if (t1 <= S) {
                    for (int d0 = t1 + 1; d0 <= S + 1; d0 += 2) {
                        const int d1 = d0 + 1;
                        const bool h1 = d1 <= S + 1;
                        const bool g0 = has2 && d0 - t2 >= 1, g1 = has2 && h1 && d1 - t2 >= 1;
                        uint32_t ra[TC_COLS], rb[TC_COLS], rc[TC_COLS], rd[TC_COLS];
                        ptx::tmem_ld_32x32b_x16(tl + (uint32_t)((d0 - t1 - 1) * 32), ra);
                        if (h1) ptx::tmem_ld_32x32b_x16(tl + (uint32_t)((d1 - t1 - 1) * 32), rb);
                        if (g0) ptx::tmem_ld_32x32b_x16(tl + (uint32_t)(G::N1 + (d0 - t2 - 1) * 32), rc);
                        if (g1) ptx::tmem_ld_32x32b_x16(tl + (uint32_t)(G::N1 + (d1 - t2 - 1) * 32), rd);
                        ptx::tmem_wait_ld();
                        uint8_t* row0 = stg + lvl_blk<S>(q, d0) * 4096 + lane * 128;
                        uint8_t* row1 = stg + lvl_blk<S>(q, h1 ? d1 : d0) * 4096 + lane * 128;
#pragma unroll
                        for (int c = 0; c < TC_COLS / 4; c++) {
                            int v0[4], v1[4];
#pragma unroll
                            for (int k = 0; k < 4; k++) {
                                // both pair sums are integers below 2^23: their fp32 sum is exact
                                float x0 = __uint_as_float(ra[c * 4 + k]);
                                if (g0) x0 += __uint_as_float(rc[c * 4 + k]);
                                float x1 = __uint_as_float(rb[c * 4 + k]);
                                if (g1) x1 += __uint_as_float(rd[c * 4 + k]);
                                v0[k] = __float2int_rn(x0);
                                v1[k] = __float2int_rn(x1);
                            }
                            const int off = ((r * (TC_COLS / 4) + c) ^ sw) << 4;
                            *reinterpret_cast<int4*>(row0 + off) = make_int4(v0[0], v0[1], v0[2], v0[3]);
                            if (h1) *reinterpret_cast<int4*>(row1 + off) = make_int4(v1[0], v1[1], v1[2], v1[3]);
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
                // 2. level sums of this thread's four elements
#pragma unroll
                for (int d = 2; d <= S + 1; d++)
#pragma unroll
                    for (int w = 0; w < G::T1; w++)
                        if (w + 2 <= d) {
                            const int4 x = *reinterpret_cast<const int4*>(stg + lvl_blk<S>(w, d) * 4096 + lane * 128 +
                                                                          ((ep ^ sw) << 4));
                            lv[d - 2][0] += x.x;
                            lv[d - 2][1] += x.y;
                            lv[d - 2][2] += x.z;
                            lv[d - 2][3] += x.w;
                        }
                ptx::mbar_arrive(sfree);
            }
            if (!ok) break;
            // 3. exact recombination, one rounding, alpha / beta, column-major C block.
            // sum_d G_d 2^(7(s-1-d)) (d from 0) = U 2^(7 (s - NU)) + V with U over the
            // first NU = min(4, s) levels and V over the rest: |U|, |V| < 2^53, so
            // both run in int64 and one 128-bit shift and add joins them.
            constexpr int NU = S < 4 ? S : 4;
            // the four elements are computed unconditionally (independent chains
            // the scheduler can interleave); only the stores are guarded
            double res[TC_EL];
#pragma unroll
            for (int k = 0; k < TC_EL; k++) {
                long long U = 0, V = 0;
#pragma unroll
                for (int d = 0; d < NU; d++) U = U * 128 + lv[d][k];
#pragma unroll
                for (int d = NU; d < S; d++) V = V * 128 + lv[d][k];
                const __int128 Sx = (__int128)U * ((__int128)1 << (7 * (S - NU))) + V;
                const double x = emul::round_i128_scaled(Sx, ei + fj[k] - 7 * (S + 1));
                res[k] = cur.old_off >= 0 ? bu.update(x, oldv[k]) : bu.scale(x);
            }
            if (row_ok) {
                double* cout = a.Cd + cur.c_off;
#pragma unroll
                for (int k = 0; k < TC_EL; k++) {
                    const int j = TC_EL * ep + k;
                    if (j < cur.n) cout[(int64_t)j * cur.m + i] = res[k];
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
