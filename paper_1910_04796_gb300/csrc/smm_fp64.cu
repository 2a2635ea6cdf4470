// smm_fp64.cu -- batched FP64 small-matrix products over the stack list.
//
// Paper, Sec. II: batches of block products C_ij += A_ik B_kj are executed by
// LIBCUSMM, CUDA kernels for small (m,n,k) auto-tuned over read/write strategy,
// threads per block, elements per thread and tiling. This file holds the
// GB300 kernels that play that role for FP64, and the per-shape dispatch that
// the autotuner's table drives.
//
// GB300 facts that shape them: the FP64 pipe does two FMAs per clock per SM
// (1.26 TFLOP/s at 2 070 MHz; the FP64 MMA is no faster), so a block product
// is arithmetic-bound once its operands are on chip (the ridge point is ~0.2
// flop/byte against 6.7 TB/s HBM). What matters is (1) keeping every lane of
// every DFMA busy (elements mapped densely onto lanes) -- and issuing no DFMA
// for idle lanes: one under a false predicate still takes its pipe cycles --
// (2) enough independent accumulators and resident warps to cover latency,
// (3) never waiting on a chain of dependent index loads per product, and
// operands in L1 before they are used, (4) reading each C block once and
// writing it once.
//
// A team of W warps owns one C block: it walks the block's products (ascending
// k, as stack generation ordered them; with W > 1 warp w takes products w,
// w+W, ... and the partial sums are added in warp order through shared
// memory), keeps the C block in registers, and writes alpha*acc + beta*C_old
// once -- no atomics on C. Each warp fetches the index data of 32 of its
// products at once (one lane per product) and broadcasts it with shuffles.
// All C blocks of a multiply run in one persistent launch: an instance with
// up to 16 elements per lane (at most 128 registers: two 256-thread CTAs, 16
// warps per SM), larger blocks in several passes of 16 per lane; work is
// handed out by atomic counters.
#include <vector>

#include "internal.cuh"
#include "smm.cuh"

namespace dbcsr {

namespace {

// Variants (the autotuner's search space): warps per C block.
//   0: 1 warp     1: 1 warp (runs as 0: the single launch has 256-thread
//                    CTAs; the number stays so that tuning tables keep their meaning)
//   2: 2-warp teams     3: 4-warp teams
constexpr int kTeamWarps[SMM_NUM_VARIANTS] = {1, 1, 2, 4};

__host__ __device__ inline int q_class(int mn) {
    const int q = (mn + 31) / 32;
    return q <= 1 ? 0 : q <= 2 ? 1 : q <= 4 ? 2 : q <= 8 ? 3 : q <= 16 ? 4 : 5;
}

// barrier of one team of W warps (named barrier team+1; teams work on different
// C blocks, so a CTA-wide barrier would couple them)
template <int W>
__device__ __forceinline__ void team_sync(int team) {
    if (W == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(W * 32) : "memory");
    }
}

// brings n elements from p into L1 ahead of their use: one 128-byte line per
// lane, every address inside the block (a C block has few products, so most
// operand blocks would otherwise arrive from L2 while the FP64 pipe waits)
template <typename T>
__device__ __forceinline__ void prefetch_block(const T* p, int n, int lane) {
    const char* b = reinterpret_cast<const char*>(p);
    const int bytes = n * (int)sizeof(T);
    for (int o = lane * 128; o < bytes; o += 32 * 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(b + o));
    if (lane == 31 && bytes > 0) asm volatile("prefetch.global.L1 [%0];" ::"l"(b + bytes - 1));
}

// one team per C block; each lane holds up to Q elements e = lane + 32*q,
// r = e % m, c = e / m (column-major order within the block). T is the
// arithmetic type: double (FP64 path) or float (FP32 path: operands read from
// FP32 copies of A and B, FP32 FMA sums, alpha/beta applied in FP64).
template <typename T, int Q, int TA, int TB, int W>
__device__ __forceinline__ void smm_body(const SmmArgs& g, const T* __restrict__ adata, const T* __restrict__ bdata,
                                         const uint32_t* __restrict__ list, int64_t nlist, int chunk,
                                         double* s_red, unsigned long long* counter) {
    constexpr int QG = Q < 2 ? Q : 2;                 // elements per inner-loop group
    const BlasUpd bu(g.alpha, g.beta);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int team = warp / W, tw = warp % W;        // team in CTA, warp in team
    __shared__ int s_cb[8];
    for (;;) {
        // a team takes 32 consecutive C blocks at a time; lane t fetches block
        // t's index data in parallel, then the blocks are processed in order
        if (tw == 0 && lane == 0) s_cb[team] = (int)atomicAdd(counter, (unsigned long long)chunk);
        team_sync<W>(team);
        const int64_t lbase = s_cb[team];
        team_sync<W>(team);
        if (lbase >= nlist) break;
        const int nbat = (int)min((int64_t)chunk, nlist - lbase);
        int my_m = 1, my_n = 1;
        long long my_p0 = 0, my_p1 = 0, my_coff = 0, my_old = -1;
        long long my_fa = -1, my_fb = 0;   // operands of this warp's first product of the block
        int my_fk = 0;
        if (lane < nbat) {
            const int64_t cbl = list ? (int64_t)list[lbase + lane] : lbase + lane;
            my_m = g.rsC[g.c_row[cbl]];
            my_n = g.csC[g.c_col[cbl]];
            my_p0 = g.c_pstart[cbl];
            my_p1 = g.c_pstart[cbl + 1];
            my_coff = g.c_off[cbl];
            const int o = g.c_old ? g.c_old[cbl] : -1;
            my_old = (o >= 0) ? (long long)g.Cold_off[o] : -1;
            if (my_p0 + tw < my_p1) {
                const int2 pr = g.prod[my_p0 + tw];
                my_fa = g.A.off[pr.x];
                my_fk = (int)(g.A.off[pr.x + 1] - my_fa) / my_m;
                my_fb = g.B.off[pr.y];
            }
        }
        for (int bt = 0; bt < nbat; bt++) {
        // first product of the next C block (and of this one at the start of a batch) into L1
        for (int x = bt == 0 ? 0 : bt + 1; x <= bt + 1 && x < nbat; x++) {
            const long long fa = __shfl_sync(0xffffffffu, my_fa, x), fb = __shfl_sync(0xffffffffu, my_fb, x);
            const int fk = __shfl_sync(0xffffffffu, my_fk, x);
            const int fm = __shfl_sync(0xffffffffu, my_m, x), fn = __shfl_sync(0xffffffffu, my_n, x);
            if (fa >= 0) {
                prefetch_block(adata + fa, fm * fk, lane);
                prefetch_block(bdata + fb, fk * fn, lane);
            }
        }
        const int m = __shfl_sync(0xffffffffu, my_m, bt), n = __shfl_sync(0xffffffffu, my_n, bt);
        const int mn = m * n;
        const int64_t p0 = __shfl_sync(0xffffffffu, my_p0, bt), p1 = __shfl_sync(0xffffffffu, my_p1, bt);
        double* cout = g.Cd + __shfl_sync(0xffffffffu, my_coff, bt);
        const long long old_off = __shfl_sync(0xffffffffu, my_old, bt);
        const double* cold = (old_off >= 0) ? g.Cold + old_off : nullptr;
        for (int e0 = 0; e0 < mn; e0 += 32 * Q) {
            const int nq = min(Q, (mn - e0 + 31) >> 5);
            T acc[Q];
            int ro[Q], co[Q];
#pragma unroll
            for (int q = 0; q < Q; q++) {
                acc[q] = T(0);
                int e = e0 + lane + 32 * q;
                if (e >= mn) e = 0;
                ro[q] = e % m;
                co[q] = e / m;
            }
            // this warp's products p0 + tw + W*t, 32 at a time: lane t fetches
            // product t's operand offsets and inner size, then they are broadcast
            for (int64_t pb = p0 + tw; pb < p1; pb += (int64_t)32 * W) {
                const int64_t pj = pb + (int64_t)lane * W;
                long long my_ao = 0, my_bo = 0;
                int my_kk = 0;
                if (pj < p1) {
                    const int2 pr = g.prod[pj];
                    my_ao = g.A.off[pr.x];
                    my_kk = (int)(g.A.off[pr.x + 1] - my_ao) / m;   // block sizes < 2^31: 32-bit division
                    my_bo = g.B.off[pr.y];
                }
                const int nb = (int)min((int64_t)32, (p1 - pb + W - 1) / W);
                for (int t = 0; t < nb; t++) {
                    const long long ao = __shfl_sync(0xffffffffu, my_ao, t);
                    const long long bo = __shfl_sync(0xffffffffu, my_bo, t);
                    const int kk = __shfl_sync(0xffffffffu, my_kk, t);
                    if (t + 1 < nb) {   // the next product's blocks into L1
                        const long long an = __shfl_sync(0xffffffffu, my_ao, t + 1);
                        const long long bn = __shfl_sync(0xffffffffu, my_bo, t + 1);
                        const int kn = __shfl_sync(0xffffffffu, my_kk, t + 1);
                        prefetch_block(adata + an, m * kn, lane);
                        prefetch_block(bdata + bn, kn * n, lane);
                    }
                    const T* __restrict__ a = adata + ao;
                    const T* __restrict__ b = bdata + bo;
                    const int astep = TA ? 1 : m;
                    const int bstep = TB ? n : 1;
                    // the lane's elements in groups of QG, each group a loop over l
                    // of its own: groups past nq are skipped by a (uniform) branch,
                    // so at most QG - 1 FMAs per step are issued for nothing.
                    // Every accumulator still sums l = 0 .. kk-1 in order.
#pragma unroll
                    for (int q0 = 0; q0 < Q; q0 += QG) {
                        if (q0 < nq) {
                            int aidx[QG], bidx[QG];
#pragma unroll
                            for (int j = 0; j < QG; j++) {
                                aidx[j] = TA ? ro[q0 + j] * kk : ro[q0 + j];
                                bidx[j] = TB ? co[q0 + j] : co[q0 + j] * kk;
                            }
                            for (int l = 0; l < kk; l++) {
#pragma unroll
                                for (int j = 0; j < QG; j++) {
                                    if (q0 + j < nq)
                                        acc[q0 + j] = fma(__ldg(a + aidx[j]), __ldg(b + bidx[j]), acc[q0 + j]);
                                    aidx[j] += astep;
                                    bidx[j] += bstep;
                                }
                            }
                        }
                    }
                }
            }
            if (W > 1) {
                // partial sums of warps 1..W-1 to shared memory, added in warp order by warp 0
                T* red = reinterpret_cast<T*>(s_red) + (size_t)team * (W - 1) * Q * 32;
                if (tw > 0) {
#pragma unroll
                    for (int q = 0; q < Q; q++) red[((tw - 1) * Q + q) * 32 + lane] = acc[q];
                }
                team_sync<W>(team);
                if (tw == 0) {
                    for (int w = 1; w < W; w++)
#pragma unroll
                        for (int q = 0; q < Q; q++) acc[q] += red[((w - 1) * Q + q) * 32 + lane];
                }
                team_sync<W>(team);
            }
            if (tw == 0) {
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    const int e = e0 + lane + 32 * q;
                    if (q < nq && e < mn) {
                        cout[e] = cold ? bu.update((double)acc[q], cold[e]) : bu.scale((double)acc[q]);
                    }
                }
            }
        }
        }   // blocks of the batch
    }
}

// Every C block of a multiply in one launch. The blocks come in up to three
// groups by team size (1, 2 or 4 warps per C block, from the tuning table),
// stored one after the other in `list` (nullptr: one group of team size 1 over
// blocks 0 .. n_all-1). A CTA works through the groups in order: its teams
// take chunks of the current group from that group's counter until it is
// exhausted, then the CTA re-forms its teams for the next group. The group
// sizes are read on the device, so the launch needs nothing from the host.
struct SmmGroups {
    const int* counts;            // C blocks per team size 1, 2, 4 (nullptr: see n_all)
    int64_t n_all;
    unsigned long long* ctr;      // one zeroed counter per group
    int64_t stride;               // group k's C blocks at list + k * stride
};

template <int Q, int TA, int TB>
__global__ void __launch_bounds__(256, Q <= 16 ? 2 : 1)
    k_smm_fp64_all(SmmArgs g, const uint32_t* __restrict__ list, SmmGroups gr) {
    extern __shared__ double s_red[];                 // [teams][W-1][Q][32] partial sums, W <= 4
#pragma unroll 1
    for (int k = 0; k < 3; k++) {
        const int64_t cnt = gr.counts ? (int64_t)gr.counts[k] : (k == 0 ? gr.n_all : 0);
        if (cnt > 0) {
            const int64_t teams = (int64_t)gridDim.x * (8 >> k);
            // C blocks per grab: up to 32, at least ~8 grabs per team
            const int chunk = (int)max((int64_t)1, min((int64_t)32, cnt / (teams * 8)));
            const uint32_t* l = list ? list + k * gr.stride : nullptr;
            if (k == 0) smm_body<double, Q, TA, TB, 1>(g, g.A.data, g.B.data, l, cnt, chunk, s_red, gr.ctr);
            else if (k == 1) smm_body<double, Q, TA, TB, 2>(g, g.A.data, g.B.data, l, cnt, chunk, s_red, gr.ctr + 1);
            else smm_body<double, Q, TA, TB, 4>(g, g.A.data, g.B.data, l, cnt, chunk, s_red, gr.ctr + 2);
            __syncthreads();   // every team done with this group's barriers and partial sums
        }
    }
}

// FP32 stack kernel: one warp per C block
template <int Q, int TA, int TB>
__global__ void __launch_bounds__(256, Q <= 16 ? 2 : 1) k_smm_fp32(SmmArgs g, const uint32_t* __restrict__ list, int64_t nlist,
                                                        int chunk) {
    smm_body<float, Q, TA, TB, 1>(g, g.A32, g.B32, list, nlist, chunk, nullptr, g.counter);
}

// FP32 stack kernel for blocks up to 32 x 32. A warp takes a chunk of up to
// 32 consecutive C blocks of the (class-sorted) order; lane q loads C block
// q's metadata (sizes, product range, C offsets), so the chunk pays one chain
// of dependent global loads instead of one per C block. The chunk is split into
// runs of one patch class, and each run is a single stream of products: the
// warp stages products NS - 1 ahead across C-block boundaries, computes them
// in order and writes each C block when its last product is done. Staging:
// op(A) and op(B) blocks go to the warp's shared memory (A(i, l) at l * SA + i,
// B(l, j) at l * SB + j, SA and SB the padded row and column counts (8, 16 or
// 32) plus 4: rows 16-byte aligned; cp.async, 4 bytes each, see f32_stage).
// Compute: each lane an R x CC patch of the C block in registers; per inner
// index l it loads R values of A's column l and CC values of B's row l (vector
// loads) and issues R * CC FMAs. FMA order per element: products in plan
// order, l ascending. The products' operand offsets and inner sizes are read 32
// stream positions at a time, one per lane. Patch rows from m and columns from
// n read whatever the staging buffer holds there and feed accumulators that are
// never stored.
constexpr int F32_WARPS = 4;
constexpr int F32_WARP_FLOATS = 2 * 2 * 32 * 36;   // two stages of 32 x 32 blocks (A and B, rows of 36)
constexpr int F32_SMEM = F32_WARPS * F32_WARP_FLOATS * (int)sizeof(float);
constexpr int F32_MAX_STAGES = 6;

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

// the copies of one product's op(A) (m x kk) and op(B) (kk x n) blocks into a
// staging buffer (row strides SA, SB). Where a stored block's contiguous
// dimension has at least 16 elements, lane x copies line x of it (one copy per
// element of the other dimension); below that, lane e copies elements e,
// e + 32, ... of the block, so that most lanes work on small blocks too. In the
// second form an element's row and column come from e / d, computed as
// (e + 1/2) * (1/d) in single precision and truncated: for e < 2^10 and d <= 32
// the quotient stays at least 1/(2d) away from an integer, far beyond the
// rounding error, so it truncates to the exact integer quotient.
template <int TA, int TB, int SA, int SB>
__device__ __forceinline__ void f32_stage(const float* ga, const float* gb, int m, int n, int kk, float* a_s,
                                          float* b_s, int lane) {
    // op(A): element (i, l) of the stored block at i + l*m (TA = 0) or l + i*kk (TA = 1)
    const int da = TA ? kk : m, oa = TA ? m : kk;   // contiguous and other dimension
    if (da >= 16) {
        if (lane < da)
            for (int t = 0; t < oa; t++) {
                const int i = TA ? t : lane, l = TA ? lane : t;
                cp_async4(a_s + l * SA + i, ga + lane + t * da);
            }
    } else {
        const float ia = 1.0f / (float)da;
        for (int e = lane; e < m * kk; e += 32) {
            const int q = (int)(((float)e + 0.5f) * ia);
            const int i = TA ? q : e - q * m, l = TA ? e - q * kk : q;
            cp_async4(a_s + l * SA + i, ga + e);
        }
    }
    // op(B): element (l, j) at l + j*kk (TB = 0) or j + l*n (TB = 1)
    const int db = TB ? n : kk, ob = TB ? kk : n;
    if (db >= 16) {
        if (lane < db)
            for (int t = 0; t < ob; t++) {
                const int l = TB ? t : lane, j = TB ? lane : t;
                cp_async4(b_s + l * SB + j, gb + lane + t * db);
            }
    } else {
        const float ib = 1.0f / (float)db;
        for (int e = lane; e < kk * n; e += 32) {
            const int q = (int)(((float)e + 0.5f) * ib);
            const int l = TB ? q : e - q * kk, j = TB ? e - q * n : q;
            cp_async4(b_s + l * SB + j, gb + e);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// X consecutive floats from 16- (X = 4) or 8-byte (X = 2) aligned shared memory
template <int X>
__device__ __forceinline__ void f32_load(const float* p, float (&v)[X]) {
    if (X == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if (X == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int x = 0; x < X; x++) v[x] = p[x];
    }
}
// one lane's C block of the warp's chunk (lanes past the chunk hold zeros)
struct F32Blk {
    int64_t p0 = 0;        // first product
    int64_t c_off = 0;     // offset of the C block in the new C
    int64_t cold = -1;     // offset of its old block (beta != 0), -1 none
    int m = 0, n = 0, cnt = 0;
};

// A run of nrun C blocks of one patch class (lanes r0 .. r0 + nrun - 1 of the
// chunk) on one warp, R x CC patches with LC lanes across the columns and
// 32 / LC down the rows; rows padded to RP and columns to CP in the staging
// buffers. skk: the warp's inner size per stage.
template <int TA, int TB, int R, int CC, int LC, int RP, int CP>
__device__ __forceinline__ void f32_run(const SmmArgs& g, const F32Blk& me, int r0, int nrun, float* wbuf,
                                        int* skk, int lane, const BlasUpd& bu) {
    constexpr int SA = RP + 4, SB = CP + 4;
    constexpr int STAGE = 32 * (SA + SB);
    constexpr int NS = F32_WARP_FLOATS / STAGE < F32_MAX_STAGES ? F32_WARP_FLOATS / STAGE : F32_MAX_STAGES;
    static_assert(NS >= 2, "two stages at least");
    const unsigned full = 0xffffffffu;
    const int row0 = (lane / LC) * R, col0 = (lane % LC) * CC;
    // the run's product stream: C block i covers positions [excl_i, incl_i)
    const bool in_run = lane >= r0 && lane < r0 + nrun;
    int64_t incl = in_run ? me.cnt : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t v = __shfl_up_sync(full, incl, d);
        if (lane >= d) incl += v;
    }
    const int64_t excl = incl - (in_run ? me.cnt : 0);
    const int64_t total = __shfl_sync(full, incl, 31);
    // lane of the C block that holds stream position s (s < total, per lane):
    // the first lane of the run whose inclusive end exceeds s. A lower-bound
    // search with a fixed six halvings (enough for 32 lanes), so that every
    // lane runs every shuffle; only the bounds update is conditional.
    auto owner_of = [&](int64_t s) {
        int first = r0, count = nrun;
#pragma unroll
        for (int it = 0; it < 6; it++) {
            const int step = count >> 1;
            const int idx = min(first + step, 31);
            const int64_t v = __shfl_sync(full, incl, idx);
            if (count > 0) {
                if (v <= s) {
                    first += step + 1;
                    count -= step + 1;
                } else {
                    count = step;
                }
            }
        }
        return first;
    };
    // descriptors of stream positions sbase .. sbase + 31, one per lane
    int64_t sbase = -32, d_ao = 0, d_bo = 0;
    int d_kk = 0;
    auto stage = [&](int64_t s2, int slot) {   // s2 uniform, ascending across calls
        if (s2 >= sbase + 32) {
            sbase = s2;
            const int64_t mine = s2 + lane;
            // every lane takes part in the searches' shuffles
            const int ow = owner_of(mine < total ? mine : total - 1);
            const int64_t p = __shfl_sync(full, me.p0, ow) + (mine - __shfl_sync(full, excl, ow));
            const int om = __shfl_sync(full, me.m, ow);
            if (mine < total) {
                const int2 pr = g.prod[p];
                d_ao = g.A.off[pr.x];
                d_kk = (int)((g.A.off[pr.x + 1] - d_ao) / om);
                d_bo = g.B.off[pr.y];
            }
        }
        const int src = (int)(s2 - sbase);
        const int64_t ao = __shfl_sync(full, d_ao, src);
        const int64_t bo = __shfl_sync(full, d_bo, src);
        const int kk = __shfl_sync(full, d_kk, src);
        const unsigned before = __ballot_sync(full, in_run && incl <= s2);
        const int ow = r0 + __popc(before);
        const int m = __shfl_sync(full, me.m, ow), n = __shfl_sync(full, me.n, ow);
        if (lane == 0) skk[slot] = kk;
        float* a_s = wbuf + slot * STAGE;
        f32_stage<TA, TB, SA, SB>(g.A32 + ao, g.B32 + bo, m, n, kk, a_s, a_s + 32 * SA, lane);
    };
#pragma unroll 1
    for (int t = 0; t < NS - 1; t++) {
        if (t < total) stage(t, t);
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }
    int64_t s = 0;   // stream position being computed
    int cs = 0;      // its slot
#pragma unroll 1
    for (int i = 0; i < nrun; i++) {
        const int li = r0 + i;
        const int cnt = __shfl_sync(full, me.cnt, li);
        float acc[R][CC];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int c = 0; c < CC; c++) acc[r][c] = 0.f;
#pragma unroll 1
        for (int c = 0; c < cnt; c++, s++) {
            // slot cs - 1 (mod NS) was last read by position s - 1, finished by every lane
            __syncwarp();
            if (s + NS - 1 < total) stage(s + NS - 1, cs == 0 ? NS - 1 : cs - 1);
            else asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");
            __syncwarp();   // position s's blocks are in shared memory for every lane
            const int cur_kk = skk[cs];
            const float* ar = wbuf + cs * STAGE + row0;
            const float* bc = wbuf + cs * STAGE + 32 * SA + col0;
#pragma unroll 2
            for (int l = 0; l < cur_kk; l++) {
                float av[R], bv[CC];
                f32_load<R>(ar + l * SA, av);
                f32_load<CC>(bc + l * SB, bv);
#pragma unroll
                for (int r = 0; r < R; r++)
#pragma unroll
                    for (int q = 0; q < CC; q++) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
            }
            cs = cs + 1 == NS ? 0 : cs + 1;
        }
        // alpha / beta in FP64, column-major C block
        const int m = __shfl_sync(full, me.m, li), n = __shfl_sync(full, me.n, li);
        double* cout = g.Cd + __shfl_sync(full, me.c_off, li);
        const int64_t co = __shfl_sync(full, me.cold, li);
        const double* cold = co >= 0 ? g.Cold + co : nullptr;
#pragma unroll
        for (int c = 0; c < CC; c++) {
            const int j = col0 + c;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int ii = row0 + r;
                if (ii < m && j < n) {
                    const int64_t e = (int64_t)j * m + ii;
                    cout[e] = cold ? bu.update((double)acc[r][c], cold[e]) : bu.scale((double)acc[r][c]);
                }
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();   // the next run's first copies overwrite the slots
}

__device__ __forceinline__ int f32_class(int x) { return x <= 8 ? 0 : (x <= 16 ? 1 : 2); }

// patch class of each C block (rows 8 / 16 / 32 x columns 8 / 16 / 32), for
// a stable sort that lets the warps of an SM run one code path at a time
// (interleaved classes thrash the instruction cache)
__global__ void k_f32_classify(int64_t nC, const int* __restrict__ c_row, const int* __restrict__ c_col,
                               const int* __restrict__ rsC, const int* __restrict__ csC, uint32_t* __restrict__ key,
                               uint32_t* __restrict__ idx) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nC) return;
    const int m = rsC[c_row[q]], n = csC[c_col[q]];
    key[q] = (uint32_t)((m <= 8 ? 0 : (m <= 16 ? 1 : 2)) * 3 + (n <= 8 ? 0 : (n <= 16 ? 1 : 2)));
    idx[q] = (uint32_t)q;
}

template <int TA, int TB>
__global__ void __launch_bounds__(32 * F32_WARPS, 3) k_smm_f32_tile(SmmArgs g, const uint32_t* __restrict__ order,
                                                                    int chunk) {
    extern __shared__ __align__(16) float f32_smem[];
    __shared__ int s_kk[F32_WARPS][F32_MAX_STAGES];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* wbuf = f32_smem + warp * F32_WARP_FLOATS;
    int* skk = s_kk[warp];
    const BlasUpd bu(g.alpha, g.beta);
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(g.counter, (unsigned long long)chunk);
        const int64_t base = (int64_t)__shfl_sync(full, b, 0);
        if (base >= g.nC) break;
        const int cnt = (int)min((int64_t)chunk, g.nC - base);   // chunk <= 32
        // lane q: C block q of the chunk
        F32Blk me;
        int cls = -1;
        if (lane < cnt) {
            const int64_t cb = order ? (int64_t)order[base + lane] : base + lane;
            me.m = g.rsC[g.c_row[cb]];
            me.n = g.csC[g.c_col[cb]];
            me.p0 = g.c_pstart[cb];
            me.cnt = (int)(g.c_pstart[cb + 1] - me.p0);
            me.c_off = g.c_off[cb];
            const int o = g.c_old ? g.c_old[cb] : -1;
            me.cold = o >= 0 ? g.Cold_off[o] : -1;
            cls = f32_class(me.m) * 3 + f32_class(me.n);
        }
        // runs of one patch class
        for (int r0 = 0; r0 < cnt;) {
            const int c0 = __shfl_sync(full, cls, r0);
            const unsigned other = __ballot_sync(full, lane > r0 && lane < cnt && cls != c0);
            const int r1 = other ? __ffs(other) - 1 : cnt;
            switch (c0) {   // patch shape by padded size (rows 8 / 16 / 32) x (columns 8 / 16 / 32)
                case 0: f32_run<TA, TB, 2, 1, 8, 8, 8>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
                case 1: f32_run<TA, TB, 2, 2, 8, 8, 16>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
                case 2: f32_run<TA, TB, 2, 4, 8, 8, 32>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
                case 3: f32_run<TA, TB, 2, 2, 4, 16, 8>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
                case 4: f32_run<TA, TB, 4, 2, 8, 16, 16>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
                case 5: f32_run<TA, TB, 4, 4, 8, 16, 32>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
                case 6: f32_run<TA, TB, 4, 2, 4, 32, 8>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
                case 7: f32_run<TA, TB, 4, 4, 4, 32, 16>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
                default: f32_run<TA, TB, 8, 4, 8, 32, 32>(g, me, r0, r1 - r0, wbuf, skk, lane, bu); break;
            }
            r0 = r1;
        }
    }
}

// FP64 -> FP32, round to nearest even
__global__ void k_to_f32(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}

template <int Q>
int launch_fp32_q(const SmmArgs& g, const uint32_t* list, int64_t nlist) {
    cudaStream_t st = ctx().stream;
    const int threads = 256, teams_per_cta = 8;
    int grid = ctx().num_sms * (2048 / threads);
    if ((int64_t)grid * teams_per_cta > nlist) grid = (int)cdiv(nlist, teams_per_cta);
    if (grid < 1) return DBCSR_OK;
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(32, nlist / ((int64_t)grid * teams_per_cta * 4)));
    const int ta = g.A.trans, tb = g.B.trans;
    if (!ta && !tb) k_smm_fp32<Q, 0, 0><<<grid, threads, 0, st>>>(g, list, nlist, chunk);
    else if (ta && !tb) k_smm_fp32<Q, 1, 0><<<grid, threads, 0, st>>>(g, list, nlist, chunk);
    else if (!ta && tb) k_smm_fp32<Q, 0, 1><<<grid, threads, 0, st>>>(g, list, nlist, chunk);
    else k_smm_fp32<Q, 1, 1><<<grid, threads, 0, st>>>(g, list, nlist, chunk);
    DB_KCHECK();
    return DBCSR_OK;
}

int launch_fp32(const SmmArgs& g, int qidx, const uint32_t* list, int64_t nlist) {
    switch (qidx) {
        case 0: return launch_fp32_q<1>(g, list, nlist);
        case 1: return launch_fp32_q<2>(g, list, nlist);
        case 2: return launch_fp32_q<4>(g, list, nlist);
        case 3: return launch_fp32_q<8>(g, list, nlist);
        default: return launch_fp32_q<16>(g, list, nlist);   // larger blocks: several passes
    }
}

// Team size of each C block (index 0: one warp, 1: two, 2: four): forced,
// else from the tuning tables -- the (m, n, k) entry when one is set for the
// block's shape and the inner size k of its first product (tab3, kdim^3
// entries, m, n, k < kdim), else the (m, n) entry (table, tdim^2 entries),
// else one warp -- and the C blocks partitioned by it: group t at lists + t*nC,
// filled in CTA-sized runs (one reservation per CTA and group, ascending order
// inside a run). counts[t] must be zero on entry. Every C block is computed by
// one team with its products in plan order, so the order inside a group
// changes no result.
__global__ void __launch_bounds__(256) k_classify_team(int64_t nC, const int* __restrict__ c_row,
                                const int* __restrict__ c_col, const int64_t* __restrict__ c_pstart,
                                const int* __restrict__ rsC, const int* __restrict__ csC,
                                const signed char* __restrict__ table, int tdim,
                                const signed char* __restrict__ tab3, int kdim, const int2* __restrict__ prod,
                                const int64_t* __restrict__ a_off, int forced, uint32_t* __restrict__ lists,
                                int* __restrict__ counts) {
    __shared__ int s_wcnt[8][3];   // blocks per warp and group
    __shared__ int s_base[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int t = -1;
    if (b < nC) {
        const int m = rsC[c_row[b]], n = csC[c_col[b]];
        int v = forced >= 0 ? forced : 0;
        if (forced < 0 && m < tdim && n < tdim) {
            int tv = table ? table[m * tdim + n] : -1;
            if (tab3 && m < kdim && n < kdim && c_pstart[b + 1] > c_pstart[b]) {
                const int ax = prod[c_pstart[b]].x;
                const int k = (int)((a_off[ax + 1] - a_off[ax]) / m);
                if (k < kdim && tab3[(m * kdim + n) * kdim + k] >= 0) tv = tab3[(m * kdim + n) * kdim + k];
            }
            if (tv >= 0) v = tv;
            // a team only pays off with at least two products per warp; a C block
            // with fewer runs on one warp (its team-mates would wait at the barrier)
            const int64_t nprod = c_pstart[b + 1] - c_pstart[b];
            if (nprod < 2 * ((v == 2) ? 2 : (v == 3) ? 4 : 1)) v = 0;   // kTeamWarps[v]
        }
        t = (v == 2) ? 1 : (v == 3) ? 2 : 0;
    }
    int rank[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const unsigned msk = __ballot_sync(0xffffffffu, t == q);
        rank[q] = __popc(msk & ((1u << lane) - 1u));
        if (lane == 0) s_wcnt[warp][q] = __popc(msk);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int q = threadIdx.x;
        int tot = 0;
        for (int w = 0; w < 8; w++) {
            const int c = s_wcnt[w][q];
            s_wcnt[w][q] = tot;   // exclusive prefix over the CTA's warps
            tot += c;
        }
        s_base[q] = tot ? atomicAdd(&counts[q], tot) : 0;
    }
    __syncthreads();
    if (t >= 0) lists[t * nC + s_base[t] + s_wcnt[warp][t] + rank[t]] = (uint32_t)b;
}

template <int Q>
int launch_all_q(const SmmArgs& g, const uint32_t* list, const SmmGroups& gr) {
    cudaStream_t st = ctx().stream;
    const size_t red = (size_t)2 * 3 * Q * 32 * sizeof(double);   // two 4-warp teams per CTA
    const int ta = g.A.trans, tb = g.B.trans;
    static int occ[4] = {0, 0, 0, 0};   // resident CTAs per SM of each instance, from its first launch
    auto go = [&](auto kern, int which) -> int {
        if (occ[which] == 0) {
            DB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red));
            int o = 0;
            DB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 256, red));
            occ[which] = o > 0 ? o : 1;
        }
        int64_t grid = (int64_t)ctx().num_sms * occ[which];
        const int64_t nC = g.nC;
        if (grid > (nC + 1) / 2) grid = (nC + 1) / 2;   // at least two C blocks per CTA
        kern<<<(unsigned)grid, 256, red, st>>>(g, list, gr);
        DB_KCHECK();
        return DBCSR_OK;
    };
    if (!ta && !tb) return go(k_smm_fp64_all<Q, 0, 0>, 0);
    if (ta && !tb) return go(k_smm_fp64_all<Q, 1, 0>, 1);
    if (!ta && tb) return go(k_smm_fp64_all<Q, 0, 1>, 2);
    return go(k_smm_fp64_all<Q, 1, 1>, 3);
}

// the one launch over all C blocks; elements per lane from the largest C
// block, at most 16 (larger blocks take several passes: 16 warps per SM beat
// 8 warps holding 32 elements per lane, measured)
int launch_all(const SmmArgs& g, int max_mn, const uint32_t* list, const SmmGroups& gr) {
    switch (q_class(max_mn)) {
        case 0: return launch_all_q<1>(g, list, gr);
        case 1: return launch_all_q<2>(g, list, gr);
        case 2: return launch_all_q<4>(g, list, gr);
        case 3: return launch_all_q<8>(g, list, gr);
        default: return launch_all_q<16>(g, list, gr);
    }
}

// (m, n) -> variant table set by dbcsr_set_tuning, and (m, n, k) -> variant
// set by dbcsr_set_tuning_mnk; -1 = not set. The device copy is kept for the
// process and uploaded again before the first multiply after a change; the
// upload first waits for the last launch that read it (an event), which may sit
// on another stream after dbcsr_init switched streams.
constexpr int TDIM = 129;
constexpr int KDIM = 33;
constexpr size_t TABLE_BYTES = TDIM * TDIM + KDIM * KDIM * KDIM;
std::vector<signed char> g_table(TABLE_BYTES, -1);
bool g_table_used = false;
bool g_tab3_used = false;
bool g_table_dirty = true;
signed char* g_dtable = nullptr;
cudaEvent_t g_table_ev = nullptr;
bool g_table_ev_pending = false;

inline int team_of(int v) { return (v == 2) ? 1 : (v == 3) ? 2 : 0; }

int device_table(const signed char** out) {
    cudaStream_t st = ctx().stream;
    if (!g_dtable) {
        cudaError_t e = cudaMalloc(&g_dtable, TABLE_BYTES);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g_dtable = nullptr;
            return fail(DBCSR_ERR_ALLOC, std::string("tuning table: ") + cudaGetErrorString(e));
        }
        DB_CUDA(cudaEventCreateWithFlags(&g_table_ev, cudaEventDisableTiming));
        g_table_dirty = true;
    }
    if (g_table_dirty) {
        if (g_table_ev_pending) DB_CUDA(cudaEventSynchronize(g_table_ev));
        DB_CUDA(cudaMemcpyAsync(g_dtable, g_table.data(), TABLE_BYTES, cudaMemcpyHostToDevice, st));
        g_table_dirty = false;
    }
    *out = g_dtable;
    return DBCSR_OK;
}

}  // namespace

int smm_set_table_mnk(const int* m, const int* n, const int* k, const int* variant, int count) {
    std::vector<signed char> t(KDIM * KDIM * KDIM, -1);
    for (int q = 0; q < count; q++) {
        if (m[q] < 1 || m[q] >= KDIM || n[q] < 1 || n[q] >= KDIM || k[q] < 1 || k[q] >= KDIM || variant[q] < 0 ||
            variant[q] >= SMM_NUM_VARIANTS)
            return fail(DBCSR_ERR_ARG, "set_tuning_mnk: entry " + std::to_string(q) + " out of range");
        t[(m[q] * KDIM + n[q]) * KDIM + k[q]] = (signed char)variant[q];
    }
    std::copy(t.begin(), t.end(), g_table.begin() + TDIM * TDIM);
    g_tab3_used = count > 0;
    g_table_dirty = true;
    return DBCSR_OK;
}

int smm_set_table(const int* m, const int* n, const int* variant, int count) {
    std::vector<signed char> t(TDIM * TDIM, -1);
    for (int q = 0; q < count; q++) {
        if (m[q] < 1 || m[q] >= TDIM || n[q] < 1 || n[q] >= TDIM || variant[q] < 0 ||
            variant[q] >= SMM_NUM_VARIANTS)
            return fail(DBCSR_ERR_ARG, "set_tuning: entry " + std::to_string(q) + " out of range");
        t[m[q] * TDIM + n[q]] = (signed char)variant[q];
    }
    std::copy(t.begin(), t.end(), g_table.begin());
    g_table_used = count > 0;
    g_table_dirty = true;
    return DBCSR_OK;
}

int smm_table_team_bound(const std::vector<int>& ms, const std::vector<int>& ns, const std::vector<int>& ks) {
    if (!g_table_used && !g_tab3_used) return 0;
    if ((double)ms.size() * (double)ns.size() * (double)(ks.size() + 1) > 4e6) return 2;
    // the classify kernel's choice for every (m, n) and inner size k of a first
    // product: the (m, n, k) entry where set, else the (m, n) entry, else 0
    int best = 0;
    for (int m : ms)
        for (int n : ns) {
            if (m >= TDIM || n >= TDIM) continue;   // untuned: variant 0
            const int vmn = std::max<int>(0, g_table[m * TDIM + n]);
            for (int k : ks) {
                int v = vmn;
                if (g_tab3_used && m < KDIM && n < KDIM && k < KDIM) {
                    const int t3 = g_table[TDIM * TDIM + (m * KDIM + n) * KDIM + k];
                    if (t3 >= 0) v = t3;
                }
                best = std::max(best, team_of(v));
            }
            if (best == 2) return 2;
        }
    return best;
}

int smm_fp64_generic(const SmmArgs& g, int max_mn) {
    if (g.nC == 0) return DBCSR_OK;
    return launch_all(g, max_mn, nullptr, SmmGroups{nullptr, g.nC, g.counter, 0});
}

// kernel: 0 = tuned tables (variant 0 for untuned shapes), v >= 1 = force variant v-1.
// One launch of the product kernel; with teams of two or four warps possible,
// a classify pass first partitions the C blocks by team size on the device.
int smm_fp64_dispatch(const SmmArgs& g, int max_mn, int kernel, int team_bound) {
    if (g.nC == 0) return DBCSR_OK;
    if (kernel < 0 || kernel > SMM_NUM_VARIANTS) return fail(DBCSR_ERR_ARG, "unknown stack kernel variant");
    if (g.nC >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "stack kernels: too many C blocks");
    const bool use_table = kernel == 0 && (g_table_used || g_tab3_used) && team_bound > 0;
    const int forced = kernel >= 1 ? kernel - 1 : -1;
    if (!use_table && (forced < 0 || kTeamWarps[forced] == 1))
        return launch_all(g, max_mn, nullptr, SmmGroups{nullptr, g.nC, g.counter, 0});
    cudaStream_t st = ctx().stream;
    const signed char* table = nullptr;
    if (use_table) DB_TRY(device_table(&table));
    DBuf<uint32_t> lists;
    DBuf<unsigned long long> grp;   // [0, 3): work counters; [3, 5): counts (int)
    DB_TRY(lists.alloc((size_t)3 * g.nC));
    DB_TRY(grp.alloc(5));
    DB_CUDA(cudaMemsetAsync(grp.p, 0, sizeof(unsigned long long) * 5, st));
    int* counts = reinterpret_cast<int*>(grp.p + 3);
    k_classify_team<<<(unsigned)cdiv(g.nC, 256), 256, 0, st>>>(
        g.nC, g.c_row, g.c_col, g.c_pstart, g.rsC, g.csC, table, TDIM,
        (table && g_tab3_used) ? table + TDIM * TDIM : nullptr, KDIM, g.prod, g.A.off, forced, lists.p, counts);
    DB_KCHECK();
    if (table) {
        DB_CUDA(cudaEventRecord(g_table_ev, st));
        g_table_ev_pending = true;
    }
    return launch_all(g, max_mn, lists.p, SmmGroups{counts, 0, grp.p, g.nC});
}

int to_f32(const double* in, int64_t n, float* out) {
    if (n <= 0) return DBCSR_OK;
    const int grid = (int)std::min<int64_t>(cdiv(n, 256), (int64_t)ctx().num_sms * 32);
    k_to_f32<<<grid, 256, 0, ctx().stream>>>(n, in, out);
    DB_KCHECK();
    return DBCSR_OK;
}

// FP32 stack kernels: blocks up to 32 x 32 on the shared-memory kernel, larger
// ones on the generic body, one warp each; one launch either way.
int smm_fp32_dispatch(const SmmArgs& g, int max_mn, int max_edge) {
    if (g.nC == 0) return DBCSR_OK;
    if (max_edge <= 32) {
        cudaStream_t st = ctx().stream;
        if (g.nC >= (int64_t)UINT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "stack kernels: too many C blocks");
        DBuf<uint32_t> key, order;
        DB_TRY(key.alloc(g.nC));
        DB_TRY(order.alloc(g.nC));
        k_f32_classify<<<(unsigned)cdiv(g.nC, 256), 256, 0, st>>>(g.nC, g.c_row, g.c_col, g.rsC, g.csC, key.p,
                                                                  order.p);
        DB_KCHECK();
        DB_TRY(radix_sort_u32(key.p, order.p, g.nC, 4));
        int grid = ctx().num_sms * 3;
        if ((int64_t)grid * F32_WARPS > g.nC) grid = (int)cdiv(g.nC, F32_WARPS);
        // C blocks per grab: up to 32 (one per lane), at least ~4 grabs per warp
        const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(32, g.nC / ((int64_t)grid * F32_WARPS * 4)));
        const int ta = g.A.trans, tb = g.B.trans;
#define DB_LAUNCH_F32(TA_, TB_)                                                                          \
    do {                                                                                                \
        DB_CUDA(cudaFuncSetAttribute(k_smm_f32_tile<TA_, TB_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     F32_SMEM));                                                        \
        k_smm_f32_tile<TA_, TB_><<<grid, 32 * F32_WARPS, F32_SMEM, st>>>(g, order.p, chunk);            \
    } while (0)
        if (!ta && !tb) DB_LAUNCH_F32(0, 0);
        else if (ta && !tb) DB_LAUNCH_F32(1, 0);
        else if (!ta && tb) DB_LAUNCH_F32(0, 1);
        else DB_LAUNCH_F32(1, 1);
#undef DB_LAUNCH_F32
        DB_KCHECK();
        return DBCSR_OK;
    }
    if (g.nC >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "stack kernels: too many C blocks");
    // larger blocks: one launch, up to 16 elements per lane (more in passes)
    return launch_fp32(g, q_class(max_mn), nullptr, g.nC);
}

}  // namespace dbcsr
