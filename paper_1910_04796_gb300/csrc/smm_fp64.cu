// smm_fp64.cu -- batched FP64 small-matrix products over the stack list.
//
// Paper, Sec. II: batches of block products C_ij += A_ik B_kj are executed by
// LIBCUSMM, CUDA kernels for small (m,n,k) auto-tuned over read/write strategy,
// threads per block, elements per thread and tiling. This file holds the
// GB300 kernels that play that role for FP64, and the per-shape dispatch that
// the autotuner's table drives.
//
// GB300 facts that shape them: FP64 runs at about 1 TFLOP/s on the whole chip
// (DFMA and DMMA alike), i.e. under two FP64 FMAs per clock per SM, so a small
// block product is arithmetic-bound (the ridge point is ~0.15 flop/byte
// against 6.7 TB/s HBM) and everything else -- loads, index arithmetic --
// hides behind the FMA pipe. What matters is (1) keeping every lane of every
// DFMA busy (elements mapped densely onto lanes), (2) enough independent
// accumulators per lane to cover the FMA latency, (3) reading each C block
// once and writing it once. A team of W warps owns one C block: it walks the
// block's products (ascending k, as stack generation ordered them; with W > 1
// warp w takes products w, w+W, ... and the partial sums are added in warp
// order through shared memory), keeps the C block in registers, and writes
// alpha*acc + beta*C_old once -- no atomics on C. Work is handed out by an
// atomic counter over a (possibly variant-filtered) list of C blocks
// (persistent grid).
#include <vector>

#include "internal.cuh"
#include "smm.cuh"

namespace dbcsr {

namespace {

// Variants (the autotuner's search space):
//   0: 1 warp per C block, 256-thread CTAs      1: 1 warp per C block, 128-thread CTAs
//   2: 2-warp teams, 256-thread CTAs            3: 4-warp teams, 256-thread CTAs
struct VariantShape {
    int team_warps;
    int cta_threads;
};
constexpr VariantShape kVariants[SMM_NUM_VARIANTS] = {{1, 256}, {1, 128}, {2, 256}, {4, 256}};

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

// one team per C block; each lane holds up to Q elements e = lane + 32*q,
// r = e % m, c = e / m (column-major order within the block)
template <int Q, int TA, int TB, int W>
__global__ void __launch_bounds__(256) k_smm_fp64(SmmArgs g, const int* __restrict__ list, int64_t nlist) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int team = warp / W, tw = warp % W;        // team in CTA, warp in team
    __shared__ int s_cb[8];
    extern __shared__ double s_red[];                 // [teams][W-1][Q][32] partial sums
    for (;;) {
        if (tw == 0 && lane == 0) s_cb[team] = (int)atomicAdd(g.counter, 1ULL);
        team_sync<W>(team);
        const int64_t li = s_cb[team];
        team_sync<W>(team);
        if (li >= nlist) break;
        const int64_t cb = list ? list[li] : li;
        const int i = g.c_row[cb], j = g.c_col[cb];
        const int m = g.rsC[i], n = g.csC[j];
        const int mn = m * n;
        const int64_t p0 = g.c_pstart[cb], p1 = g.c_pstart[cb + 1];
        double* cout = g.Cd + g.c_off[cb];
        const int old = g.c_old ? g.c_old[cb] : -1;
        const double* cold = (old >= 0) ? g.Cold + g.Cold_off[old] : nullptr;
        for (int e0 = 0; e0 < mn; e0 += 32 * Q) {
            const int nq = min(Q, (mn - e0 + 31) >> 5);
            double acc[Q];
            int ro[Q], co[Q];
#pragma unroll
            for (int q = 0; q < Q; q++) {
                acc[q] = 0.0;
                int e = e0 + lane + 32 * q;
                if (e >= mn) e = 0;
                ro[q] = e % m;
                co[q] = e / m;
            }
            for (int64_t p = p0 + tw; p < p1; p += W) {
                const int2 pr = g.prod[p];
                const int64_t ao = g.A.off[pr.x];
                const int kk = (int)((g.A.off[pr.x + 1] - ao) / m);
                const double* __restrict__ a = g.A.data + ao;
                const double* __restrict__ b = g.B.data + g.B.off[pr.y];
                int aidx[Q], bidx[Q];
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    aidx[q] = TA ? ro[q] * kk : ro[q];
                    bidx[q] = TB ? co[q] : co[q] * kk;
                }
                const int astep = TA ? 1 : m;
                const int bstep = TB ? n : 1;
                for (int l = 0; l < kk; l++) {
#pragma unroll
                    for (int q = 0; q < Q; q++) {
                        if (q < nq) acc[q] = fma(__ldg(a + aidx[q]), __ldg(b + bidx[q]), acc[q]);
                        aidx[q] += astep;
                        bidx[q] += bstep;
                    }
                }
            }
            if (W > 1) {
                // partial sums of warps 1..W-1 to shared memory, added in warp order by warp 0
                double* red = s_red + (size_t)team * (W - 1) * Q * 32;
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
                        double v = __dmul_rn(g.alpha, acc[q]);
                        if (cold) v = __dadd_rn(v, __dmul_rn(g.beta, cold[e]));
                        cout[e] = v;
                    }
                }
            }
        }
    }
}

template <int Q, int W>
int launch_qw(const SmmArgs& g, const int* list, int64_t nlist, int threads) {
    cudaStream_t st = ctx().stream;
    const int teams_per_cta = threads / (32 * W);
    int grid = ctx().num_sms * (2048 / threads);
    if ((int64_t)grid * teams_per_cta > nlist) grid = (int)cdiv(nlist, teams_per_cta);
    if (grid < 1) return DBCSR_OK;
    const size_t red = (W > 1) ? (size_t)teams_per_cta * (W - 1) * Q * 32 * sizeof(double) : 0;
    const int ta = g.A.trans, tb = g.B.trans;
#define DB_LAUNCH_SMM(TA_, TB_)                                                                             \
    do {                                                                                                   \
        if (red > 0)                                                                                       \
            DB_CUDA(cudaFuncSetAttribute(k_smm_fp64<Q, TA_, TB_, W>,                                       \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red));          \
        k_smm_fp64<Q, TA_, TB_, W><<<grid, threads, red, st>>>(g, list, nlist);                             \
    } while (0)
    if (!ta && !tb) DB_LAUNCH_SMM(0, 0);
    else if (ta && !tb) DB_LAUNCH_SMM(1, 0);
    else if (!ta && tb) DB_LAUNCH_SMM(0, 1);
    else DB_LAUNCH_SMM(1, 1);
#undef DB_LAUNCH_SMM
    DB_KCHECK();
    return DBCSR_OK;
}

template <int W>
int launch_w(const SmmArgs& g, const int* list, int64_t nlist, int threads, int max_mn) {
    const int q = (max_mn + 31) / 32;
    if (q <= 1) return launch_qw<1, W>(g, list, nlist, threads);
    if (q <= 2) return launch_qw<2, W>(g, list, nlist, threads);
    if (q <= 4) return launch_qw<4, W>(g, list, nlist, threads);
    if (q <= 8) return launch_qw<8, W>(g, list, nlist, threads);
    if (q <= 16) return launch_qw<16, W>(g, list, nlist, threads);
    return launch_qw<32, W>(g, list, nlist, threads);   // larger blocks loop over element chunks
}

int launch_variant(const SmmArgs& g, int variant, const int* list, int64_t nlist, int max_mn) {
    const VariantShape v = kVariants[variant];
    switch (v.team_warps) {
        case 1: return launch_w<1>(g, list, nlist, v.cta_threads, max_mn);
        case 2: return launch_w<2>(g, list, nlist, v.cta_threads, max_mn);
        default: return launch_w<4>(g, list, nlist, v.cta_threads, max_mn);
    }
}

// variant of every C block from the (m, n) table; counts per variant
__global__ void k_classify(int64_t nC, const int* __restrict__ c_row, const int* __restrict__ c_col,
                           const int* __restrict__ rsC, const int* __restrict__ csC,
                           const signed char* __restrict__ table, int tdim, int dflt, int* __restrict__ var,
                           int* __restrict__ counts) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nC) return;
    const int m = rsC[c_row[b]], n = csC[c_col[b]];
    int v = dflt;
    if (m < tdim && n < tdim) {
        const int t = table[m * tdim + n];
        if (t >= 0) v = t;
    }
    var[b] = v;
    atomicAdd(&counts[v], 1);
}

// stable per-variant lists (one CTA, ordered scan over the blocks)
__global__ void k_partition(int64_t nC, const int* __restrict__ var, const int* __restrict__ start,
                            int* __restrict__ list) {
    __shared__ int cursor[SMM_NUM_VARIANTS];
    if (threadIdx.x < SMM_NUM_VARIANTS) cursor[threadIdx.x] = start[threadIdx.x];
    __syncthreads();
    for (int64_t base = 0; base < nC; base += blockDim.x) {
        const int64_t b = base + threadIdx.x;
        const int v = b < nC ? var[b] : -1;
        for (int w = 0; w < SMM_NUM_VARIANTS; w++) {
            const unsigned mask = __ballot_sync(0xffffffffu, v == w);
            __shared__ int warp_cnt[32];
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            if (lane == 0) warp_cnt[wid] = __popc(mask);
            __syncthreads();
            int before = 0;
            for (int q = 0; q < wid; q++) before += warp_cnt[q];
            if (v == w) list[cursor[w] + before + __popc(mask & ((1u << lane) - 1u))] = (int)b;
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int q = 0; q < (int)(blockDim.x >> 5); q++) tot += warp_cnt[q];
                cursor[w] += tot;
            }
            __syncthreads();
        }
    }
}

// (m, n) -> variant table set by dbcsr_set_tuning; -1 = default
constexpr int TDIM = 129;
std::vector<signed char> g_table(TDIM* TDIM, -1);
bool g_table_used = false;

}  // namespace

int smm_set_table(const int* m, const int* n, const int* variant, int count) {
    std::vector<signed char> t(TDIM * TDIM, -1);
    for (int q = 0; q < count; q++) {
        if (m[q] < 1 || m[q] >= TDIM || n[q] < 1 || n[q] >= TDIM || variant[q] < 0 ||
            variant[q] >= SMM_NUM_VARIANTS)
            return fail(DBCSR_ERR_ARG, "set_tuning: entry " + std::to_string(q) + " out of range");
        t[m[q] * TDIM + n[q]] = (signed char)variant[q];
    }
    g_table = t;
    g_table_used = count > 0;
    return DBCSR_OK;
}

int smm_fp64_generic(const SmmArgs& g, int max_mn) { return launch_variant(g, 0, nullptr, g.nC, max_mn); }

// kernel: 0 = tuned table (default variant 0 for untuned shapes), v >= 1 = force variant v-1
int smm_fp64_dispatch(const SmmArgs& g, int max_mn, int kernel) {
    if (g.nC == 0) return DBCSR_OK;
    if (kernel < 0 || kernel > SMM_NUM_VARIANTS) return fail(DBCSR_ERR_ARG, "unknown stack kernel variant");
    if (kernel >= 1 || !g_table_used) return launch_variant(g, kernel >= 1 ? kernel - 1 : 0, nullptr, g.nC, max_mn);
    cudaStream_t st = ctx().stream;
    DBuf<signed char> table;
    DBuf<int> var, counts, list;
    DB_TRY(table.alloc(TDIM * TDIM));
    DB_TRY(var.alloc(g.nC));
    DB_TRY(counts.alloc(SMM_NUM_VARIANTS));
    DB_TRY(list.alloc(g.nC));
    DB_CUDA(cudaMemcpyAsync(table.p, g_table.data(), TDIM * TDIM, cudaMemcpyHostToDevice, st));
    DB_CUDA(cudaMemsetAsync(counts.p, 0, sizeof(int) * SMM_NUM_VARIANTS, st));
    k_classify<<<(unsigned)cdiv(g.nC, 256), 256, 0, st>>>(g.nC, g.c_row, g.c_col, g.rsC, g.csC, table.p, TDIM, 0,
                                                          var.p, counts.p);
    DB_KCHECK();
    int h_counts[SMM_NUM_VARIANTS];
    DB_CUDA(cudaMemcpyAsync(h_counts, counts.p, sizeof(h_counts), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    int used = 0, only = 0;
    for (int v = 0; v < SMM_NUM_VARIANTS; v++)
        if (h_counts[v]) { used++; only = v; }
    if (used <= 1) return launch_variant(g, only, nullptr, g.nC, max_mn);
    int h_start[SMM_NUM_VARIANTS];
    int run = 0;
    for (int v = 0; v < SMM_NUM_VARIANTS; v++) { h_start[v] = run; run += h_counts[v]; }
    DBuf<int> start;
    DB_TRY(start.alloc(SMM_NUM_VARIANTS));
    DB_CUDA(cudaMemcpyAsync(start.p, h_start, sizeof(h_start), cudaMemcpyHostToDevice, st));
    k_partition<<<1, 1024, 0, st>>>(g.nC, var.p, start.p, list.p);
    DB_KCHECK();
    // each variant's launch works through its own list with its own counter
    DBuf<unsigned long long> ctr;
    DB_TRY(ctr.alloc(SMM_NUM_VARIANTS));
    DB_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned long long) * SMM_NUM_VARIANTS, st));
    for (int v = 0; v < SMM_NUM_VARIANTS; v++) {
        if (!h_counts[v]) continue;
        SmmArgs gv = g;
        gv.counter = ctr.p + v;
        DB_TRY(launch_variant(gv, v, list.p + h_start[v], h_counts[v], max_mn));
    }
    DB_CUDA(cudaStreamSynchronize(st));   // h_start / h_counts above are stack memory
    return DBCSR_OK;
}

}  // namespace dbcsr
