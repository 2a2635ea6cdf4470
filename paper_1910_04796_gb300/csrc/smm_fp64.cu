// smm_fp64.cu -- batched FP64 small-matrix products over the stack list.
//
// Paper, Sec. II: batches of block products C_ij += A_ik B_kj are executed by
// LIBCUSMM, CUDA kernels for small (m,n,k) auto-tuned over read/write strategy,
// threads per block, elements per thread and tiling. This file holds the
// GB300 kernels that play that role for FP64.
//
// GB300 facts that shape them: FP64 runs at about 1 TFLOP/s on the whole chip
// (DFMA and DMMA alike), i.e. under two FP64 FMAs per clock per SM, so a small
// block product is arithmetic-bound (the ridge point is ~0.15 flop/byte
// against 6.7 TB/s HBM) and everything else -- loads, index arithmetic --
// hides behind the FMA pipe. What matters is (1) keeping every lane of every
// DFMA busy (elements mapped densely onto lanes), (2) enough independent
// accumulators per lane to cover the FMA latency, (3) reading each C block
// once and writing it once. One warp owns one C block: it walks the block's
// products (ascending k, as stack generation ordered them), keeps the C block
// in registers, and writes alpha*acc + beta*C_old once at the end -- no
// atomics on C. Work is handed out by an atomic counter (persistent grid).
#include "internal.cuh"
#include "smm.cuh"

namespace dbcsr {

namespace {

// one warp per C block; each lane holds up to Q elements e = lane + 32*q,
// r = e % m, c = e / m (column-major order within the block)
template <int Q, int TA, int TB>
__global__ void __launch_bounds__(256) k_smm_fp64_warp(SmmArgs g) {
    const int lane = threadIdx.x & 31;
    const int nwarp_cta = blockDim.x >> 5;
    __shared__ int s_cb[8];
    const int w = threadIdx.x >> 5;
    for (;;) {
        if (lane == 0) s_cb[w] = (int)atomicAdd(g.counter, 1ULL);
        __syncwarp();
        const int64_t cb = s_cb[w];
        __syncwarp();
        if (cb >= g.nC) break;
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
            for (int64_t p = p0; p < p1; p++) {
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

template <int Q>
int launch_q(const SmmArgs& g, int grid) {
    cudaStream_t st = ctx().stream;
    const int ta = g.A.trans, tb = g.B.trans;
    if (!ta && !tb) k_smm_fp64_warp<Q, 0, 0><<<grid, 256, 0, st>>>(g);
    else if (ta && !tb) k_smm_fp64_warp<Q, 1, 0><<<grid, 256, 0, st>>>(g);
    else if (!ta && tb) k_smm_fp64_warp<Q, 0, 1><<<grid, 256, 0, st>>>(g);
    else k_smm_fp64_warp<Q, 1, 1><<<grid, 256, 0, st>>>(g);
    DB_KCHECK();
    return DBCSR_OK;
}

}  // namespace

int smm_fp64_generic(const SmmArgs& g, int max_mn) {
    if (g.nC == 0) return DBCSR_OK;
    const int q = (max_mn + 31) / 32;
    int grid = ctx().num_sms * 8;
    if ((int64_t)grid * 8 > g.nC) grid = (int)cdiv(g.nC, 8);
    if (q <= 1) return launch_q<1>(g, grid);
    if (q <= 2) return launch_q<2>(g, grid);
    if (q <= 4) return launch_q<4>(g, grid);
    if (q <= 8) return launch_q<8>(g, grid);
    if (q <= 16) return launch_q<16>(g, grid);
    return launch_q<32>(g, grid);   // larger blocks loop over element chunks
}

}  // namespace dbcsr
