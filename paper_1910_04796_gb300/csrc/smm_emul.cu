// smm_emul.cu -- the stack path in emulated FP64: batched small block
// products with 7-bit integer slices on the tensor cores (mma.sync bf16).
//
// Same emulation as the dense path (Ozaki, Ogita, Oishi & Rump 2012, integer
// form), applied without densifying: the row exponents e come from the whole
// element rows of op(A) (max over all stored blocks of the block row), the
// column exponents f from the whole element columns of op(B), every stored
// block is cut into s slices once, and each C block accumulates its exact
// level sums G_d = sum_k sum_{t+u=d} S^A_t(i,k) S^B_u(k,j) over its products.
// Because G_d is exact, the result is identical to the dense emulation of the
// densified operands (the oracle checks this bit for bit).
//
// Kernel: one CTA (4 warps) per C block up to 32 x 32, each warp a 16 x 16
// quadrant. Per product, the s slices of the A block and of the B block are
// staged in shared memory (cp.async); each warp runs m16n8k16 bf16 MMAs for
// every pair t + u <= s + 1 into per-level fp32 accumulators. fp32 sums of
// integer products are exact below 2^24, so the accumulators are flushed into
// per-level int32 sums every F products (F * s * k <= 1040); int32 is exact
// while products * s * k * 127^2 < 2^31 (checked on the host). At the end the
// level sums are recombined in FP64 exactly as the dense path does.
#include <cuda_bf16.h>

#include "emul.cuh"
#include "emul_common.cuh"
#include "internal.cuh"
#include "smm.cuh"
#include "smm_emul.cuh"

namespace dbcsr {

namespace {

constexpr int SE_THREADS = 128;
constexpr int SE_MAXB = EMUL_STACK_MAX_EDGE;    // largest block edge on this path
constexpr int SE_RS = 40;      // shared-memory row stride (bf16): 32 + 8, conflict-free fragments

__host__ __device__ inline int ru16(int x) { return (x + 15) & ~15; }

// max |x| over each op() line: warp per stored block, lane per line
__global__ void k_se_linemax(SliceGeom G, unsigned long long* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = w0; b < G.nblks; b += nw) {
        int X, L, xs, ls;
        int64_t xbase;
        geom_block(G, b, X, L, xs, ls, xbase);
        const double* d = G.data + G.off[b];
        for (int x = lane; x < X; x += 32) {
            unsigned long long mx = 0;
            for (int l = 0; l < L; l++) {
                unsigned long long v = emul::abs_bits(d[(int64_t)x * xs + (int64_t)l * ls]);
                mx = v > mx ? v : mx;
            }
            if (mx) atomicMax(&out[xbase + x], mx);
        }
    }
}

__global__ void k_se_exponents(int64_t n, const unsigned long long* __restrict__ bits, int* __restrict__ e) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) e[i] = emul::exponent_of_bits(bits[i]);
}

__global__ void k_se_slice_sizes(SliceGeom G, int64_t* __restrict__ sz) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= G.nblks) return;
    int X, L, xs, ls;
    int64_t xbase;
    geom_block(G, b, X, L, xs, ls, xbase);
    sz[b] = (int64_t)ru16(X) * ru16(L);
}

// slices of every stored block, row-like (x, l) layout padded to 16 x 16
__global__ void k_se_slice(SliceGeom G, const int* __restrict__ ex, int s, const int64_t* __restrict__ soff,
                           int64_t total, __nv_bfloat16* __restrict__ S) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = w0; b < G.nblks; b += nw) {
        int X, L, xs, ls;
        int64_t xbase;
        geom_block(G, b, X, L, xs, ls, xbase);
        const int Xp = ru16(X), Lp = ru16(L);
        const double* d = G.data + G.off[b];
        const int npairs = Xp * Lp / 2;
        for (int e2 = lane; e2 < npairs; e2 += 32) {
            const int x = (2 * e2) / Lp, l = (2 * e2) % Lp;
            long long q0 = 0, q1 = 0;
            if (x < X) {
                const int e = ex[xbase + x];
                if (l < L) q0 = emul::fixed_point(d[(int64_t)x * xs + (int64_t)l * ls], e, s);
                if (l + 1 < L) q1 = emul::fixed_point(d[(int64_t)x * xs + (int64_t)(l + 1) * ls], e, s);
            }
            for (int t = 1; t <= s; t++) {
                __nv_bfloat162 pr;
                pr.x = emul::slice_bf16(q0, t, s);
                pr.y = emul::slice_bf16(q1, t, s);
                *reinterpret_cast<__nv_bfloat162*>(S + (int64_t)(t - 1) * total + soff[b] + 2 * e2) = pr;
            }
        }
    }
}

struct SeArgs {
    int64_t nC;
    const int* c_row;
    const int* c_col;
    const int64_t* c_off;
    const int* c_old;
    const int64_t* c_pstart;
    const int2* prod;
    const int64_t* a_off;       // stored A element offsets (sentinel at nblks)
    const int* rsC;
    const int* csC;
    const int64_t* croff;       // element row offsets of C
    const int64_t* ccoff;       // element column offsets of C
    const int* e;               // row exponents (C element rows)
    const int* f;               // column exponents (C element columns)
    const __nv_bfloat16* SA;
    const __nv_bfloat16* SB;
    int64_t totA, totB;         // elements per slice of all A / B blocks
    const int64_t* soffA;
    const int64_t* soffB;
    double* Cd;
    const double* Cold;
    const int64_t* Cold_off;
    double alpha, beta;
    int flush_every;            // products between exact fp32 -> int32 flushes
    unsigned long long* counter;
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage the s slices of product p's A and B blocks into one shared-memory
// buffer (16-byte cp.async chunks, rows padded to SE_RS).
template <int S>
__device__ __forceinline__ void stage_product(const SeArgs& a, int64_t p, int m, int n, __nv_bfloat16* sA,
                                              __nv_bfloat16* sB, int tid) {
    const int2 pr = a.prod[p];
    const int kk = (int)((a.a_off[pr.x + 1] - a.a_off[pr.x]) / m);
    const int kp = ru16(kk), mp = ru16(m), np = ru16(n);
    const int cpr = kp / 8;   // chunks per row
    const int na = S * mp * cpr, nb = S * np * cpr;
    const __nv_bfloat16* ga = a.SA + a.soffA[pr.x];
    const __nv_bfloat16* gb = a.SB + a.soffB[pr.y];
    for (int c = tid; c < na + nb; c += SE_THREADS) {
        if (c < na) {
            const int t = c / (mp * cpr), rem = c % (mp * cpr), x = rem / cpr, ch = rem % cpr;
            cp_async16(sA + (t * SE_MAXB + x) * SE_RS + ch * 8, ga + (int64_t)t * a.totA + x * kp + ch * 8);
        } else {
            const int c2 = c - na;
            const int t = c2 / (np * cpr), rem = c2 % (np * cpr), x = rem / cpr, ch = rem % cpr;
            cp_async16(sB + (t * SE_MAXB + x) * SE_RS + ch * 8, gb + (int64_t)t * a.totB + x * kp + ch * 8);
        }
    }
}

template <int S>
__global__ void __launch_bounds__(SE_THREADS) k_smm_emul(SeArgs a) {
    extern __shared__ __align__(16) unsigned char se_smem[];
    // two buffers, each [S][32][SE_RS] for A then [S][32][SE_RS] for B
    __nv_bfloat16* buf0 = reinterpret_cast<__nv_bfloat16*>(se_smem);
    constexpr int BUF = 2 * S * SE_MAXB * SE_RS;
    __shared__ int s_cb;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int g = lane >> 2, q = lane & 3;
    const BlasUpd bu(a.alpha, a.beta);
    for (;;) {
        if (tid == 0) s_cb = (int)atomicAdd(a.counter, 1ULL);
        __syncthreads();
        const int64_t cb = s_cb;
        __syncthreads();
        if (cb >= a.nC) break;
        const int i = a.c_row[cb], j = a.c_col[cb];
        const int m = a.rsC[i], n = a.csC[j];
        const bool active = (wm * 16 < m) && (wn * 16 < n);
        const int64_t p0 = a.c_pstart[cb], p1 = a.c_pstart[cb + 1];
        float acc[S][2][4];
        int gi[S][2][4];
#pragma unroll
        for (int d = 0; d < S; d++)
#pragma unroll
            for (int nt = 0; nt < 2; nt++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    acc[d][nt][r] = 0.f;
                    gi[d][nt][r] = 0;
                }
        int since = 0;
        if (p0 < p1) stage_product<S>(a, p0, m, n, buf0, buf0 + S * SE_MAXB * SE_RS, tid);
        cp_async_commit();
        for (int64_t p = p0; p < p1; p++) {
            const int cur = (int)((p - p0) & 1);
            __nv_bfloat16* sA = buf0 + cur * BUF;
            __nv_bfloat16* sB = sA + S * SE_MAXB * SE_RS;
            // prefetch the next product into the other buffer while this one computes
            if (p + 1 < p1) {
                __nv_bfloat16* nA = buf0 + (cur ^ 1) * BUF;
                stage_product<S>(a, p + 1, m, n, nA, nA + S * SE_MAXB * SE_RS, tid);
            }
            cp_async_commit();
            cp_async_wait_group<1>();
            __syncthreads();
            if (active) {
                const int2 pr = a.prod[p];
                const int kk = (int)((a.a_off[pr.x + 1] - a.a_off[pr.x]) / m);
                const int nks = ru16(kk) / 16;
                // every B-slice fragment of this warp's 16 columns, once per product
                uint32_t bf[S][2][2][2];
#pragma unroll
                for (int u = 0; u < S; u++)
#pragma unroll
                    for (int nt = 0; nt < 2; nt++)
#pragma unroll
                        for (int ks = 0; ks < 2; ks++) {
                            if (ks < nks) {
                                const __nv_bfloat16* bb =
                                    sB + (u * SE_MAXB + wn * 16 + nt * 8 + g) * SE_RS + ks * 16 + 2 * q;
                                bf[u][nt][ks][0] = *reinterpret_cast<const uint32_t*>(bb);
                                bf[u][nt][ks][1] = *reinterpret_cast<const uint32_t*>(bb + 8);
                            }
                        }
#pragma unroll
                for (int t = 0; t < S; t++) {
                    uint32_t af[2][4];
#pragma unroll
                    for (int ks = 0; ks < 2; ks++) {
                        if (ks < nks) {
                            const __nv_bfloat16* base = sA + (t * SE_MAXB + wm * 16 + g) * SE_RS + ks * 16 + 2 * q;
                            af[ks][0] = *reinterpret_cast<const uint32_t*>(base);
                            af[ks][1] = *reinterpret_cast<const uint32_t*>(base + 8 * SE_RS);
                            af[ks][2] = *reinterpret_cast<const uint32_t*>(base + 8);
                            af[ks][3] = *reinterpret_cast<const uint32_t*>(base + 8 * SE_RS + 8);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < S - t; u++)
#pragma unroll
                        for (int nt = 0; nt < 2; nt++)
#pragma unroll
                            for (int ks = 0; ks < 2; ks++)
                                if (ks < nks) mma_bf16_16816(acc[t + u][nt], af[ks], bf[u][nt][ks]);
                }
            }
            __syncthreads();   // this buffer is refilled two products later
            if (++since == a.flush_every || p + 1 == p1) {
                since = 0;
#pragma unroll
                for (int d = 0; d < S; d++)
#pragma unroll
                    for (int nt = 0; nt < 2; nt++)
#pragma unroll
                        for (int r = 0; r < 4; r++) {
                            gi[d][nt][r] += __float2int_rn(acc[d][nt][r]);
                            acc[d][nt][r] = 0.f;
                        }
            }
        }
        cp_async_wait_group<0>();
        if (!active) continue;
        // FP64 recombination, then alpha / beta, into the column-major C block
        const int64_t rbase = a.croff[i], cbase = a.ccoff[j];
        double* cout = a.Cd + a.c_off[cb];
        const int old = a.c_old ? a.c_old[cb] : -1;
        const double* cold = (old >= 0) ? a.Cold + a.Cold_off[old] : nullptr;
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int row = wm * 16 + g + 8 * (r >> 1);
                const int colm = wn * 16 + nt * 8 + 2 * q + (r & 1);
                if (row < m && colm < n) {
                    __int128 Sx = 0;   // exact sum of the level sums, each shifted to its weight
#pragma unroll
                    for (int d = 0; d < S; d++) Sx += (__int128)gi[d][nt][r] << (7 * (S - 1 - d));
                    const double x = emul::recombined(Sx, a.e[rbase + row] + a.f[cbase + colm], 7 * (S + 1));
                    const int64_t eidx = (int64_t)colm * m + row;
                    cout[eidx] = cold ? bu.update(x, cold[eidx]) : bu.scale(x);
                }
            }
    }
}

// the largest product count of any C block
__global__ void k_max_span(int64_t nC, const int64_t* __restrict__ pstart, unsigned long long* out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < nC) atomicMax(out, (unsigned long long)(pstart[b + 1] - pstart[b]));
}

template <int S>
int launch_se(const SeArgs& a, int grid) {
    const int smem = 4 * S * SE_MAXB * SE_RS * (int)sizeof(__nv_bfloat16);   // two buffers of A + B
    DB_CUDA(cudaFuncSetAttribute(k_smm_emul<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_smm_emul<S><<<grid, SE_THREADS, smem, ctx().stream>>>(a);
    DB_KCHECK();
    return DBCSR_OK;
}

int slices_of(dbcsr_matrix_s* M, bool x_is_row, const int* ex, int s, DBuf<int64_t>& soff, int64_t* total,
              DBuf<__nv_bfloat16>& S) {
    cudaStream_t st = ctx().stream;
    const SliceGeom G = slice_geom(M, x_is_row);
    DB_TRY(soff.alloc(M->nblks + 1));
    if (M->nblks > 0) {
        k_se_slice_sizes<<<(unsigned)cdiv(M->nblks, 256), 256, 0, st>>>(G, soff.p);
        DB_KCHECK();
    }
    DBuf<int64_t> tot;
    DB_TRY(tot.alloc(1));
    DB_TRY(scan_i64(soff.p, soff.p, M->nblks, tot.p));
    DB_CUDA(cudaMemcpyAsync(soff.p + M->nblks, tot.p, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    DB_CUDA(cudaMemcpyAsync(total, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    DB_TRY(S.alloc((size_t)s * (*total > 0 ? *total : 1)));
    if (M->nblks > 0) {
        const int grid = (int)std::min<int64_t>(cdiv(M->nblks, 8), (int64_t)ctx().num_sms * 32);
        k_se_slice<<<grid, 256, 0, st>>>(G, ex, s, soff.p, *total, S.p);
        DB_KCHECK();
    }
    return DBCSR_OK;
}


}  // namespace

int line_exponents(dbcsr_matrix_s* M, bool x_is_row, int64_t nlines, DBuf<int>& ex) {
    cudaStream_t st = ctx().stream;
    const SliceGeom G = slice_geom(M, x_is_row);
    DBuf<unsigned long long> bits;
    DB_TRY(bits.alloc(nlines ? nlines : 1));
    DB_CUDA(cudaMemsetAsync(bits.p, 0, sizeof(unsigned long long) * (nlines ? nlines : 1), st));
    if (M->nblks > 0) {
        const int grid = (int)std::min<int64_t>(cdiv(M->nblks, 8), (int64_t)ctx().num_sms * 32);
        k_se_linemax<<<grid, 256, 0, st>>>(G, bits.p);
        DB_KCHECK();
    }
    DB_TRY(ex.alloc(nlines ? nlines : 1));
    if (nlines > 0) {
        k_se_exponents<<<(unsigned)cdiv(nlines, 256), 256, 0, st>>>(nlines, bits.p, ex.p);
        DB_KCHECK();
    }
    return DBCSR_OK;
}

int smm_emulated(const SmmArgs& g, dbcsr_matrix_s* A, bool ta, dbcsr_matrix_s* B, bool tb, dbcsr_matrix_s* C,
                 const dbcsr_opts& o, int64_t nprod, double* main_flops, const CRanges* ranges) {
    if (o.precision != DBCSR_PREC_OZAKI)
        return fail(DBCSR_ERR_ARG, "the stack path runs in FP64 or emulated FP64; TF32 needs the dense path");
    const int s = o.ozaki_slices > 0 ? o.ozaki_slices : 7;
    if (s > 8) return fail(DBCSR_ERR_ARG, "ozaki_slices must be 1..8");
    const int maxb = std::max(std::max(A->max_rs, A->max_cs), std::max(B->max_rs, B->max_cs));
    if (maxb > SE_MAXB)
        return fail(DBCSR_ERR_ARG, "emulated stack path: blocks larger than 32 need the dense path");
    if (g.nC == 0) return DBCSR_OK;
    cudaStream_t st = ctx().stream;
    // exactness budget of the int32 level sums
    DBuf<unsigned long long> span;
    DB_TRY(span.alloc(1));
    DB_CUDA(cudaMemsetAsync(span.p, 0, sizeof(unsigned long long), st));
    k_max_span<<<(unsigned)cdiv(g.nC, 256), 256, 0, st>>>(g.nC, g.c_pstart, span.p);
    DB_KCHECK();
    unsigned long long h_span = 0;
    DB_CUDA(cudaMemcpyAsync(&h_span, span.p, sizeof(h_span), cudaMemcpyDeviceToHost, st));
    DB_CUDA(cudaStreamSynchronize(st));
    const int kp = ru16(ta ? A->max_rs : A->max_cs);
    const double bound = (double)h_span * s * kp * 127.0 * 127.0;
    if (bound >= 2147483647.0)
        return fail(DBCSR_ERR_OVERFLOW, "emulated stack path: a C block has " + std::to_string(h_span) +
                                            " products, beyond the exact int32 budget; use the dense path");
    // exponents over the element rows of op(A) / columns of op(B)
    const int64_t Mop = C->h_roff[C->nbr], Nop = C->h_coff[C->nbc];
    DBuf<int> e, f;
    DB_TRY(line_exponents(A, !ta, Mop, e));
    DB_TRY(line_exponents(B, tb, Nop, f));
    // kernel: 0 = tcgen05 when the mean block edge is at least 12, else
    // mma.sync; 1 = mma.sync; 2 = tcgen05. Measured on GB300: 22 x 22 blocks
    // padded to 32 x 32 run 5.8x faster on tcgen05, the mixed 5..32 blocks of
    // the uneven workload (mean edge 17.9) 1.18x faster; the mma.sync kernel
    // pads to 16 instead of 32, which pays only for small blocks
    double esum = 0.0;
    int64_t ecount = 0;
    for (const std::vector<int>* v : {&A->h_rs, &A->h_cs, &B->h_rs, &B->h_cs}) {
        for (int x : *v) esum += x;
        ecount += (int64_t)v->size();
    }
    const bool tc_ok = smm_emul_tc_usable();
    if (o.kernel == 2 && !tc_ok) return fail(DBCSR_ERR_STATE, "tcgen05 emulated stack kernel unavailable");
    if (o.kernel == 2 || (o.kernel == 0 && ecount > 0 && esum >= 12.0 * (double)ecount && tc_ok))
        return smm_emul_tc(g, A, ta, B, tb, C, e.p, f.p, s, nprod, main_flops, ranges);
    DBuf<int64_t> soffA, soffB;
    DBuf<__nv_bfloat16> SA, SB;
    int64_t totA = 0, totB = 0;
    DB_TRY(slices_of(A, !ta, e.p, s, soffA, &totA, SA));
    DB_TRY(slices_of(B, tb, f.p, s, soffB, &totB, SB));
    SeArgs a;
    a.nC = g.nC;
    a.c_row = g.c_row;
    a.c_col = g.c_col;
    a.c_off = g.c_off;
    a.c_old = g.c_old;
    a.c_pstart = g.c_pstart;
    a.prod = g.prod;
    a.a_off = A->d_off;
    a.rsC = g.rsC;
    a.csC = g.csC;
    a.croff = C->d_roff;
    a.ccoff = C->d_coff;
    a.e = e.p;
    a.f = f.p;
    a.SA = SA.p;
    a.SB = SB.p;
    a.totA = totA;
    a.totB = totB;
    a.soffA = soffA.p;
    a.soffB = soffB.p;
    a.Cd = g.Cd;
    a.Cold = g.Cold;
    a.Cold_off = g.Cold_off;
    a.alpha = g.alpha;
    a.beta = g.beta;
    a.flush_every = std::max(1, 1040 / (s * kp));
    a.counter = g.counter;
    // one launch per C-block range (all C blocks when no ranges are given)
    const CRanges all{{0, g.nC}};
    const CRanges& rr = ranges ? *ranges : all;
    int rc = DBCSR_OK;
    timer_kernel_begin();
    for (const auto& r : rr) {
        if (r.second <= r.first) continue;
        SeArgs ar = a;
        ar.nC = r.second - r.first;
        ar.c_row += r.first;
        ar.c_col += r.first;
        ar.c_off += r.first;
        if (ar.c_old) ar.c_old += r.first;
        ar.c_pstart += r.first;
        DB_CUDA(cudaMemsetAsync(ar.counter, 0, sizeof(unsigned long long), st));
        int grid = ctx().num_sms * 4;
        if (grid > ar.nC) grid = (int)ar.nC;
        switch (s) {
            case 1: rc = launch_se<1>(ar, grid); break;
            case 2: rc = launch_se<2>(ar, grid); break;
            case 3: rc = launch_se<3>(ar, grid); break;
            case 4: rc = launch_se<4>(ar, grid); break;
            case 5: rc = launch_se<5>(ar, grid); break;
            case 6: rc = launch_se<6>(ar, grid); break;
            case 7: rc = launch_se<7>(ar, grid); break;
            default: rc = launch_se<8>(ar, grid); break;
        }
        if (rc) break;
    }
    timer_kernel_end();
    if (rc) return rc;
    if (main_flops)   // MMA work issued: every pair t + u <= s + 1 on shapes padded to 16
        *main_flops = (double)nprod * (s * (s + 1) / 2) * 2.0 * ru16(C->max_rs) * ru16(C->max_cs) * kp;
    return DBCSR_OK;
}

}  // namespace dbcsr
