// prims.cu -- device-wide prefix sums and a stable LSD radix sort.
//
// These are the "prefix sums" and "radix sort by shape" building blocks of
// stack generation (the paper's Generation phase, Sec. II, organises block
// products into batches of one (m,n,k) kind). Both are hand-written: a
// reduce-then-scan over tiles of 4096 elements, and an 8-bit-digit LSD radix
// sort whose scatter ranks equal digits in input order (stable), so that a
// sort by shape keeps the (i, j, k) order that stack generation produced.
#include "internal.cuh"

namespace dbcsr {

namespace {

constexpr int SC_NT = 512;
constexpr int SC_IPT = 8;
constexpr int SC_TILE = SC_NT * SC_IPT;

template <class T>
__device__ T warp_incl_scan(T x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread across the block; *total = block sum.
template <class T, int NT>
__device__ T block_excl_scan(T v, T* total, T* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = warp_incl_scan(v, lane);
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        T s = (lane < NT / 32) ? sh[lane] : T(0);
        s = warp_incl_scan(s, lane);
        if (lane < NT / 32) sh[lane] = s;
    }
    __syncthreads();
    T base = (w > 0) ? sh[w - 1] : T(0);
    *total = sh[NT / 32 - 1];
    __syncthreads();
    return base + x - v;
}

template <class Tin>
__global__ void k_tile_reduce(const Tin* __restrict__ in, int64_t n, int64_t* __restrict__ part) {
    __shared__ int64_t sh[SC_NT / 32];
    int64_t base = (int64_t)blockIdx.x * SC_TILE;
    int64_t s = 0;
    for (int i = threadIdx.x; i < SC_TILE; i += SC_NT) {
        int64_t g = base + i;
        if (g < n) s += (int64_t)in[g];
    }
    int64_t tot;
    block_excl_scan<int64_t, SC_NT>(s, &tot, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Scan one tile: thread t owns SC_IPT consecutive elements.
template <class Tin, class Tout>
__global__ void k_tile_scan(const Tin* in, Tout* out, int64_t n, const int64_t* __restrict__ part_excl,
                            int64_t* d_total) {
    __shared__ int64_t sh[SC_NT / 32];
    int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_IPT;
    int64_t v[SC_IPT];
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < SC_IPT; q++) {
        int64_t g = base + q;
        v[q] = (g < n) ? (int64_t)in[g] : 0;
        s += v[q];
    }
    int64_t tot;
    int64_t ex = block_excl_scan<int64_t, SC_NT>(s, &tot, sh);
    int64_t off = (part_excl ? part_excl[blockIdx.x] : 0) + ex;
#pragma unroll
    for (int q = 0; q < SC_IPT; q++) {
        int64_t g = base + q;
        if (g < n) out[g] = (Tout)off;
        off += v[q];
    }
    if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *d_total = (part_excl ? part_excl[blockIdx.x] : 0) + tot;
}

template <class Tin, class Tout>
int scan_impl(const Tin* in, Tout* out, int64_t n, int64_t* d_total) {
    cudaStream_t st = ctx().stream;
    if (n <= 0) {
        if (d_total) DB_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int64_t), st));
        return DBCSR_OK;
    }
    int64_t ntiles = cdiv(n, SC_TILE);
    if (ntiles == 1) {
        k_tile_scan<Tin, Tout><<<1, SC_NT, 0, st>>>(in, out, n, nullptr, d_total);
        DB_KCHECK();
        return DBCSR_OK;
    }
    DBuf<int64_t> part;
    DB_TRY(part.alloc(ntiles));
    k_tile_reduce<Tin><<<(unsigned)ntiles, SC_NT, 0, st>>>(in, n, part.p);
    DB_KCHECK();
    DB_TRY((scan_impl<int64_t, int64_t>(part.p, part.p, ntiles, nullptr)));
    k_tile_scan<Tin, Tout><<<(unsigned)ntiles, SC_NT, 0, st>>>(in, out, n, part.p, d_total);
    DB_KCHECK();
    return DBCSR_OK;
}

// ------------------------------------------------------------ radix sort
constexpr int RS_NT = 256;     // = number of digit values (8-bit digits)
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_NT * RS_IPT;
constexpr int RS_WARPS = RS_NT / 32;

__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int64_t ntiles,
                          int* __restrict__ hist) {
    __shared__ int h[RS_NT];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_NT) {
        int64_t g = base + i;
        if (g < n) atomicAdd(&h[(keys[g] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                             int shift, int64_t ntiles, const int* __restrict__ offs) {
    __shared__ int base[RS_NT];
    __shared__ int wcnt[RS_WARPS][RS_NT];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
    for (int q = 0; q < RS_WARPS; q++) wcnt[q][tid] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_IPT; r++) {
        int64_t g = t0 + (int64_t)r * RS_NT + tid;
        bool valid = g < n;
        uint32_t key = valid ? kin[g] : 0u;
        uint32_t val = valid ? vin[g] : 0u;
        uint32_t dig = valid ? ((key >> shift) & 255u) : 0xffffffffu;
        uint32_t peers = __match_any_sync(0xffffffffu, dig);
        int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[w][dig] = __popc(peers);
        __syncthreads();
        {   // thread `tid` owns digit `tid`: exclusive prefix over warps
            int run = base[tid];
#pragma unroll
            for (int q = 0; q < RS_WARPS; q++) {
                int c = wcnt[q][tid];
                wcnt[q][tid] = run;
                run += c;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int pos = wcnt[w][dig] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RS_WARPS; q++) wcnt[q][tid] = 0;
        __syncthreads();
    }
}

}  // namespace

int scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* d_total) {
    return scan_impl<int64_t, int64_t>(in, out, n, d_total);
}

int scan_i32(const int* in, int* out, int64_t n, int64_t* d_total) {
    return scan_impl<int, int>(in, out, n, d_total);
}

int radix_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n, int bits) {
    if (n <= 1 || bits <= 0) return DBCSR_OK;
    if (n >= (int64_t)INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "radix sort: too many items");
    cudaStream_t st = ctx().stream;
    int64_t ntiles = cdiv(n, RS_TILE);
    DBuf<uint32_t> k2, v2;
    DBuf<int> hist;
    DB_TRY(k2.alloc(n));
    DB_TRY(v2.alloc(n));
    DB_TRY(hist.alloc(ntiles * RS_NT));
    uint32_t *ka = keys, *va = vals, *kb = k2.p, *vb = v2.p;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, passes++) {
        k_rs_hist<<<(unsigned)ntiles, RS_NT, 0, st>>>(ka, n, shift, ntiles, hist.p);
        DB_KCHECK();
        DB_TRY(scan_i32(hist.p, hist.p, ntiles * RS_NT, nullptr));
        k_rs_scatter<<<(unsigned)ntiles, RS_NT, 0, st>>>(ka, va, kb, vb, n, shift, ntiles, hist.p);
        DB_KCHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {
        DB_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        DB_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    return DBCSR_OK;
}

}  // namespace dbcsr
