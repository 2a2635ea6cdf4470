// api.cu -- the C ABI (include/dbcsr_gb.h): context, allocator, matrix
// create/release/query and the multiply driver.
//
// The multiply follows the paper's local multiplication (Sec. II): build the
// stacks of block products, execute them with batched small-GEMM kernels, or
// take the densified path of Sec. III when both operands are dense.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <unordered_map>

#include "internal.cuh"
#include "dense.cuh"
#include "emul.cuh"
#include "smm.cuh"
#include "smm_emul.cuh"
#include "stackgen.cuh"

namespace dbcsr {

namespace {
thread_local std::string g_last_error;
thread_local dbcsr_stats g_stats;
std::atomic<int64_t> g_launches{0};
std::atomic<uint64_t> g_uid{1};
Context g_ctx;
std::mutex g_init_mutex;
// allocations made through caller hooks, so each is returned to the hook that made it
struct HookAlloc {
    dbcsr_free_fn free;
    void* ctx;
};
std::unordered_map<void*, HookAlloc> g_hook_allocs;
std::mutex g_hook_mutex;
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
Context& ctx() { return g_ctx; }

int ensure_device() {
    if (g_ctx.device >= 0) return DBCSR_OK;
    std::lock_guard<std::mutex> lk(g_init_mutex);
    if (g_ctx.device >= 0) return DBCSR_OK;
    int dev = 0;
    DB_CUDA(cudaGetDevice(&dev));
    int sms = 0;
    DB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaMemPool_t pool;
    DB_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t thr = UINT64_MAX;   // keep freed blocks in the pool (memory-pool buffers, Sec. III)
    DB_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    g_ctx.num_sms = sms;
    cudaError_t e = cudaMalloc(&g_ctx.d_flags, 64 * sizeof(int));
    if (e != cudaSuccess) return fail(DBCSR_ERR_ALLOC, std::string("flag buffer: ") + cudaGetErrorString(e));
    DB_CUDA(cudaStreamCreateWithFlags(&g_ctx.xfer, cudaStreamNonBlocking));
    DB_CUDA(cudaEventCreateWithFlags(&g_ctx.order_ev, cudaEventDisableTiming));
    g_ctx.device = dev;
    return DBCSR_OK;
}

int dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (g_ctx.alloc) {
        *p = g_ctx.alloc(bytes, (void*)g_ctx.stream, g_ctx.alloc_ctx);
        if (!*p) return fail(DBCSR_ERR_ALLOC, "allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
        std::lock_guard<std::mutex> lk(g_hook_mutex);
        g_hook_allocs[*p] = HookAlloc{g_ctx.free, g_ctx.alloc_ctx};
        return DBCSR_OK;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, g_ctx.stream);
    if (e != cudaSuccess || !*p) {
        cudaGetLastError();
        *p = nullptr;
        return fail(DBCSR_ERR_ALLOC, std::string("device allocation of ") + std::to_string(bytes) +
                                         " bytes failed: " + cudaGetErrorString(e));
    }
    return DBCSR_OK;
}

void dev_free(void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    HookAlloc h{nullptr, nullptr};
    {
        std::lock_guard<std::mutex> lk(g_hook_mutex);
        auto it = g_hook_allocs.find(p);
        if (it != g_hook_allocs.end()) {
            h = it->second;
            g_hook_allocs.erase(it);
        }
    }
    if (h.free) {
        h.free(p, bytes, (void*)g_ctx.stream, h.ctx);
        return;
    }
    cudaFreeAsync(p, g_ctx.stream);
}

int h2d(void* dst, const void* src, size_t bytes) {
    if (bytes) DB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, g_ctx.stream));
    return DBCSR_OK;
}
int d2h(void* dst, const void* src, size_t bytes) {
    if (bytes) DB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, g_ctx.stream));
    return DBCSR_OK;
}
int sync_stream() {
    DB_CUDA(cudaStreamSynchronize(g_ctx.stream));
    return DBCSR_OK;
}

int await_data(dbcsr_matrix_s* m) {
    if (m && m->pending) {
        DB_CUDA(cudaStreamWaitEvent(g_ctx.stream, m->ready, 0));
        m->pending = false;
    }
    return DBCSR_OK;
}

// Copy n host values into m->d_data. From page-locked memory the copy runs
// on the transfer stream, after everything the library stream has queued so
// far (the allocation of d_data, earlier reads of it), and the library stream
// waits for it at the next use of m. From pageable memory, which the copy
// engine cannot read directly, it is done on the library stream before the
// call returns.
int upload_data(dbcsr_matrix_s* m, const double* data, int64_t n) {
    DB_TRY(await_data(m));
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, data) != cudaSuccess || at.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        DB_CUDA(cudaMemcpyAsync(m->d_data, data, sizeof(double) * n, cudaMemcpyHostToDevice, g_ctx.stream));
        return sync_stream();
    }
    if (!m->ready) DB_CUDA(cudaEventCreateWithFlags(&m->ready, cudaEventDisableTiming));
    DB_CUDA(cudaEventRecord(g_ctx.order_ev, g_ctx.stream));
    DB_CUDA(cudaStreamWaitEvent(g_ctx.xfer, g_ctx.order_ev, 0));
    DB_CUDA(cudaMemcpyAsync(m->d_data, data, sizeof(double) * n, cudaMemcpyHostToDevice, g_ctx.xfer));
    DB_CUDA(cudaEventRecord(m->ready, g_ctx.xfer));
    m->pending = true;
    return DBCSR_OK;
}

void free_index(dbcsr_matrix_s* m) {
    await_data(m);   // a pending upload finishes before its target is freed
    dfree(m->d_rowptr, (size_t)m->nbr + 1);
    dfree(m->d_col, (size_t)(m->nblks ? m->nblks : 1));
    dfree(m->d_row_of, (size_t)(m->nblks ? m->nblks : 1));
    dfree(m->d_off, (size_t)m->nblks + 1);
    dfree(m->d_data, (size_t)(m->nelems ? m->nelems : 1));
    dfree(m->d_tptr, (size_t)m->nbc + 1);
    dfree(m->d_tidx, (size_t)(m->nblks ? m->nblks : 1));
    dfree(m->d_tpos, (size_t)(m->nblks ? m->nblks : 1));
    m->t_valid = false;
    m->h_valid = false;
}

int download_index(dbcsr_matrix_s* m) {
    if (m->h_valid) return DBCSR_OK;
    m->h_rowptr.resize(m->nbr + 1);
    m->h_col.resize(m->nblks);
    m->h_off.resize(m->nblks + 1);
    DB_TRY(d2h(m->h_rowptr.data(), m->d_rowptr, sizeof(int) * (m->nbr + 1)));
    DB_TRY(d2h(m->h_col.data(), m->d_col, sizeof(int) * m->nblks));
    DB_TRY(d2h(m->h_off.data(), m->d_off, sizeof(int64_t) * (m->nblks + 1)));
    DB_TRY(sync_stream());
    m->h_row_cs.assign(m->nbr, 0.0);
    m->h_row_n.assign(m->nbr, 0);
    m->h_col_rs.assign(m->nbc, 0.0);
    m->h_col_n.assign(m->nbc, 0);
    for (int i = 0; i < m->nbr; i++)
        for (int q = m->h_rowptr[i]; q < m->h_rowptr[i + 1]; q++) {
            const int j = m->h_col[q];
            m->h_row_cs[i] += m->h_cs[j];
            m->h_row_n[i]++;
            m->h_col_rs[j] += m->h_rs[i];
            m->h_col_n[j]++;
        }
    m->h_valid = true;
    return DBCSR_OK;
}

namespace {

bool is_trans(char t) { return t == 'T' || t == 't' || t == 'C' || t == 'c'; }
bool valid_trans(char t) { return t == 'N' || t == 'n' || is_trans(t); }

__global__ void k_gather_blocks(int64_t nblks, const int64_t* __restrict__ src_off,
                                const int64_t* __restrict__ dst_off, const double* __restrict__ src,
                                double* __restrict__ dst) {
    for (int64_t b = blockIdx.x; b < nblks; b += gridDim.x) {
        const int64_t s = src_off[b], d = dst_off[b], n = dst_off[b + 1] - d;
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) dst[d + e] = src[s + e];
    }
}

// set sizes + offsets (host and device) of a new matrix
int setup_sizes(dbcsr_matrix_s* m, int nbr, int nbc, const int* rs, const int* cs) {
    m->nbr = nbr;
    m->nbc = nbc;
    m->h_rs.assign(rs, rs + nbr);
    m->h_cs.assign(cs, cs + nbc);
    m->h_roff.assign(nbr + 1, 0);
    m->h_coff.assign(nbc + 1, 0);
    for (int i = 0; i < nbr; i++) m->h_roff[i + 1] = m->h_roff[i] + rs[i];
    for (int j = 0; j < nbc; j++) m->h_coff[j + 1] = m->h_coff[j] + cs[j];
    m->max_rs = nbr ? *std::max_element(rs, rs + nbr) : 0;
    m->max_cs = nbc ? *std::max_element(cs, cs + nbc) : 0;
    for (auto* u : {&m->u_rs, &m->u_cs}) {
        *u = (u == &m->u_rs) ? m->h_rs : m->h_cs;
        std::sort(u->begin(), u->end());
        u->erase(std::unique(u->begin(), u->end()), u->end());
    }
    DB_TRY(dalloc(&m->d_rs, (size_t)nbr + 1));
    DB_TRY(dalloc(&m->d_cs, (size_t)nbc + 1));
    DB_TRY(dalloc(&m->d_roff, (size_t)nbr + 1));
    DB_TRY(dalloc(&m->d_coff, (size_t)nbc + 1));
    DB_TRY(h2d(m->d_rs, rs, sizeof(int) * nbr));
    DB_TRY(h2d(m->d_cs, cs, sizeof(int) * nbc));
    DB_TRY(h2d(m->d_roff, m->h_roff.data(), sizeof(int64_t) * (nbr + 1)));
    DB_TRY(h2d(m->d_coff, m->h_coff.data(), sizeof(int64_t) * (nbc + 1)));
    return DBCSR_OK;
}

// A kept stack plan: the product list of one multiply and a CUDA graph of its
// FP64 product kernel, replayed in place on the C it produced while the
// operands' patterns (uid + version) and the scalars are unchanged.
struct ReusePlan {
    uint64_t a_uid = 0, a_ver = 0, b_uid = 0, b_ver = 0, c_ver = 0;
    bool ta = false, tb = false, use_old = false;
    double alpha = 0.0, beta = 0.0;
    int64_t nC = 0, nprod = 0;
    int64_t* c_pstart = nullptr;
    int2* prod = nullptr;
    int* c_ident = nullptr;          // identity map: block b of C is its own old block
    unsigned long long* counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~ReusePlan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        dfree(c_pstart, (size_t)nC + 1);
        dfree(prod, (size_t)(nprod ? nprod : 1));
        dfree(c_ident, (size_t)(nC ? nC : 1));
        dfree(counter, 1);
    }
};

void free_plan(dbcsr_matrix_s* m) {
    delete static_cast<ReusePlan*>(m->plan);
    m->plan = nullptr;
}

void destroy(dbcsr_matrix_s* m) {
    if (!m) return;
    // a copy from the caller's page-locked memory still in flight: the caller
    // may free that memory once the matrix is released
    if (m->pending) cudaEventSynchronize(m->ready);
    free_plan(m);
    free_index(m);
    dfree(m->d_rs, (size_t)m->nbr + 1);
    dfree(m->d_cs, (size_t)m->nbc + 1);
    dfree(m->d_roff, (size_t)m->nbr + 1);
    dfree(m->d_coff, (size_t)m->nbc + 1);
    if (m->ready) cudaEventDestroy(m->ready);
    delete m;
}

// Install a new index + data into m (takes ownership of the device arrays).
void install(dbcsr_matrix_s* m, int64_t nblks, int64_t nelems, int* rowptr, int* col, int* row_of, int64_t* off,
             double* data) {
    free_index(m);
    m->nblks = nblks;
    m->nelems = nelems;
    m->d_rowptr = rowptr;
    m->d_col = col;
    m->d_row_of = row_of;
    m->d_off = off;
    m->d_data = data;
    m->version++;
}

}  // namespace
}  // namespace dbcsr

using namespace dbcsr;

extern "C" {

const char* dbcsr_last_error(void) { return g_last_error.c_str(); }
const char* dbcsr_version(void) { return "dbcsr-gb300 0.1 (sm_103a)"; }

int dbcsr_init(void* cuda_stream) {
    g_last_error.clear();
    DB_TRY(ensure_device());
    g_ctx.stream = (cudaStream_t)cuda_stream;
    return DBCSR_OK;
}

int dbcsr_set_allocator(dbcsr_alloc_fn alloc, dbcsr_free_fn free_fn, void* actx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(DBCSR_ERR_ARG, "set_allocator: alloc and free must both be set or both be NULL");
    g_ctx.alloc = alloc;
    g_ctx.free = free_fn;
    g_ctx.alloc_ctx = actx;
    return DBCSR_OK;
}

int dbcsr_sync(void) {
    if (g_ctx.xfer) DB_CUDA(cudaStreamSynchronize(g_ctx.xfer));
    return sync_stream();
}

int dbcsr_create(dbcsr_matrix* out, int nbr, int nbc, const int* rs, const int* cs, int64_t nblks,
                 const int* br, const int* bc, const double* data, int data_on_device) {
    g_last_error.clear();
    if (!out) return fail(DBCSR_ERR_ARG, "create: out is NULL");
    *out = nullptr;
    if (nbr < 0 || nbc < 0 || nblks < 0) return fail(DBCSR_ERR_ARG, "create: negative size");
    if ((nbr > 0 && !rs) || (nbc > 0 && !cs)) return fail(DBCSR_ERR_ARG, "create: block size array is NULL");
    if (nblks > 0 && (!br || !bc)) return fail(DBCSR_ERR_ARG, "create: block index array is NULL");
    if (nblks >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "create: too many blocks");
    for (int i = 0; i < nbr; i++)
        if (rs[i] < 1) return fail(DBCSR_ERR_ARG, "create: row block size < 1 at " + std::to_string(i));
    for (int j = 0; j < nbc; j++)
        if (cs[j] < 1) return fail(DBCSR_ERR_ARG, "create: col block size < 1 at " + std::to_string(j));
    // coordinates in range, and whether the blocks already come in CSR order
    // (row, then column, no duplicates) -- one pass
    bool sorted = true;
    for (int64_t b = 0; b < nblks; b++) {
        if (br[b] < 0 || br[b] >= nbr || bc[b] < 0 || bc[b] >= nbc)
            return fail(DBCSR_ERR_ARG, "create: block coordinate out of range at " + std::to_string(b));
        if (b > 0 && (br[b] < br[b - 1] || (br[b] == br[b - 1] && bc[b] <= bc[b - 1]))) sorted = false;
    }
    DB_TRY(ensure_device());

    // CSR order of the blocks (row, then column), duplicates rejected
    std::vector<int64_t> perm;
    if (!sorted) {
        perm.resize(nblks);
        std::iota(perm.begin(), perm.end(), 0);
        std::stable_sort(perm.begin(), perm.end(), [&](int64_t x, int64_t y) {
            return br[x] != br[y] ? br[x] < br[y] : bc[x] < bc[y];
        });
        for (int64_t q = 1; q < nblks; q++)
            if (br[perm[q]] == br[perm[q - 1]] && bc[perm[q]] == bc[perm[q - 1]])
                return fail(DBCSR_ERR_ARG, "create: duplicate block (" + std::to_string(br[perm[q]]) + "," +
                                               std::to_string(bc[perm[q]]) + ")");
    }
    auto* m = new dbcsr_matrix_s();
    m->uid = g_uid.fetch_add(1);
    int rc = setup_sizes(m, nbr, nbc, rs, cs);
    if (rc) { destroy(m); return rc; }
    // host index in CSR order
    std::vector<int> rowptr(nbr + 1, 0), col(nblks), row_of(nblks);
    std::vector<int64_t> off(nblks + 1, 0), src_off;
    for (int64_t q = 0; q < nblks; q++) {
        const int64_t b = sorted ? q : perm[q];
        rowptr[br[b] + 1]++;
        col[q] = bc[b];
        row_of[q] = br[b];
        off[q + 1] = off[q] + (int64_t)rs[br[b]] * cs[bc[b]];
    }
    for (int i = 0; i < nbr; i++) rowptr[i + 1] += rowptr[i];
    const int64_t nelems = off[nblks];
    int *d_rowptr = nullptr, *d_col = nullptr, *d_row_of = nullptr;
    int64_t* d_off = nullptr;
    double* d_data = nullptr;
    if ((rc = dalloc(&d_rowptr, (size_t)nbr + 1)) || (rc = dalloc(&d_col, (size_t)(nblks ? nblks : 1))) ||
        (rc = dalloc(&d_row_of, (size_t)(nblks ? nblks : 1))) || (rc = dalloc(&d_off, (size_t)nblks + 1)) ||
        (rc = dalloc(&d_data, (size_t)(nelems ? nelems : 1)))) {
        dfree(d_rowptr, nbr + 1); dfree(d_col, 1); dfree(d_row_of, 1); dfree(d_off, 1); dfree(d_data, 1);
        destroy(m);
        return rc;
    }
    install(m, nblks, nelems, d_rowptr, d_col, d_row_of, d_off, d_data);
    if ((rc = h2d(d_rowptr, rowptr.data(), sizeof(int) * (nbr + 1))) ||
        (rc = h2d(d_col, col.data(), sizeof(int) * nblks)) ||
        (rc = h2d(d_row_of, row_of.data(), sizeof(int) * nblks)) ||
        (rc = h2d(d_off, off.data(), sizeof(int64_t) * (nblks + 1)))) {
        destroy(m);
        return rc;
    }
    if (!data) {
        if (nelems) {
            cudaError_t e = cudaMemsetAsync(d_data, 0, sizeof(double) * nelems, g_ctx.stream);
            if (e != cudaSuccess) { destroy(m); return fail(DBCSR_ERR_CUDA, cudaGetErrorString(e)); }
        }
    } else if (sorted && !data_on_device) {
        // host values on the transfer stream: the call returns while they copy
        if ((rc = upload_data(m, data, nelems))) { destroy(m); return rc; }
    } else if (sorted) {
        cudaError_t e = cudaMemcpyAsync(d_data, data, sizeof(double) * nelems, cudaMemcpyDeviceToDevice,
                                        g_ctx.stream);
        if (e != cudaSuccess) { destroy(m); return fail(DBCSR_ERR_CUDA, cudaGetErrorString(e)); }
    } else {
        // offsets of the blocks in the caller's order, gathered into CSR order
        std::vector<int64_t> in_off(nblks + 1, 0);
        for (int64_t b = 0; b < nblks; b++) in_off[b + 1] = in_off[b] + (int64_t)rs[br[b]] * cs[bc[b]];
        if (!data_on_device) {
            std::vector<double> tmp(nelems);
            for (int64_t q = 0; q < nblks; q++) {
                int64_t b = perm[q];
                std::memcpy(tmp.data() + off[q], data + in_off[b], sizeof(double) * (off[q + 1] - off[q]));
            }
            if ((rc = h2d(d_data, tmp.data(), sizeof(double) * nelems)) || (rc = sync_stream())) {
                destroy(m);
                return rc;
            }
        } else {
            std::vector<int64_t> soff(nblks);
            for (int64_t q = 0; q < nblks; q++) soff[q] = in_off[perm[q]];
            DBuf<int64_t> d_soff;
            if ((rc = d_soff.alloc(nblks)) || (rc = h2d(d_soff.p, soff.data(), sizeof(int64_t) * nblks))) {
                destroy(m);
                return rc;
            }
            int grid = (int)std::min<int64_t>(nblks, (int64_t)g_ctx.num_sms * 16);
            k_gather_blocks<<<grid, 256, 0, g_ctx.stream>>>(nblks, d_soff.p, d_off, data, d_data);
            count_launch();
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { destroy(m); return fail(DBCSR_ERR_CUDA, cudaGetErrorString(e)); }
            if ((rc = sync_stream())) { destroy(m); return rc; }
        }
    }
    // host vectors above are sources of async copies: finish before they go
    if ((rc = sync_stream())) { destroy(m); return rc; }
    *out = m;
    return DBCSR_OK;
}

int dbcsr_release(dbcsr_matrix* m) {
    if (!m || !*m) return DBCSR_OK;
    destroy(*m);
    *m = nullptr;
    return DBCSR_OK;
}

int dbcsr_get_info(dbcsr_matrix m, int* nbr, int* nbc, int64_t* nblks, int64_t* nelems) {
    if (!m) return fail(DBCSR_ERR_ARG, "get_info: NULL matrix");
    if (nbr) *nbr = m->nbr;
    if (nbc) *nbc = m->nbc;
    if (nblks) *nblks = m->nblks;
    if (nelems) *nelems = m->nelems;
    return DBCSR_OK;
}

int dbcsr_get_index(dbcsr_matrix m, int* br, int* bc, int64_t* off) {
    if (!m) return fail(DBCSR_ERR_ARG, "get_index: NULL matrix");
    DB_TRY(download_index(m));
    for (int i = 0; i < m->nbr; i++)
        for (int q = m->h_rowptr[i]; q < m->h_rowptr[i + 1]; q++) {
            if (br) br[q] = i;
            if (bc) bc[q] = m->h_col[q];
            if (off) off[q] = m->h_off[q];
        }
    return DBCSR_OK;
}

int dbcsr_get_data(dbcsr_matrix m, double* out, int out_on_device) {
    if (!m || (!out && m->nelems)) return fail(DBCSR_ERR_ARG, "get_data: NULL argument");
    if (m->nelems == 0) return DBCSR_OK;
    DB_TRY(await_data(m));
    DB_CUDA(cudaMemcpyAsync(out, m->d_data, sizeof(double) * m->nelems,
                            out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g_ctx.stream));
    if (!out_on_device) DB_TRY(sync_stream());
    return DBCSR_OK;
}

int dbcsr_set_data(dbcsr_matrix m, const double* data, int data_on_device) {
    if (!m || (!data && m->nelems)) return fail(DBCSR_ERR_ARG, "set_data: NULL argument");
    if (m->nelems == 0) return DBCSR_OK;
    if (!data_on_device) return upload_data(m, data, m->nelems);
    DB_TRY(await_data(m));
    DB_CUDA(cudaMemcpyAsync(m->d_data, data, sizeof(double) * m->nelems, cudaMemcpyDeviceToDevice, g_ctx.stream));
    DB_TRY(sync_stream());
    return DBCSR_OK;
}

int dbcsr_data_ptr(dbcsr_matrix m, double** p) {
    if (!m || !p) return fail(DBCSR_ERR_ARG, "data_ptr: NULL argument");
    if (m->pending) {   // the caller may read the values on any stream: the upload completes first
        DB_CUDA(cudaEventSynchronize(m->ready));
        m->pending = false;
    }
    *p = m->d_data;
    return DBCSR_OK;
}

int dbcsr_get_block(dbcsr_matrix m, int row, int col, double* out, int* found) {
    if (!m || !found) return fail(DBCSR_ERR_ARG, "get_block: NULL argument");
    *found = 0;
    if (row < 0 || row >= m->nbr || col < 0 || col >= m->nbc)
        return fail(DBCSR_ERR_ARG, "get_block: coordinates outside the block grid");
    DB_TRY(download_index(m));
    const int* b = m->h_col.data() + m->h_rowptr[row];
    const int* e = m->h_col.data() + m->h_rowptr[row + 1];
    const int* it = std::lower_bound(b, e, col);
    if (it == e || *it != col) return DBCSR_OK;
    int64_t q = it - m->h_col.data();
    if (!out) return fail(DBCSR_ERR_ARG, "get_block: out is NULL");
    DB_TRY(await_data(m));
    DB_TRY(d2h(out, m->d_data + m->h_off[q], sizeof(double) * (m->h_off[q + 1] - m->h_off[q])));
    DB_TRY(sync_stream());
    *found = 1;
    return DBCSR_OK;
}

int dbcsr_set_tuning(const int* m, const int* n, const int* variant, int count) {
    if (count < 0 || (count > 0 && (!m || !n || !variant))) return fail(DBCSR_ERR_ARG, "set_tuning: bad arguments");
    return smm_set_table(m, n, variant, count);
}

int dbcsr_set_tuning_mnk(const int* m, const int* n, const int* k, const int* variant, int count) {
    if (count < 0 || (count > 0 && (!m || !n || !k || !variant)))
        return fail(DBCSR_ERR_ARG, "set_tuning_mnk: bad arguments");
    return smm_set_table_mnk(m, n, k, variant, count);
}

int dbcsr_get_stats(dbcsr_stats* out) {
    if (!out) return fail(DBCSR_ERR_ARG, "get_stats: NULL");
    *out = g_stats;
    return DBCSR_OK;
}

}  // extern "C"

namespace dbcsr {
namespace {

// CUDA events on the library stream around the phases of one multiply
struct PhaseTimer {
    bool on = false;
    bool kernel_marked = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void init(bool enable) {
        on = enable;
        if (!on) return;
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) on = false;
    }
    void mark(int i) {
        if (on) cudaEventRecord(ev[i], g_ctx.stream);
        if (on && i == 5) kernel_marked = true;
    }
    void finish(dbcsr_stats& s) {
        if (!on) return;
        cudaEventSynchronize(ev[3]);
        cudaEventElapsedTime(&s.ms_setup, ev[0], ev[1]);
        cudaEventElapsedTime(&s.ms_main, ev[1], ev[2]);
        cudaEventElapsedTime(&s.ms_finish, ev[2], ev[3]);
        cudaEventElapsedTime(&s.ms_total, ev[0], ev[3]);
        if (kernel_marked) cudaEventElapsedTime(&s.ms_kernel, ev[4], ev[5]);
        else s.ms_kernel = s.ms_main;
    }
    ~PhaseTimer() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};
PhaseTimer* g_timer = nullptr;
inline void mark(int i) {
    if (g_timer) g_timer->mark(i);
}

}  // namespace

// around the dominant kernel of a multiply (events 4 and 5 of the phase timer)
void timer_kernel_begin() { mark(4); }
void timer_kernel_end() { mark(5); }

namespace {

int check_conformant(bool ta, bool tb, dbcsr_matrix_s* A, dbcsr_matrix_s* B, dbcsr_matrix_s* C) {
    const std::vector<int>& a_rows = ta ? A->h_cs : A->h_rs;
    const std::vector<int>& a_cols = ta ? A->h_rs : A->h_cs;
    const std::vector<int>& b_rows = tb ? B->h_cs : B->h_rs;
    const std::vector<int>& b_cols = tb ? B->h_rs : B->h_cs;
    if (a_cols.size() != b_rows.size())
        return fail(DBCSR_ERR_DIM, "multiply: inner block grids differ (" + std::to_string(a_cols.size()) + " vs " +
                                       std::to_string(b_rows.size()) + ")");
    if (a_rows.size() != C->h_rs.size() || b_cols.size() != C->h_cs.size())
        return fail(DBCSR_ERR_DIM, "multiply: C block grid does not match op(A) x op(B)");
    if (a_cols != b_rows) return fail(DBCSR_ERR_DIM, "multiply: inner block sizes of op(A) and op(B) differ");
    if (a_rows != C->h_rs || b_cols != C->h_cs)
        return fail(DBCSR_ERR_DIM, "multiply: C block sizes do not match op(A) x op(B)");
    return DBCSR_OK;
}

double useful_flops_host(bool ta, bool tb, dbcsr_matrix_s* A, dbcsr_matrix_s* B, int64_t* nprod) {
    // sum over k of (2 * k_size * sum_{i in col k of op A} m_i * sum_{j in row k of op B} n_j)
    // computed on the host from the downloaded indices
    // (the per-line sums are kept with each matrix's host index: an operand
    // that does not change costs one pass over its blocks, once)
    download_index(A);
    download_index(B);
    const int nk = ta ? A->nbr : A->nbc;
    const std::vector<double>& am = ta ? A->h_row_cs : A->h_col_rs;
    const std::vector<int64_t>& ac = ta ? A->h_row_n : A->h_col_n;
    const std::vector<double>& bn = tb ? B->h_col_rs : B->h_row_cs;
    const std::vector<int64_t>& bc = tb ? B->h_col_n : B->h_row_n;
    double f = 0.0;
    int64_t np = 0;
    const std::vector<int>& ks = ta ? A->h_rs : A->h_cs;
    for (int k = 0; k < nk; k++) {
        f += 2.0 * ks[k] * am[k] * bn[k];
        np += ac[k] * bc[k];
    }
    if (nprod) *nprod = np;
    return f;
}

__global__ void k_iota_i32(int64_t n, int* __restrict__ out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < n) out[b] = (int)b;
}

bool plan_matches(const ReusePlan* rp, bool ta, bool tb, double alpha, double beta, dbcsr_matrix_s* A,
                  dbcsr_matrix_s* B, dbcsr_matrix_s* C) {
    return rp && rp->exec && rp->a_uid == A->uid && rp->a_ver == A->version && rp->b_uid == B->uid &&
           rp->b_ver == B->version && rp->c_ver == C->version && rp->ta == ta && rp->tb == tb &&
           rp->alpha == alpha && rp->beta == beta && rp->use_old == (beta != 0.0);
}

// The FP64 product kernels over C blocks [b0, b1) of the plan (one contiguous
// run of C block rows): the same arguments with the C-block arrays offset.
int fp64_stack_run(const SmmArgs& g0, int64_t b0, int64_t b1, dbcsr_matrix_s* C, const dbcsr_opts& o,
                   int team_bound) {
    if (b1 <= b0) return DBCSR_OK;
    SmmArgs g = g0;
    g.nC = b1 - b0;
    g.c_row += b0;
    g.c_col += b0;
    g.c_off += b0;
    if (g.c_old) g.c_old += b0;
    g.c_pstart += b0;
    DB_CUDA(cudaMemsetAsync(g.counter, 0, sizeof(unsigned long long), g_ctx.stream));
    return smm_fp64_dispatch(g, C->max_rs * C->max_cs, o.kernel, team_bound);
}

// Hybrid partial densification: Sec. III coalesces all blocks of a dense
// operand into one block; here the decision is taken per panel of consecutive
// block rows of op(A). A panel whose stored elements fill at least
// hybrid_fill_pct % of it (with op(B) at least as full) is densified:
// dense panel of op(A) x dense op(B) (+ beta x the dense panel of old C) in one
// GEMM of the requested precision, then split into the plan's C blocks of
// those rows; the other panels run the stack kernels on their C blocks. Every
// C block is written by exactly one of the two.
int hybrid_products(const SmmArgs& g, const StackPlan& P, double* data, bool ta, bool tb, double alpha,
                    dbcsr_matrix_s* A, dbcsr_matrix_s* B, double beta, bool use_old, dbcsr_matrix_s* C,
                    const dbcsr_opts& o) {
    if (o.precision == DBCSR_PREC_TF32 || o.precision == DBCSR_PREC_FP32)
        return fail(DBCSR_ERR_ARG, "hybrid path: FP64 or emulated FP64 only (TF32 has no stack kernels, FP32 no "
                                   "dense GEMM)");
    const int nrows = C->nbr;
    const int64_t N = C->h_coff[C->nbc];
    const int64_t K = ta ? A->h_roff[A->nbr] : A->h_coff[A->nbc];
    const std::vector<int>& rsz = C->h_rs;
    // stored elements of op(A) per block row
    DB_TRY(download_index(A));
    std::vector<double> rowel(nrows, 0.0);
    for (int i = 0; i < A->nbr; i++)
        for (int b = A->h_rowptr[i]; b < A->h_rowptr[i + 1]; b++) {
            const int j = A->h_col[b];
            rowel[ta ? j : i] += (double)A->h_rs[i] * A->h_cs[j];
        }
    const double fillB = (K > 0 && N > 0) ? (double)B->nelems / ((double)K * (double)N) : 0.0;
    const double theta = (o.hybrid_fill_pct > 0 ? o.hybrid_fill_pct : 50) / 100.0;
    int prow = o.hybrid_panel;
    if (prow <= 0) {
        const double avg = nrows > 0 ? (double)C->h_roff[nrows] / nrows : 1.0;
        prow = std::max(1, (int)std::ceil(1024.0 / std::max(avg, 1.0)));
    }
    // runs of consecutive panels with the same decision
    std::vector<std::pair<int, int>> runs;   // [r0, r1)
    std::vector<char> dense_run;
    for (int r0 = 0; r0 < nrows; r0 += prow) {
        const int r1 = std::min(nrows, r0 + prow);
        double el = 0.0, cap = 0.0;
        for (int r = r0; r < r1; r++) {
            el += rowel[r];
            cap += (double)rsz[r] * (double)K;
        }
        const bool dense = K > 0 && cap > 0.0 && el / cap >= theta && fillB >= theta;
        g_stats.dense_panels += dense ? 1 : 0;
        if (!runs.empty() && (bool)dense_run.back() == dense && runs.back().second == r0)
            runs.back().second = r1;
        else {
            runs.push_back({r0, r1});
            dense_run.push_back(dense ? 1 : 0);
        }
    }
    // C block ranges of block rows and product ranges of C blocks (host copies)
    std::vector<int> crp(nrows + 1);
    DB_TRY(d2h(crp.data(), P.c_rowptr, sizeof(int) * (nrows + 1)));
    std::vector<int64_t> ps(P.nC + 1);
    DB_TRY(d2h(ps.data(), P.c_pstart, sizeof(int64_t) * (P.nC + 1)));
    // stack runs first; the dense panels are gathered into one GEMM (separate
    // panel GEMMs would each fill only part of the GPU)
    double flops = 0.0, useful_dense = 0.0;   // useful_dense: products of the dense runs
    int64_t Md = 0;
    std::vector<int64_t> at(runs.size(), 0);
    CRanges sparse;
    int64_t sparse_prod = 0;
    for (size_t q = 0; q < runs.size(); q++) {
        const int r0 = runs[q].first, r1 = runs[q].second;
        const int64_t b0 = crp[r0], b1 = crp[r1];
        if (!dense_run[q]) {
            if (o.precision == DBCSR_PREC_FP64) {
                DB_TRY(fp64_stack_run(g, b0, b1, C, o, smm_table_team_bound(C->u_rs, C->u_cs, ta ? A->u_rs : A->u_cs)));
            } else {
                sparse.push_back({b0, b1});   // emulated: one call, operands sliced once
                sparse_prod += ps[b1] - ps[b0];
            }
            continue;
        }
        at[q] = Md;
        Md += C->h_roff[r1] - C->h_roff[r0];
        useful_dense += ps[b1] - ps[b0];
    }
    if (!sparse.empty()) {
        double f = 0.0;
        DB_CUDA(cudaMemsetAsync(g.counter, 0, sizeof(unsigned long long), g_ctx.stream));
        DB_TRY(smm_emulated(g, A, ta, B, tb, C, o, sparse_prod, &f, &sparse));
        flops += f;
    }
    if (Md > 0) {
        cudaStream_t st = g_ctx.stream;
        DBuf<double> dB, dA, dC;
        DB_TRY(dB.alloc((size_t)std::max<int64_t>(K * N, 1)));
        DB_TRY(densify(B, tb, dB.p, K, B->nblks != (int64_t)B->nbr * B->nbc));
        DB_TRY(dA.alloc((size_t)std::max<int64_t>(Md * K, 1)));
        DB_TRY(dC.alloc((size_t)std::max<int64_t>(Md * N, 1)));
        if (Md * K > 0) DB_CUDA(cudaMemsetAsync(dA.p, 0, sizeof(double) * (size_t)(Md * K), st));
        if (use_old && Md * N > 0) DB_CUDA(cudaMemsetAsync(dC.p, 0, sizeof(double) * (size_t)(Md * N), st));
        for (size_t q = 0; q < runs.size(); q++) {
            if (!dense_run[q]) continue;
            DB_TRY(densify_rows(A, ta, runs[q].first, runs[q].second, dA.p, Md, at[q]));
            if (use_old) DB_TRY(densify_rows(C, false, runs[q].first, runs[q].second, dC.p, Md, at[q]));
        }
        const double beta_eff = use_old ? beta : 0.0;
        if (o.precision == DBCSR_PREC_FP64) {
            DB_TRY(dgemm_fp64(Md, N, K, alpha, dA.p, Md, dB.p, K, beta_eff, dC.p, Md));
            flops += 2.0 * (double)Md * (double)N * (double)K;
        } else {
            double f = 0.0;
            DB_TRY(dgemm_emulated(Md, N, K, alpha, dA.p, Md, dB.p, K, beta_eff, dC.p, Md, o, &f));
            flops += f;
        }
        for (size_t q = 0; q < runs.size(); q++) {
            if (!dense_run[q]) continue;
            const int r0 = runs[q].first, r1 = runs[q].second;
            DB_TRY(undensify_blocks(crp[r0], crp[r1], P.c_row, P.c_col, P.c_off, data, C, dC.p, Md,
                                    C->h_roff[r0] - at[q]));
        }
    }
    // main_flops: the dense GEMMs' arithmetic, plus for FP64 stack runs their
    // products at the average useful flops per product (emulated runs report
    // their own tensor-core arithmetic)
    if (o.precision == DBCSR_PREC_FP64) {
        const double avg = P.nprod > 0 ? g_stats.useful_flops / (double)P.nprod : 0.0;
        flops += avg * ((double)P.nprod - useful_dense);
    }
    g_stats.main_flops = flops;
    return DBCSR_OK;
}

int multiply_stacks(bool ta, bool tb, double alpha, dbcsr_matrix_s* A, dbcsr_matrix_s* B, double beta,
                    dbcsr_matrix_s* C, const dbcsr_opts& o) {
    const bool reuse = o.reuse_plan != 0 && o.precision == DBCSR_PREC_FP64 && o.path != DBCSR_PATH_HYBRID;
    if (reuse && plan_matches(static_cast<ReusePlan*>(C->plan), ta, tb, alpha, beta, A, B, C)) {
        // same patterns into the C this plan produced: replay the product kernel in place
        ReusePlan* rp = static_cast<ReusePlan*>(C->plan);
        mark(0);
        mark(1);
        timer_kernel_begin();
        DB_CUDA(cudaGraphLaunch(rp->exec, g_ctx.stream));
        count_launch();
        timer_kernel_end();
        mark(2);
        mark(3);
        g_stats.main_flops = g_stats.useful_flops;
        g_stats.main_bytes = 8.0 * ((double)A->nelems + (double)B->nelems + (double)C->nelems *
                                                                              (rp->use_old ? 2.0 : 1.0));
        g_stats.c_blocks = C->nblks;
        return DBCSR_OK;
    }
    if (ta) DB_TRY(build_transpose_index(A));
    if (tb) DB_TRY(build_transpose_index(B));
    OpView va = make_view(A, ta), vb = make_view(B, tb);
    const bool use_old = beta != 0.0 && C->nblks > 0;
    StackPlan P;
    mark(0);
    DB_TRY(build_stacks(va, vb, use_old ? C : nullptr, C->d_rs, C->d_cs, P));
    double* data = nullptr;
    DB_TRY(dalloc(&data, (size_t)(P.nelem ? P.nelem : 1)));
    DBuf<unsigned long long> counter;
    DB_TRY(counter.alloc(1));
    DB_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), g_ctx.stream));
    SmmArgs g;
    g.nC = P.nC;
    g.c_row = P.c_row;
    g.c_col = P.c_col;
    g.c_off = P.c_off;
    g.c_old = use_old ? P.c_old : nullptr;
    g.c_pstart = P.c_pstart;
    g.prod = P.prod;
    g.A = va;
    g.B = vb;
    g.rsC = C->d_rs;
    g.csC = C->d_cs;
    g.Cd = data;
    g.Cold = use_old ? C->d_data : nullptr;
    g.Cold_off = use_old ? C->d_off : nullptr;
    g.alpha = alpha;
    g.beta = beta;
    g.counter = counter.p;
    g.A32 = nullptr;
    g.B32 = nullptr;
    DBuf<float> a32, b32;
    if (o.precision == DBCSR_PREC_FP32) {
        // FP32 copies of the operands' stored data (same offsets)
        DB_TRY(a32.alloc((size_t)std::max<int64_t>(A->nelems, 1)));
        DB_TRY(b32.alloc((size_t)std::max<int64_t>(B->nelems, 1)));
        DB_TRY(to_f32(A->d_data, A->nelems, a32.p));
        DB_TRY(to_f32(B->d_data, B->nelems, b32.p));
        g.A32 = a32.p;
        g.B32 = b32.p;
    }
    int rc;
    mark(1);
    if (o.path == DBCSR_PATH_HYBRID) {
        rc = hybrid_products(g, P, data, ta, tb, alpha, A, B, beta, use_old, C, o);
    } else if (o.precision == DBCSR_PREC_FP64) {
        timer_kernel_begin();
        rc = smm_fp64_dispatch(g, C->max_rs * C->max_cs, o.kernel,
                               smm_table_team_bound(C->u_rs, C->u_cs, ta ? A->u_rs : A->u_cs));
        timer_kernel_end();
        g_stats.main_flops = g_stats.useful_flops;
    } else if (o.precision == DBCSR_PREC_FP32) {
        timer_kernel_begin();
        rc = smm_fp32_dispatch(g, C->max_rs * C->max_cs,
                               std::max(std::max(A->max_rs, A->max_cs), std::max(B->max_rs, B->max_cs)));
        timer_kernel_end();
        g_stats.main_flops = g_stats.useful_flops;
    } else {
        rc = smm_emulated(g, A, ta, B, tb, C, o, P.nprod, &g_stats.main_flops);
    }
    mark(2);
    if (rc) { dfree(data, (size_t)(P.nelem ? P.nelem : 1)); return rc; }
    // minimal traffic: every stored A and B block read once, C written once (+ read once)
    g_stats.main_bytes = 8.0 * ((double)A->nelems + (double)B->nelems + (double)P.nelem +
                                (use_old ? (double)C->nelems : 0.0));
    g_stats.n_products = P.nprod;
    g_stats.c_blocks = P.nC;
    // hand C the new index (the plan's arrays change owner)
    int* rowptr = P.c_rowptr;
    int* col = P.c_col;
    int* row_of = P.c_row;
    int64_t* off = P.c_off;
    P.c_rowptr = nullptr;
    P.c_col = nullptr;
    P.c_row = nullptr;
    P.c_off = nullptr;
    const int64_t nC = P.nC, ne = P.nelem;
    P.nC = 0;   // arrays above no longer belong to P
    dfree(P.c_old, (size_t)(nC ? nC : 1));
    int64_t* pstart = P.c_pstart;
    P.c_pstart = nullptr;
    free_plan(C);
    install(C, nC, ne, rowptr, col, row_of, off, data);
    if (!reuse) {
        dfree(pstart, (size_t)nC + 1);
        mark(3);
        return DBCSR_OK;
    }
    // keep the product list with C and capture the in-place product kernel
    auto* rp = new ReusePlan();
    rp->a_uid = A->uid; rp->a_ver = A->version; rp->b_uid = B->uid; rp->b_ver = B->version;
    rp->c_ver = C->version; rp->ta = ta; rp->tb = tb; rp->alpha = alpha; rp->beta = beta;
    rp->use_old = beta != 0.0;
    rp->nC = nC;
    rp->nprod = P.nprod;
    rp->c_pstart = pstart;
    rp->prod = P.prod;
    P.prod = nullptr;
    P.nprod = 0;
    C->plan = rp;
    DB_TRY(dalloc(&rp->c_ident, (size_t)(nC ? nC : 1)));
    DB_TRY(dalloc(&rp->counter, 1));
    if (nC > 0) {
        k_iota_i32<<<(unsigned)cdiv(nC, 256), 256, 0, g_ctx.stream>>>(nC, rp->c_ident);
        DB_KCHECK();
    }
    SmmArgs r = g;
    r.c_row = C->d_row_of;
    r.c_col = C->d_col;
    r.c_off = C->d_off;
    r.c_pstart = rp->c_pstart;
    r.prod = rp->prod;
    r.Cd = C->d_data;
    r.c_old = rp->use_old ? rp->c_ident : nullptr;
    r.Cold = rp->use_old ? C->d_data : nullptr;      // in place: each owner reads then writes its block
    r.Cold_off = rp->use_old ? C->d_off : nullptr;
    r.counter = rp->counter;
    DB_CUDA(cudaStreamSynchronize(g_ctx.stream));
    cudaStream_t cap;
    DB_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = g_ctx.stream;
    g_ctx.stream = cap;
    int rc2 = DBCSR_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(rp->counter, 0, sizeof(unsigned long long), cap);
        rc2 = smm_fp64_generic(r, C->max_rs * C->max_cs);
        e = cudaStreamEndCapture(cap, &rp->graph);
        if (e == cudaSuccess && rc2 == DBCSR_OK) e = cudaGraphInstantiate(&rp->exec, rp->graph, 0);
    }
    g_ctx.stream = saved;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || rc2 != DBCSR_OK) {
        cudaGetLastError();
        free_plan(C);
        return rc2 != DBCSR_OK ? rc2 : fail(DBCSR_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    mark(3);
    return DBCSR_OK;
}

__global__ void k_full_index(int nbr, int nbc, const int* __restrict__ rs, const int* __restrict__ cs,
                             const int64_t* __restrict__ roff, const int64_t* __restrict__ coff, int64_t N,
                             int* __restrict__ rowptr, int* __restrict__ col, int* __restrict__ row_of,
                             int64_t* __restrict__ off) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nb = (int64_t)nbr * nbc;
    if (b < nb) {
        int i = (int)(b / nbc), j = (int)(b % nbc);
        col[b] = j;
        row_of[b] = i;
        off[b] = roff[i] * N + (int64_t)rs[i] * coff[j];
    }
    if (b <= nbr && b >= 0) rowptr[b] = (int)(b * nbc);
    if (b == 0) off[nb] = roff[nbr] * N;
}

// Give C the fully occupied index (every block, CSR order) with fresh data.
int install_full_index(dbcsr_matrix_s* C, int64_t M, int64_t N) {
    const int64_t nb = (int64_t)C->nbr * C->nbc;
    if (nb >= INT32_MAX) return fail(DBCSR_ERR_OVERFLOW, "multiply: result has too many blocks");
    int *rowptr = nullptr, *col = nullptr, *row_of = nullptr;
    int64_t* off = nullptr;
    double* data = nullptr;
    DB_TRY(dalloc(&rowptr, (size_t)C->nbr + 1));
    DB_TRY(dalloc(&col, (size_t)nb));
    DB_TRY(dalloc(&row_of, (size_t)nb));
    DB_TRY(dalloc(&off, (size_t)nb + 1));
    DB_TRY(dalloc(&data, (size_t)(M * N)));
    int64_t cnt = std::max<int64_t>(nb, C->nbr + 1);
    k_full_index<<<(unsigned)cdiv(cnt, 256), 256, 0, g_ctx.stream>>>(C->nbr, C->nbc, C->d_rs, C->d_cs, C->d_roff,
                                                                     C->d_coff, N, rowptr, col, row_of, off);
    DB_KCHECK();
    install(C, nb, M * N, rowptr, col, row_of, off, data);
    return DBCSR_OK;
}

int multiply_dense(bool ta, bool tb, double alpha, dbcsr_matrix_s* A, dbcsr_matrix_s* B, double beta,
                   dbcsr_matrix_s* C, const dbcsr_opts& o) {
    const int64_t M = C->h_roff[C->nbr], N = C->h_coff[C->nbc];
    const int64_t K = ta ? A->h_roff[A->nbr] : A->h_coff[A->nbc];
    const bool a_full = A->nblks == (int64_t)A->nbr * A->nbc;
    const bool b_full = B->nblks == (int64_t)B->nbr * B->nbc;
    const bool use_old = beta != 0.0 && C->nblks > 0;
    const int nbk = ta ? A->nbr : A->nbc;
    const bool c_full = C->nblks == (int64_t)C->nbr * C->nbc && C->nblks > 0;
    // Emulated FP64 with fully occupied operands: slices cut straight from the
    // blocks and the result recombined straight into C's blocks (no dense
    // copies of A, B, C). C is (made) fully occupied; its old values are used
    // in place when beta != 0.
    if (o.precision == DBCSR_PREC_OZAKI && a_full && b_full && nbk > 0 && M > 0 && N > 0 && K > 0 &&
        (!use_old || c_full) && ozaki_blocks_ok(N)) {
        const int s = o.ozaki_slices > 0 ? o.ozaki_slices : 7;
        if (s > 8) return fail(DBCSR_ERR_ARG, "ozaki_slices must be 1..8");
        mark(0);
        if (!c_full) DB_TRY(install_full_index(C, M, N));
        mark(1);
        DB_TRY(dgemm_ozaki_blocks(A, ta, B, tb, C, alpha, use_old ? beta : 0.0, s, &g_stats.main_flops, o.kernel));
        mark(2);
        mark(3);
        g_stats.c_blocks = C->nblks;
        return DBCSR_OK;
    }
    DB_TRY(await_data(A));
    DB_TRY(await_data(B));
    DB_TRY(await_data(C));
    // TF32 with fully occupied operands of one block size per dimension: the
    // TF32 operands straight from the blocks and the GEMM's result straight
    // into C's blocks (no dense copies)
    if (o.precision == DBCSR_PREC_TF32 && a_full && b_full && nbk > 0 && M > 0 && N > 0 && K > 0 &&
        (!use_old || c_full) && tf32_blocks_ok(A, B, N)) {
        mark(0);
        if (!c_full) DB_TRY(install_full_index(C, M, N));
        mark(1);
        DB_TRY(dgemm_tf32_blocks(A, ta, B, tb, C, alpha, use_old ? beta : 0.0, &g_stats.main_flops));
        mark(2);
        mark(3);
        g_stats.c_blocks = C->nblks;
        return DBCSR_OK;
    }
    // result pattern: full when both operands are full (and K > 0); else the
    // symbolic product (through stack generation's pattern pass)
    DBuf<double> dA, dB, dC;
    mark(0);
    DB_TRY(dA.alloc((size_t)std::max<int64_t>(M * K, 1)));
    DB_TRY(dB.alloc((size_t)std::max<int64_t>(K * N, 1)));
    DB_TRY(dC.alloc((size_t)std::max<int64_t>(M * N, 1)));
    DB_TRY(densify(A, ta, dA.p, M, !a_full));
    DB_TRY(densify(B, tb, dB.p, K, !b_full));
    if (use_old) DB_TRY(densify(C, false, dC.p, M, C->nblks != (int64_t)C->nbr * C->nbc));
    const double beta_eff = use_old ? beta : 0.0;
    mark(1);
    if (o.precision == DBCSR_PREC_FP64) {
        DB_TRY(dgemm_fp64(M, N, K, alpha, dA.p, M, dB.p, K, beta_eff, dC.p, M));
        g_stats.main_flops = 2.0 * (double)M * (double)N * (double)K;
    } else {
        DB_TRY(dgemm_emulated(M, N, K, alpha, dA.p, M, dB.p, K, beta_eff, dC.p, M, o, &g_stats.main_flops));
    }
    mark(2);
    if (o.precision != DBCSR_PREC_OZAKI)
        g_stats.main_bytes = 8.0 * ((double)M * K + (double)K * N + (double)M * N * (beta_eff != 0.0 ? 2 : 1));
    // new C index
    if (a_full && b_full && nbk > 0) {
        const bool same = C->nblks == (int64_t)C->nbr * C->nbc;   // old C already full, CSR-ordered
        if (!same) DB_TRY(install_full_index(C, M, N));
        DB_TRY(undensify(C, dC.p, M));
        mark(3);
        g_stats.c_blocks = C->nblks;
        return DBCSR_OK;
    }
    // sparse operands forced onto the dense path: pattern from the symbolic pass
    if (ta) DB_TRY(build_transpose_index(A));
    if (tb) DB_TRY(build_transpose_index(B));
    OpView va = make_view(A, ta), vb = make_view(B, tb);
    StackPlan P;
    DB_TRY(build_stacks(va, vb, use_old ? C : nullptr, C->d_rs, C->d_cs, P));
    double* data = nullptr;
    DB_TRY(dalloc(&data, (size_t)(P.nelem ? P.nelem : 1)));
    const int64_t nC = P.nC, ne = P.nelem;
    install(C, nC, ne, P.c_rowptr, P.c_col, P.c_row, P.c_off, data);
    P.c_rowptr = nullptr;
    P.c_col = nullptr;
    P.c_row = nullptr;
    P.c_off = nullptr;
    P.nC = 0;
    dfree(P.c_old, (size_t)(nC ? nC : 1));
    dfree(P.c_pstart, (size_t)nC + 1);
    DB_TRY(undensify(C, dC.p, M));
    mark(3);
    g_stats.c_blocks = nC;
    return DBCSR_OK;
}

}  // namespace
}  // namespace dbcsr

extern "C" int dbcsr_multiply(char transa, char transb, double alpha, dbcsr_matrix A, dbcsr_matrix B, double beta,
                              dbcsr_matrix C, const dbcsr_opts* opts) {
    g_last_error.clear();
    if (!A || !B || !C) return fail(DBCSR_ERR_ARG, "multiply: NULL matrix");
    if (C == A || C == B) return fail(DBCSR_ERR_ARG, "multiply: C must differ from A and B");
    if (!valid_trans(transa) || !valid_trans(transb))
        return fail(DBCSR_ERR_ARG, "multiply: trans must be 'N', 'T' or 'C'");
    dbcsr_opts o{};
    if (opts) o = *opts;
    if (o.path < 0 || o.path > 3 || o.precision < 0 || o.precision > 3 || o.ozaki_slices < 0 ||
        o.ozaki_slices > 12 || o.hybrid_panel < 0 || o.hybrid_fill_pct < 0 || o.hybrid_fill_pct > 100)
        return fail(DBCSR_ERR_ARG, "multiply: invalid options");
    DB_TRY(ensure_device());
    const bool ta = is_trans(transa), tb = is_trans(transb);
    DB_TRY(check_conformant(ta, tb, A, B, C));
    const int64_t launches0 = g_launches.load();
    std::memset(&g_stats, 0, sizeof(g_stats));
    int64_t np = 0;
    g_stats.useful_flops = useful_flops_host(ta, tb, A, B, &np);
    g_stats.n_products = np;
    int path = o.path;
    if (path == DBCSR_PATH_AUTO) {
        // Sec. III: densify when both operands are dense. Sec. II: blocks beyond
        // the small-matrix kernels' range go to a GEMM -- here the emulated
        // stack kernels take edges up to 32, so larger blocks take the
        // densified GEMM, as does TF32 (no stack kernel) on sparse operands.
        const bool a_full = A->nblks == (int64_t)A->nbr * A->nbc && A->nblks > 0;
        const bool b_full = B->nblks == (int64_t)B->nbr * B->nbc && B->nblks > 0;
        const int max_edge = std::max(std::max(A->max_rs, A->max_cs), std::max(B->max_rs, B->max_cs));
        if (o.precision == DBCSR_PREC_FP32) path = DBCSR_PATH_STACKS;
        else if (a_full && b_full)
            // FP64 blocks up to 32 x 32 run faster on the stack kernels than
            // densified on the FP64 tensor-core GEMM, whatever the occupancy
            path = (o.precision == DBCSR_PREC_FP64 && max_edge <= 32) ? DBCSR_PATH_STACKS : DBCSR_PATH_DENSE;
        else if (o.precision == DBCSR_PREC_TF32) path = DBCSR_PATH_DENSE;
        else if (o.precision == DBCSR_PREC_OZAKI && max_edge > EMUL_STACK_MAX_EDGE) path = DBCSR_PATH_DENSE;
        else path = DBCSR_PATH_STACKS;
    }
    if (path == DBCSR_PATH_DENSE && o.precision == DBCSR_PREC_FP32)
        return fail(DBCSR_ERR_ARG, "multiply: FP32 runs on the stack path (the dense path offers TF32)");
    g_stats.path = path;
    g_stats.precision = o.precision;
    // uploads still in flight: the emulated and TF32 dense paths wait for each
    // operand where they first read it (the copies of B and C then overlap the
    // work on A); every other path waits here
    if (!(path == DBCSR_PATH_DENSE && (o.precision == DBCSR_PREC_OZAKI || o.precision == DBCSR_PREC_TF32))) {
        DB_TRY(await_data(A));
        DB_TRY(await_data(B));
        DB_TRY(await_data(C));
    }
    PhaseTimer timer;
    timer.init(o.timing != 0);
    g_timer = timer.on ? &timer : nullptr;
    // the hybrid path is the stack path with some panels of C block rows densified
    int rc = (path == DBCSR_PATH_DENSE) ? multiply_dense(ta, tb, alpha, A, B, beta, C, o)
                                        : multiply_stacks(ta, tb, alpha, A, B, beta, C, o);
    g_timer = nullptr;
    if (rc == DBCSR_OK) rc = sync_stream();
    if (rc == DBCSR_OK) timer.finish(g_stats);
    g_stats.kernel_launches = (int)(g_launches.load() - launches0);
    C->h_valid = false;
    C->t_valid = false;
    return rc;
}

extern "C" int dbcsr_set_wait_limit(int64_t ns) {
    g_last_error.clear();
    g_ctx.wait_ns = ns > 0 ? (uint64_t)ns : 4000000000ull;
    return DBCSR_OK;
}

extern "C" int dbcsr_get_stacks(char transa, char transb, dbcsr_matrix A, dbcsr_matrix B, int stack_cap, int* out,
                                int64_t cap, int64_t* n_out) {
    g_last_error.clear();
    if (!A || !B || !n_out) return fail(DBCSR_ERR_ARG, "get_stacks: NULL argument");
    if (!valid_trans(transa) || !valid_trans(transb))
        return fail(DBCSR_ERR_ARG, "get_stacks: trans must be 'N', 'T' or 'C'");
    DB_TRY(ensure_device());
    const bool ta = is_trans(transa), tb = is_trans(transb);
    const std::vector<int>& a_cols = ta ? A->h_rs : A->h_cs;
    const std::vector<int>& b_rows = tb ? B->h_cs : B->h_rs;
    if (a_cols != b_rows) return fail(DBCSR_ERR_DIM, "get_stacks: inner block sizes differ");
    if (ta) DB_TRY(build_transpose_index(A));
    if (tb) DB_TRY(build_transpose_index(B));
    OpView va = make_view(A, ta), vb = make_view(B, tb);
    StackPlan P;
    DB_TRY(build_stacks(va, vb, nullptr, va.rs, vb.cs, P));
    *n_out = P.nprod;
    std::vector<int> sizes;
    sizes.insert(sizes.end(), A->h_rs.begin(), A->h_rs.end());
    sizes.insert(sizes.end(), A->h_cs.begin(), A->h_cs.end());
    sizes.insert(sizes.end(), B->h_rs.begin(), B->h_rs.end());
    sizes.insert(sizes.end(), B->h_cs.begin(), B->h_cs.end());
    int64_t nst = 0, nsh = 0;
    if (out && cap >= P.nprod) DB_TRY(export_stacks(va, P, va.rs, vb.cs, sizes, stack_cap, out, &nst, &nsh));
    return DBCSR_OK;
}
