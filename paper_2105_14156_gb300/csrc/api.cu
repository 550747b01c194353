// C ABI: handle, scratch memory, planner and the symbolic / numeric calls.
//
// The planner follows the paper's Window Distribution Phase: count each row's
// products from the row pointers, decide dense or sparse per row by a
// threshold, and group rows so that each group's tables fit on-chip memory
// (here: one block's shared memory instead of a PIUMA block's scratchpad).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "kernels.h"
#include "smash.h"

using namespace smash;

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Event timing of kernel launches (tracing).
struct PendingTime {
    int slot;  // index into totals
    cudaEvent_t e0, e1;
};

struct smash_handle {
    bool timing = false;
    std::vector<PendingTime> pending;
    std::vector<smash_kernel_time> totals;
    std::vector<cudaEvent_t> spare_events;
    int device = 0;
    int sms = 0;
    smash_params params{};
    smash_alloc_fn alloc = nullptr;
    smash_free_fn free_fn = nullptr;
    void *ctx = nullptr;
    DevBuf ws;         // per-call arrays
    DevBuf tables;     // spill hash tables
    DevBuf dense_acc;  // dense accumulators (kept zero between rows)
    DevBuf split;      // column slices of B for cluster-wide dense rows
    DevBuf hot;        // hot-column tables of B
    DevBuf err;        // kNumErr ints (+ scratch words)
    long long *host = nullptr;  // pinned host staging
    smash_stats stats{};
};

namespace {

constexpr int kHostWords = 256;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

void *default_alloc(size_t bytes, void *) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void default_free(void *p, void *) { cudaFree(p); }

int release(smash_handle *h, DevBuf &b) {
    if (b.ptr) {
        cudaDeviceSynchronize();
        h->free_fn(b.ptr, h->ctx);
    }
    b.ptr = nullptr;
    b.bytes = 0;
    return SMASH_OK;
}

// Grow-only buffer. Growing synchronises the stream first (the old buffer may
// still be read by queued kernels).
int ensure(smash_handle *h, DevBuf &b, size_t need, cudaStream_t s, bool zero = false) {
    if (need == 0) need = 256;
    if (b.bytes >= need) return SMASH_OK;
    cudaStreamSynchronize(s);
    if (b.ptr) h->free_fn(b.ptr, h->ctx);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = need + need / 4;
    want = (want + 4095) & ~size_t(4095);
    void *p = h->alloc(want, h->ctx);
    if (!p) {
        want = (need + 4095) & ~size_t(4095);
        p = h->alloc(want, h->ctx);
    }
    if (!p) return SMASH_ERR_ALLOC;
    b.ptr = p;
    b.bytes = want;
    if (zero && cudaMemsetAsync(p, 0, want, s) != cudaSuccess) return SMASH_ERR_CUDA;
    return SMASH_OK;
}

cudaEvent_t take_event(smash_handle *h) {
    if (!h->spare_events.empty()) {
        cudaEvent_t e = h->spare_events.back();
        h->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one kernel launch with events when timing is on.
struct LaunchTimer {
    smash_handle *h;
    cudaStream_t s;
    int slot = -1;
    cudaEvent_t e0 = nullptr;
    LaunchTimer(smash_handle *hh, cudaStream_t ss, const char *name, int bin, int threads, long long rows,
                long long a_nnz, long long products, long long c_nnz)
        : h(hh), s(ss) {
        if (!h->timing) return;
        for (size_t k = 0; k < h->totals.size(); ++k)
            if (h->totals[k].bin == bin && strncmp(h->totals[k].name, name, sizeof(h->totals[k].name)) == 0)
                slot = (int)k;
        if (slot < 0) {
            smash_kernel_time kt;
            memset(&kt, 0, sizeof(kt));
            strncpy(kt.name, name, sizeof(kt.name) - 1);
            kt.bin = bin;
            h->totals.push_back(kt);
            slot = (int)h->totals.size() - 1;
        }
        smash_kernel_time &kt = h->totals[slot];
        kt.threads = threads;
        kt.launches += 1;
        kt.rows += rows;
        kt.a_nnz += a_nnz;
        kt.products += products;
        kt.c_nnz += c_nnz;
        e0 = take_event(h);
        cudaEventRecord(e0, s);
    }
    ~LaunchTimer() {
        if (!h->timing || slot < 0) return;
        cudaEvent_t e1 = take_event(h);
        cudaEventRecord(e1, s);
        h->pending.push_back(PendingTime{slot, e0, e1});
    }
};

void resolve_timings(smash_handle *h) {
    for (const PendingTime &p : h->pending) {
        cudaEventSynchronize(p.e1);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) h->totals[p.slot].ms += ms;
        h->spare_events.push_back(p.e0);
        h->spare_events.push_back(p.e1);
    }
    h->pending.clear();
    cudaGetLastError();
}

struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *p) : base((char *)p) {}
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *r = (T *)(base + off);
        off += count * sizeof(T);
        return r;
    }
};
template <typename T>
size_t carve_size(size_t &acc, size_t count) {
    acc = (acc + 255) & ~size_t(255);
    acc += count * sizeof(T);
    return acc;
}

int status_from_flags(const long long *flags_as_ll) {
    const int *f = (const int *)flags_as_ll;
    if (f[kErrBadIndex] || f[kErrBadRowPtr] || f[kErrCountMismatch]) return SMASH_ERR_INVALID_ARG;
    if (f[kErrBRowTooLong]) return SMASH_ERR_UNSUPPORTED;
    if (f[kErrTimeout]) return SMASH_ERR_TIMEOUT;
    if (f[kErrTableFull]) return SMASH_ERR_INTERNAL;
    return SMASH_OK;
}

int check_params(const smash_params *p) {
    if (!p) return SMASH_ERR_INVALID_ARG;
    if (p->hash_kind < 0 || p->hash_kind > 2) return SMASH_ERR_INVALID_ARG;
    if (!(p->max_load > 0.05f && p->max_load <= 0.95f)) return SMASH_ERR_INVALID_ARG;
    if (p->sym_max_tbits < kMinTBits || p->sym_max_tbits > 15) return SMASH_ERR_INVALID_ARG;
    if (p->num_max_tbits < kMinTBits || p->num_max_tbits > 14) return SMASH_ERR_INVALID_ARG;
    if (p->group_shift < 0 || p->group_shift > 10) return SMASH_ERR_INVALID_ARG;
    if (p->dense_ratio < 0 || p->bitmap_ratio < 0) return SMASH_ERR_INVALID_ARG;
    if (p->spill_blocks_per_sm < 0 || p->spill_blocks_per_sm > 8) return SMASH_ERR_INVALID_ARG;
    if (p->sym_dense_ratio < 0) return SMASH_ERR_INVALID_ARG;
    if (p->hot_cols < 0 || p->hot_cols > 512 || p->hot_factor < 1) return SMASH_ERR_INVALID_ARG;
    if (p->cluster_max != 1 && p->cluster_max != 2 && p->cluster_max != 4 && p->cluster_max != 8)
        return SMASH_ERR_INVALID_ARG;
    return SMASH_OK;
}

int check_csr(const smash_csr *M, bool need_val) {
    if (!M) return SMASH_ERR_INVALID_ARG;
    if (M->rows < 0 || M->cols < 0 || M->nnz < 0) return SMASH_ERR_INVALID_ARG;
    if (M->rows >= (1ll << 31) || M->cols >= (1ll << 31)) return SMASH_ERR_UNSUPPORTED;
    if (!M->row_ptr) return SMASH_ERR_INVALID_ARG;
    if (M->nnz > 0 && !M->col_idx) return SMASH_ERR_INVALID_ARG;
    if (need_val && M->nnz > 0 && !M->val) return SMASH_ERR_INVALID_ARG;
    return SMASH_OK;
}

int colbits_of(int64_t ncols) {
    int b = 0;
    while ((1ll << b) < ncols) ++b;
    return b;
}

RawOperands raw_ops(const smash_csr *A, const smash_csr *B) {
    RawOperands r;
    r.a_rp = A->row_ptr;
    r.a_ci = A->col_idx;
    r.a_val = A->val;
    r.b_rp = B->row_ptr;
    r.b_ci = B->col_idx;
    r.b_val = B->val;
    r.a_rows = A->rows;
    r.a_nnz = A->nnz;
    r.b_nnz = B->nnz;
    r.b_rows = (int32_t)B->rows;
    r.ncols = (int32_t)B->cols;
    return r;
}

// Per-call planning buffers carved from h->ws.
struct Plan {
    BinBuffers bb;
    long long *bound;
    int *nnz;
    void *scan;
    long long *total;
};

int plan_buffers(smash_handle *h, int64_t n, bool symbolic, cudaStream_t s, Plan &pl) {
    size_t need = 0;
    carve_size<uint8_t>(need, (size_t)n);
    carve_size<int>(need, 16 * 3);
    carve_size<long long>(need, 16 + 4 + 1);
    carve_size<int>(need, (size_t)n);
    carve_size<int>(need, 17);
    carve_size<long long>(need, 48);
    if (symbolic) {
        carve_size<long long>(need, (size_t)n);
        carve_size<int>(need, (size_t)n);
        carve_size<char>(need, scan_scratch_bytes(n));
    }
    int st = ensure(h, h->ws, need, s);
    if (st) return st;
    Carver c(h->ws.ptr);
    pl.bb.bin = c.take<uint8_t>((size_t)n);
    int *ctr = c.take<int>(16 * 3);
    long long *ll = c.take<long long>(16 + 4 + 1);
    pl.bb.counts = ctr;
    pl.bb.cursor = ctr + 16;
    pl.bb.tokens = ctr + 32;
    pl.bb.maxsize = ll;
    pl.bb.stats = ll + 16;
    pl.total = ll + 20;
    pl.bb.rows = c.take<int>((size_t)n);
    pl.bb.offsets = c.take<int>(17);
    pl.bb.sums = c.take<long long>(48);
    pl.bound = nullptr;
    pl.nnz = nullptr;
    pl.scan = nullptr;
    if (symbolic) {
        pl.bound = c.take<long long>((size_t)n);
        pl.nnz = c.take<int>((size_t)n);
        pl.scan = c.take<char>(scan_scratch_bytes(n));
    }
    // zero counters, cursors, tokens, maxsize, stats, total
    if (cudaMemsetAsync(ctr, 0, 16 * 3 * sizeof(int), s) != cudaSuccess) return SMASH_ERR_CUDA;
    if (cudaMemsetAsync(ll, 0, (16 + 4 + 1) * sizeof(long long), s) != cudaSuccess) return SMASH_ERR_CUDA;
    if (cudaMemsetAsync(pl.bb.sums, 0, 48 * sizeof(long long), s) != cudaSuccess) return SMASH_ERR_CUDA;
    return SMASH_OK;
}

// Copy bin counts (16 int), offsets (17 int), maxsize (16 ll), stats (4 ll)
// to the pinned host buffer and wait.
int fetch_bins(smash_handle *h, const Plan &pl, cudaStream_t s, int *counts, int *offsets, long long *maxsize,
               long long *stats, long long *sums) {
    char *hb = (char *)h->host;
    if (cudaMemcpyAsync(hb, pl.bb.counts, 16 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hb + 64, pl.bb.offsets, 17 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hb + 256, pl.bb.maxsize, 20 * sizeof(long long), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(hb + 512, pl.bb.sums, 48 * sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SMASH_ERR_CUDA;
    memcpy(counts, hb, 16 * sizeof(int));
    memcpy(offsets, hb + 64, 17 * sizeof(int));
    memcpy(maxsize, hb + 256, 16 * sizeof(long long));
    memcpy(stats, hb + 256 + 16 * sizeof(long long), 4 * sizeof(long long));
    memcpy(sums, hb + 512, 48 * sizeof(long long));
    for (int b = 0; b < 16; ++b) {
        h->stats.rows_per_bin[b] = b < kNumBins ? counts[b] : 0;
        h->stats.a_nnz_per_bin[b] = sums[b];
        h->stats.products_per_bin[b] = sums[16 + b];
        h->stats.c_nnz_per_bin[b] = sums[32 + b];
    }
    h->stats.products = stats[0];
    h->stats.max_row_products = stats[1];
    return SMASH_OK;
}

int read_flags(smash_handle *h, cudaStream_t s, bool clear) {
    char *hb = (char *)h->host + 1024;
    if (cudaMemcpyAsync(hb, h->err.ptr, kNumErr * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    if (clear && cudaMemsetAsync(h->err.ptr, 0, kNumErr * sizeof(int), s) != cudaSuccess) return SMASH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SMASH_ERR_CUDA;
    const int st = status_from_flags((const long long *)hb);
    // a row that failed may have left a dense accumulator dirty: drop them
    if (st != SMASH_OK) release(h, h->dense_acc);
    return st;
}

int last_cuda_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMASH_OK : SMASH_ERR_CUDA;
}

BinRule sym_rule(const smash_handle *h, int64_t ncols) {
    BinRule r;
    r.inv_load = 1.0f / h->params.max_load;
    int mt = h->params.sym_max_tbits;
    // key-only table of 2^mt ints plus the staging of a 1024-thread group
    while (mt > kMinTBits && ((size_t)4 << mt) + 24 * 1024 > (size_t)max_smem_per_block()) --mt;
    r.max_tbits = mt;
    r.dense_ok = (h->params.sym_dense_ratio > 0 && ncols <= dense_bitmap_max_cols()) ? 1 : 0;
    r.dense_min = r.dense_ok ? (ncols + h->params.sym_dense_ratio - 1) / h->params.sym_dense_ratio : (1ll << 62);
    if (r.dense_min < 1) r.dense_min = 1;
    return r;
}

BinRule num_rule(const smash_handle *h, int64_t ncols, int dtype) {
    BinRule r;
    r.inv_load = 1.0f / h->params.max_load;
    const bool dense_fits = num_dense_cluster_size(dtype, (int)ncols, h->params.cluster_max,
                                                   h->params.hot_cols) > 0 ||
                            ncols <= dense_bitmap_max_cols();
    r.dense_ok = (h->params.dense_ratio > 0 && dense_fits) ? 1 : 0;
    r.dense_min = r.dense_ok ? (ncols + h->params.dense_ratio - 1) / h->params.dense_ratio : (1ll << 62);
    if (r.dense_min < 1) r.dense_min = 1;
    int mt = h->params.num_max_tbits;
    // The largest tables are one 1024-thread group; if their rows would want
    // the bitmap write-out but it does not fit, let them take the dense path.
    while (mt > kMinTBits) {
        const int words = (int)((ncols + 31) / 32);
        const long long n_small = (long long)((1ll << (mt - 1)) * h->params.max_load);
        const bool want_bm = h->params.bitmap_ratio > 0 && words <= (long long)h->params.bitmap_ratio * n_small;
        const bool fits_plain = num_hash_bitmap_fits(dtype, mt, 0);
        const bool fits_bm = num_hash_bitmap_fits(dtype, mt, (int)ncols);
        if (fits_plain && (!want_bm || fits_bm || !r.dense_ok)) break;
        --mt;
    }
    r.max_tbits = mt;
    return r;
}

int group_threads(const HashLaunch &hl) {
    int t = 1 << (hl.tbits > hl.group_shift ? hl.tbits - hl.group_shift : 0);
    return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

HashLaunch hash_launch(const smash_handle *h, int tbits, int64_t ncols) {
    HashLaunch hl;
    hl.tbits = tbits;
    hl.group_shift = h->params.group_shift;
    hl.hash_kind = h->params.hash_kind;
    hl.colbits = colbits_of(ncols);
    hl.sms = h->sms;
    hl.blocks_per_sm = h->params.spill_blocks_per_sm > 0 ? h->params.spill_blocks_per_sm : 1;
    hl.cluster_max = h->params.cluster_max;
    return hl;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int smash_default_params(smash_params *p) {
    if (!p) return SMASH_ERR_INVALID_ARG;
    memset(p, 0, sizeof(*p));
    p->hash_kind = 1;
    p->max_load = 0.5f;
    p->sym_max_tbits = 15;
    p->num_max_tbits = 14;
    p->group_shift = 3;
    p->dense_ratio = 4;
    p->bitmap_ratio = 4;
    p->spill_blocks_per_sm = 1;
    p->sym_dense_ratio = 64;
    p->cluster_max = 8;
    p->hot_cols = 128;
    p->hot_factor = 16;
    return SMASH_OK;
}

const char *smash_status_string(int s) {
    switch (s) {
        case SMASH_OK: return "SMASH_OK";
        case SMASH_ERR_INVALID_ARG: return "SMASH_ERR_INVALID_ARG";
        case SMASH_ERR_SHAPE_MISMATCH: return "SMASH_ERR_SHAPE_MISMATCH";
        case SMASH_ERR_UNSUPPORTED: return "SMASH_ERR_UNSUPPORTED";
        case SMASH_ERR_ALLOC: return "SMASH_ERR_ALLOC";
        case SMASH_ERR_CUDA: return "SMASH_ERR_CUDA";
        case SMASH_ERR_TIMEOUT: return "SMASH_ERR_TIMEOUT";
        case SMASH_ERR_INTERNAL: return "SMASH_ERR_INTERNAL";
        default: return "SMASH_ERR_UNKNOWN";
    }
}

int smash_create(smash_handle **out, int device, const smash_params *params) {
    if (!out) return SMASH_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return SMASH_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return SMASH_ERR_INVALID_ARG;
    smash_params p;
    if (params) {
        if (check_params(params)) return SMASH_ERR_INVALID_ARG;
        p = *params;
    } else {
        smash_default_params(&p);
    }
    smash_handle *h = new (std::nothrow) smash_handle();
    if (!h) return SMASH_ERR_ALLOC;
    DeviceGuard g(device);
    h->device = device;
    h->params = p;
    h->alloc = default_alloc;
    h->free_fn = default_free;
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMallocHost((void **)&h->host, kHostWords * 8 * 8) != cudaSuccess) {
        delete h;
        return SMASH_ERR_ALLOC;
    }
    if (ensure(h, h->err, 256, 0) != SMASH_OK || cudaMemset(h->err.ptr, 0, h->err.bytes) != cudaSuccess) {
        cudaFreeHost(h->host);
        delete h;
        return SMASH_ERR_ALLOC;
    }
    *out = h;
    return SMASH_OK;
}

int smash_destroy(smash_handle *h) {
    if (!h) return SMASH_ERR_INVALID_ARG;
    {
        DeviceGuard g(h->device);
        cudaDeviceSynchronize();
        resolve_timings(h);
        for (cudaEvent_t e : h->spare_events) cudaEventDestroy(e);
        h->spare_events.clear();
        release(h, h->ws);
        release(h, h->tables);
        release(h, h->dense_acc);
        release(h, h->split);
        release(h, h->hot);
        release(h, h->err);
        if (h->host) cudaFreeHost(h->host);
    }
    delete h;
    return SMASH_OK;
}

int smash_set_params(smash_handle *h, const smash_params *params) {
    if (!h || check_params(params)) return SMASH_ERR_INVALID_ARG;
    h->params = *params;
    return SMASH_OK;
}

int smash_get_params(const smash_handle *h, smash_params *params) {
    if (!h || !params) return SMASH_ERR_INVALID_ARG;
    *params = h->params;
    return SMASH_OK;
}

int smash_set_allocator(smash_handle *h, smash_alloc_fn alloc, smash_free_fn free_fn, void *ctx) {
    if (!h || (!alloc) != (!free_fn)) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    release(h, h->ws);
    release(h, h->tables);
    release(h, h->dense_acc);
    release(h, h->split);
    release(h, h->hot);
    // the error words move to the new allocator as well
    release(h, h->err);
    h->alloc = alloc ? alloc : default_alloc;
    h->free_fn = free_fn ? free_fn : default_free;
    h->ctx = alloc ? ctx : nullptr;
    if (ensure(h, h->err, 256, 0) != SMASH_OK) return SMASH_ERR_ALLOC;
    if (cudaMemset(h->err.ptr, 0, h->err.bytes) != cudaSuccess) return SMASH_ERR_CUDA;
    return SMASH_OK;
}

int smash_set_timing(smash_handle *h, int enable) {
    if (!h) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    resolve_timings(h);
    h->totals.clear();
    h->timing = enable != 0;
    return SMASH_OK;
}

int smash_get_timings(smash_handle *h, smash_kernel_time *out, int capacity, int *count) {
    if (!h || !count || capacity < 0 || (capacity > 0 && !out)) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    resolve_timings(h);
    *count = (int)h->totals.size();
    for (int k = 0; k < capacity && k < (int)h->totals.size(); ++k) out[k] = h->totals[k];
    return SMASH_OK;
}

int smash_get_stats(const smash_handle *h, smash_stats *out) {
    if (!h || !out) return SMASH_ERR_INVALID_ARG;
    *out = h->stats;
    return SMASH_OK;
}

int smash_check(smash_handle *h, void *stream) {
    if (!h) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    return read_flags(h, (cudaStream_t)stream, true);
}

int spgemm_symbolic(smash_handle *h, const smash_csr *A, const smash_csr *B, int64_t *c_row_ptr,
                    int64_t *c_nnz, void *stream) {
    if (!h || !c_row_ptr || !c_nnz) return SMASH_ERR_INVALID_ARG;
    int st = check_csr(A, false);
    if (st) return st;
    if ((st = check_csr(B, false))) return st;
    if (A->cols != B->rows) return SMASH_ERR_SHAPE_MISMATCH;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->rows;
    memset(&h->stats, 0, sizeof(h->stats));
    if (n == 0 || A->nnz == 0 || B->nnz == 0) {
        if (cudaMemsetAsync(c_row_ptr, 0, sizeof(int64_t) * (size_t)(n + 1), s) != cudaSuccess) return SMASH_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SMASH_ERR_CUDA;
        *c_nnz = 0;
        h->stats.rows_per_bin[kBinEmpty] = n;
        return SMASH_OK;
    }
    Plan pl;
    if ((st = plan_buffers(h, n, true, s, pl))) return st;
    const RawOperands op = raw_ops(A, B);
    const BinRule rule = sym_rule(h, B->cols);
    int *err = (int *)h->err.ptr;
    {
        LaunchTimer lt(h, s, "sym_rowinfo", -1, 256, n, A->nnz, 0, 0);
        launch_sym_rowinfo(op, rule, pl.bb, pl.bound, pl.nnz, err, h->sms, s);
    }
    {
        LaunchTimer lt(h, s, "bin_scatter", -1, 256, n, 0, 0, 0);
        launch_bin_scatter(n, pl.bb, s);
    }
    if ((st = last_cuda_status())) return st;
    int counts[16], offsets[17];
    long long maxsize[16], stats[4], sums[48];
    if ((st = fetch_bins(h, pl, s, counts, offsets, maxsize, stats, sums))) return st;
    for (int b = 1; b < kNumBins; ++b) {
        if (!counts[b]) continue;
        const int *rows = pl.bb.rows + offsets[b];
        int *tok = pl.bb.tokens + b;
        if (b == kBinDense) {
            LaunchTimer lt(h, s, "sym_dense", b, 1024, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_sym_dense(op, rows, counts[b], tok, hash_launch(h, 0, B->cols), pl.nnz, err, s);
        } else if (b == kBinSpill) {
            const int tb = table_bits(maxsize[b], rule.inv_load);
            const HashLaunch hl = hash_launch(h, tb, B->cols);
            const size_t need = ((size_t)sym_spill_grid(hl) << tb) * sizeof(int);
            if ((st = ensure(h, h->tables, need, s))) return st;
            LaunchTimer lt(h, s, "sym_spill", b, 1024, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_sym_spill(op, rows, counts[b], tok, hl, rule.inv_load, pl.bound, tb, (int *)h->tables.ptr,
                             pl.nnz, err, s);
        } else {
            const HashLaunch hl = hash_launch(h, tbits_of_bin(b), B->cols);
            LaunchTimer lt(h, s, "sym_hash", b, group_threads(hl), counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_sym_hash(op, rows, counts[b], tok, hl, pl.nnz, err, s);
        }
        if ((st = last_cuda_status())) return st;
    }
    {
        LaunchTimer lt(h, s, "scan_rowptr", -1, 512, n, 0, 0, 0);
        launch_scan_rowptr(pl.nnz, n, c_row_ptr, pl.total, pl.scan, s);
    }
    if ((st = last_cuda_status())) return st;
    if (cudaMemcpyAsync(h->host, pl.total, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    st = read_flags(h, s, true);
    *c_nnz = h->host[0];
    h->stats.c_nnz = h->host[0];
    return st;
}

int spgemm_numeric(smash_handle *h, const smash_csr *A, const smash_csr *B, smash_dtype dtype, smash_csr *C,
                   void *stream) {
    if (!h) return SMASH_ERR_INVALID_ARG;
    if (dtype != SMASH_F32 && dtype != SMASH_F64) return SMASH_ERR_UNSUPPORTED;
    int st = check_csr(A, true);
    if (st) return st;
    if ((st = check_csr(B, true))) return st;
    if ((st = check_csr(C, true))) return st;
    if (A->cols != B->rows) return SMASH_ERR_SHAPE_MISMATCH;
    if (C->rows != A->rows || C->cols != B->cols) return SMASH_ERR_SHAPE_MISMATCH;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->rows;
    memset(&h->stats, 0, sizeof(h->stats));
    h->stats.c_nnz = C->nnz;
    if (n == 0 || C->nnz == 0) return SMASH_OK;
    Plan pl;
    if ((st = plan_buffers(h, n, false, s, pl))) return st;
    const RawOperands op = raw_ops(A, B);
    const int dt = dtype == SMASH_F64 ? 1 : 0;
    const BinRule rule = num_rule(h, B->cols, dt);
    int *err = (int *)h->err.ptr;
    {
        LaunchTimer lt(h, s, "num_rowinfo", -1, 256, n, A->nnz, 0, C->nnz);
        launch_num_rowinfo(op, C->row_ptr, C->nnz, rule, pl.bb, err, h->sms, s);
    }
    {
        LaunchTimer lt(h, s, "bin_scatter", -1, 256, n, 0, 0, 0);
        launch_bin_scatter(n, pl.bb, s);
    }
    if ((st = last_cuda_status())) return st;
    int counts[16], offsets[17];
    long long maxsize[16], stats[4], sums[48];
    if ((st = fetch_bins(h, pl, s, counts, offsets, maxsize, stats, sums))) return st;
    h->stats.c_nnz = C->nnz;
    const NumOut out{C->row_ptr, C->col_idx, C->val, C->nnz};
    const size_t vsz = dt ? 8 : 4;
    for (int b = 1; b < kNumBins; ++b) {
        if (!counts[b]) continue;
        const int *rows = pl.bb.rows + offsets[b];
        int *tok = pl.bb.tokens + b;
        if (b == kBinDense) {
            const HashLaunch hl = hash_launch(h, 0, B->cols);
            void *acc = nullptr;
            const int H = h->params.hot_cols;
            int cs = num_dense_cluster_size(dt, (int)B->cols, h->params.cluster_max, H);
            BSlices sl;
            if (cs == 0) {
                const size_t need = (size_t)num_dense_grid(dt, hl, (int)B->cols) * (size_t)B->cols * vsz;
                if ((st = ensure(h, h->dense_acc, need, s, true))) return st;
                acc = h->dense_acc.ptr;
            } else {
                const int cap = num_dense_cap(dt, H);
                int cpc = cap;
                if (cs == 1) cpc = (int)((B->cols + 31) & ~31ll);
                const size_t need = dense_plan_bytes(op, cs, cpc, H, vsz);
                if ((st = ensure(h, h->split, need, s))) return st;
                LaunchTimer lt(h, s, "dense_plan", -1, 256, B->rows, A->nnz, 0, B->nnz);
                launch_dense_plan(dt, op, cs, cap, cpc, H, h->params.hot_factor, h->split.ptr, sl, h->sms, s);
                sl.nslices = cs;
                sl.cpc = cpc;
            }
            LaunchTimer lt(h, s, cs ? "num_dense_cluster" : "num_dense_global", b, 1024, counts[b], sums[b],
                           sums[16 + b], sums[32 + b]);
            launch_num_dense(dt, op, rows, counts[b], tok, hl, acc, sl, out, err, s);
        } else if (b == kBinSpill) {
            const int tb = table_bits(maxsize[b], rule.inv_load);
            const HashLaunch hl = hash_launch(h, tb, B->cols);
            const size_t need = ((size_t)num_spill_grid(dt, hl) << tb) * (4 + vsz);
            if ((st = ensure(h, h->tables, need, s))) return st;
            LaunchTimer lt(h, s, "num_spill", b, 1024, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_num_spill(dt, op, rows, counts[b], tok, hl, rule.inv_load, tb, h->tables.ptr, out, err, s);
        } else {
            const HashLaunch hl = hash_launch(h, tbits_of_bin(b), B->cols);
            LaunchTimer lt(h, s, "num_hash", b, group_threads(hl), counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_num_hash(dt, op, rows, counts[b], tok, hl, rule.inv_load, h->params.bitmap_ratio, out, err, s);
        }
        if ((st = last_cuda_status())) return st;
    }
    return SMASH_OK;
}

}  // extern "C"
