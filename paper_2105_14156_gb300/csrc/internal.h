// Host-side internals shared by the C ABI translation units: the handle,
// scratch-memory management, launch timing and the row planner.
//
// The planner follows the paper's Window Distribution Phase: count each row's
// products from the row pointers, decide dense or sparse per row by a
// threshold, and group rows so that each group's tables fit on-chip memory
// (here: one block's shared memory instead of a PIUMA block's scratchpad).
#pragma once

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


namespace smash {

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Event timing of kernel launches (tracing).
struct PendingTime {
    int slot;  // index into totals
    cudaEvent_t e0, e1;
};

}  // namespace smash

struct smash_handle {
    bool timing = false;
    std::vector<smash::PendingTime> pending;
    std::vector<smash_kernel_time> totals;
    std::vector<cudaEvent_t> spare_events;
    int device = 0;
    int sms = 0;
    smash_params params{};
    smash_alloc_fn alloc = nullptr;
    smash_free_fn free_fn = nullptr;
    void *ctx = nullptr;
    smash::DevBuf ws;         // per-call arrays
    smash::DevBuf tables;     // spill hash tables
    smash::DevBuf split;      // dense rows: slices of B by column window, item counter
    smash::DevBuf wslot;      // dense rows: count slot per row of A (-1: none)
    smash::DevBuf wcnt;       // dense rows: distinct columns per kSubCols block, per slot (uint16)
    // What wslot / wcnt describe: the structure of the (A, B) pair whose dense
    // rows they count (device pointers and sizes), the number of column blocks
    // and the slots in use. Set by the symbolic phase, extended by numeric
    // count passes, cleared by calls that may change the structure.
    struct {
        bool valid = false;
        const void *ptr[4] = {nullptr, nullptr, nullptr, nullptr};
        int64_t dims[5] = {0, 0, 0, 0, 0};
        int nsub = 0;
        int64_t slots = 0;
    } wcache;
    // The slices of B by column window last built in h->split (reused within
    // one call only: B's values may change between calls).
    struct {
        bool valid = false;
        const void *b_rp = nullptr, *b_ci = nullptr, *b_val = nullptr;
        int64_t b_nnz = 0, b_rows = 0, ncols = 0;
        int cpc = 0, nw = 0, per = 1, dt = 0;
        smash::BSlices sl;
    } plan_cache;
    // Per-row counts (flop_i, nnz(A_i), longest row of B) recorded by the last
    // full symbolic planning, for the numeric planning of the same operands.
    smash::DevBuf rcache;
    struct {
        bool valid = false;
        const void *ptr[4] = {nullptr, nullptr, nullptr, nullptr};
        int64_t dims[5] = {0, 0, 0, 0, 0};
    } rkey;
    smash::DevBuf stage;      // learned path: capacity-padded staging of C
    smash::DevBuf arena;      // learned path: dense rows' windows
    smash::DevBuf learn;      // learned path: per-row arrays
    smash::DevBuf err;        // kNumErr ints (+ scratch words)
    long long *host = nullptr;  // pinned host staging (mapped)
    long long *host_dev = nullptr;  // the same buffer as the kernels see it
    smash_stats stats{};
    // Streams that run the bins of one phase side by side (created on first
    // use): a bin's kernel starts on SMs that the kernels before it release,
    // so the tails of the large bins and the small bins overlap.
    static constexpr int kAux = 3;
    cudaStream_t aux[kAux] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kAux] = {nullptr, nullptr, nullptr};
};

namespace smash {
namespace host {

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

inline void *default_alloc(size_t bytes, void *) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
inline void default_free(void *p, void *) { cudaFree(p); }

inline int release(smash_handle *h, DevBuf &b) {
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
inline int ensure(smash_handle *h, DevBuf &b, size_t need, cudaStream_t s, bool zero = false) {
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

// Grow-only buffer whose first `keep` bytes survive the growth.
inline int ensure_keep(smash_handle *h, DevBuf &b, size_t need, size_t keep, cudaStream_t s) {
    if (need == 0) need = 256;
    if (b.bytes >= need) return SMASH_OK;
    size_t want = need + need / 4;
    want = (want + 4095) & ~size_t(4095);
    void *p = h->alloc(want, h->ctx);
    if (!p) return SMASH_ERR_ALLOC;
    if (keep > b.bytes) keep = b.bytes;
    if (keep && b.ptr && cudaMemcpyAsync(p, b.ptr, keep, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        h->free_fn(p, h->ctx);
        return SMASH_ERR_CUDA;
    }
    cudaStreamSynchronize(s);
    if (b.ptr) h->free_fn(b.ptr, h->ctx);
    b.ptr = p;
    b.bytes = want;
    return SMASH_OK;
}

// Identity of the structure of an operand pair, for the dense-row counts.
inline bool wcache_matches(const smash_handle *h, const RawOperands &op) {
    const auto &c = h->wcache;
    return c.valid && c.ptr[0] == op.a_rp && c.ptr[1] == op.a_ci && c.ptr[2] == op.b_rp && c.ptr[3] == op.b_ci &&
           c.dims[0] == op.a_rows && c.dims[1] == op.a_nnz && c.dims[2] == op.b_rows && c.dims[3] == op.b_nnz &&
           c.dims[4] == op.ncols;
}

inline void wcache_set(smash_handle *h, const RawOperands &op, int nsub, int64_t slots) {
    auto &c = h->wcache;
    c.valid = true;
    c.ptr[0] = op.a_rp;
    c.ptr[1] = op.a_ci;
    c.ptr[2] = op.b_rp;
    c.ptr[3] = op.b_ci;
    c.dims[0] = op.a_rows;
    c.dims[1] = op.a_nnz;
    c.dims[2] = op.b_rows;
    c.dims[3] = op.b_nnz;
    c.dims[4] = op.ncols;
    c.nsub = nsub;
    c.slots = slots;
}

// Identity of the operands whose per-row counts h->rcache holds.
inline bool rcache_matches(const smash_handle *h, const RawOperands &op) {
    const auto &c = h->rkey;
    return c.valid && c.ptr[0] == op.a_rp && c.ptr[1] == op.a_ci && c.ptr[2] == op.b_rp && c.ptr[3] == op.b_ci &&
           c.dims[0] == op.a_rows && c.dims[1] == op.a_nnz && c.dims[2] == op.b_rows && c.dims[3] == op.b_nnz &&
           c.dims[4] == op.ncols;
}

inline void rcache_set(smash_handle *h, const RawOperands &op) {
    auto &c = h->rkey;
    c.valid = true;
    c.ptr[0] = op.a_rp;
    c.ptr[1] = op.a_ci;
    c.ptr[2] = op.b_rp;
    c.ptr[3] = op.b_ci;
    c.dims[0] = op.a_rows;
    c.dims[1] = op.a_nnz;
    c.dims[2] = op.b_rows;
    c.dims[3] = op.b_nnz;
    c.dims[4] = op.ncols;
}

inline cudaEvent_t take_event(smash_handle *h) {
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
                long long a_nnz, long long products, long long c_nnz, int kernels = 1)
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
        kt.kernels += kernels;
        e0 = take_event(h);
        cudaEventRecord(e0, s);
    }
    // kernels known only once launched
    void add_kernels(int k) {
        if (h->timing && slot >= 0) h->totals[slot].kernels += k;
    }
    ~LaunchTimer() {
        if (!h->timing || slot < 0) return;
        cudaEvent_t e1 = take_event(h);
        cudaEventRecord(e1, s);
        h->pending.push_back(PendingTime{slot, e0, e1});
    }
};

inline void resolve_timings(smash_handle *h) {
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
inline size_t carve_size(size_t &acc, size_t count) {
    acc = (acc + 255) & ~size_t(255);
    acc += count * sizeof(T);
    return acc;
}

inline int status_from_flags(const long long *flags_as_ll) {
    const int *f = (const int *)flags_as_ll;
    if (f[kErrBadIndex] || f[kErrBadRowPtr] || f[kErrCountMismatch]) return SMASH_ERR_INVALID_ARG;
    if (f[kErrBRowTooLong]) return SMASH_ERR_UNSUPPORTED;
    if (f[kErrTimeout]) return SMASH_ERR_TIMEOUT;
    if (f[kErrTableFull]) return SMASH_ERR_INTERNAL;
    return SMASH_OK;
}

inline int check_params(const smash_params *p) {
    if (!p) return SMASH_ERR_INVALID_ARG;
    if (p->hash_kind < 0 || p->hash_kind > 2) return SMASH_ERR_INVALID_ARG;
    if (!(p->max_load > 0.05f && p->max_load <= 0.95f)) return SMASH_ERR_INVALID_ARG;
    if (p->sym_max_tbits < kMinTBits || p->sym_max_tbits > 15) return SMASH_ERR_INVALID_ARG;
    if (p->num_max_tbits < kMinTBits || p->num_max_tbits > 14) return SMASH_ERR_INVALID_ARG;
    if (p->group_shift < 0 || p->group_shift > 10) return SMASH_ERR_INVALID_ARG;
    if (p->dense_ratio < 0 || p->bitmap_ratio < 0) return SMASH_ERR_INVALID_ARG;
    if (p->spill_blocks_per_sm < 0 || p->spill_blocks_per_sm > 8) return SMASH_ERR_INVALID_ARG;
    if (p->sym_dense_ratio < 0) return SMASH_ERR_INVALID_ARG;
    if (p->dense_blocks != 0 && p->dense_blocks != 1 && p->dense_blocks != 2 && p->dense_blocks != 4)
        return SMASH_ERR_INVALID_ARG;
    if (p->sym_dense_blocks != 0 && p->sym_dense_blocks != 1 && p->sym_dense_blocks != 2 &&
        p->sym_dense_blocks != 4 && p->sym_dense_blocks != 8)
        return SMASH_ERR_INVALID_ARG;
    if (p->warp_rows != 0 && p->warp_rows != 1) return SMASH_ERR_INVALID_ARG;
    if (p->bulk_copy != 0 && p->bulk_copy != 1) return SMASH_ERR_INVALID_ARG;
    if (p->group_rows != 0 && p->group_rows != 1) return SMASH_ERR_INVALID_ARG;
    if (p->row_window != 0 && (p->row_window < 2 || p->row_window > 32)) return SMASH_ERR_INVALID_ARG;
    if (p->row_window_tbits < kMinTBits || p->row_window_tbits > 8) return SMASH_ERR_INVALID_ARG;
    if (p->dense_owner != 0 && p->dense_owner != 1) return SMASH_ERR_INVALID_ARG;
    return SMASH_OK;
}

inline int check_csr(const smash_csr *M, bool need_val) {
    if (!M) return SMASH_ERR_INVALID_ARG;
    if (M->rows < 0 || M->cols < 0 || M->nnz < 0) return SMASH_ERR_INVALID_ARG;
    if (M->rows >= (1ll << 31) || M->cols >= (1ll << 31)) return SMASH_ERR_UNSUPPORTED;
    if (!M->row_ptr) return SMASH_ERR_INVALID_ARG;
    if (M->nnz > 0 && !M->col_idx) return SMASH_ERR_INVALID_ARG;
    if (need_val && M->nnz > 0 && !M->val) return SMASH_ERR_INVALID_ARG;
    return SMASH_OK;
}

inline int colbits_of(int64_t ncols) {
    int b = 0;
    while ((1ll << b) < ncols) ++b;
    return b;
}

inline RawOperands raw_ops(const smash_csr *A, const smash_csr *B) {
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

inline int plan_buffers(smash_handle *h, int64_t n, bool symbolic, cudaStream_t s, Plan &pl) {
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

// Reads `bytes` (a multiple of 4) of device memory at src into the handle's
// pinned host buffer at byte offset off, by a kernel that writes the mapped
// buffer: no copy engine, so a small read never queues behind the caller's
// bulk copies on other streams. Does not wait.
inline int read_small(smash_handle *h, size_t off, const void *src, size_t bytes, cudaStream_t s) {
    LaunchTimer lt(h, s, "read_small", -1, 256, 0, 0, 0, 0);
    launch_read_small(src, (char *)h->host_dev + off, bytes, s);
    return cudaPeekAtLastError() == cudaSuccess ? SMASH_OK : SMASH_ERR_CUDA;
}

// Copy bin counts (16 int), offsets (17 int), maxsize (16 ll), stats (4 ll)
// to the pinned host buffer and wait.
inline int fetch_bins(smash_handle *h, const Plan &pl, cudaStream_t s, int *counts, int *offsets, long long *maxsize,
               long long *stats, long long *sums) {
    char *hb = (char *)h->host;
    if (read_small(h, 0, pl.bb.counts, 16 * sizeof(int), s) || read_small(h, 64, pl.bb.offsets, 17 * sizeof(int), s) ||
        read_small(h, 256, pl.bb.maxsize, 20 * sizeof(long long), s) ||
        read_small(h, 512, pl.bb.sums, 48 * sizeof(long long), s))
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

inline int read_flags(smash_handle *h, cudaStream_t s, bool clear) {
    char *hb = (char *)h->host + 1024;
    if (read_small(h, 1024, h->err.ptr, kNumErr * sizeof(int), s)) return SMASH_ERR_CUDA;
    if (clear && cudaMemsetAsync(h->err.ptr, 0, kNumErr * sizeof(int), s) != cudaSuccess) return SMASH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SMASH_ERR_CUDA;
    const int st = status_from_flags((const long long *)hb);
    // after a failure the kept counts may not describe the inputs any more
    if (st != SMASH_OK) {
        h->wcache.valid = false;
        h->rkey.valid = false;
    }
    return st;
}

// Fork of the caller's stream s into s and the handle's auxiliary streams for
// the launches of one phase, joined back into s when the Fork goes out of
// scope. Buffers that more than one of the forked launches use must be
// allocated before the fork.
struct Fork {
    smash_handle *h;
    cudaStream_t s;
    int n = 1;   // streams in use: s and n - 1 auxiliary ones
    Fork(smash_handle *hh, cudaStream_t ss) : h(hh), s(ss) {
        bool ok = true;
        if (!h->fork_ev) ok = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < smash_handle::kAux; ++k) {
            if (!h->aux[k]) ok = cudaStreamCreateWithFlags(&h->aux[k], cudaStreamNonBlocking) == cudaSuccess;
            if (ok && !h->join_ev[k]) ok = cudaEventCreateWithFlags(&h->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            return;   // everything on s
        }
        if (cudaEventRecord(h->fork_ev, s) != cudaSuccess) return;
        for (int k = 0; k < smash_handle::kAux; ++k) cudaStreamWaitEvent(h->aux[k], h->fork_ev, 0);
        n = 1 + smash_handle::kAux;
    }
    cudaStream_t get(int k) const { return (k % n) == 0 ? s : h->aux[(k % n) - 1]; }
    ~Fork() {
        for (int k = 0; k + 1 < n; ++k) {
            cudaEventRecord(h->join_ev[k], h->aux[k]);
            cudaStreamWaitEvent(s, h->join_ev[k], 0);
        }
    }
};

inline void destroy_streams(smash_handle *h) {
    for (int k = 0; k < smash_handle::kAux; ++k) {
        if (h->aux[k]) cudaStreamDestroy(h->aux[k]);
        if (h->join_ev[k]) cudaEventDestroy(h->join_ev[k]);
        h->aux[k] = nullptr;
        h->join_ev[k] = nullptr;
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    h->fork_ev = nullptr;
}

// Order in which the bins of a phase are launched (round-robin over the
// streams): largest tables first (the dense and spill bins, then the shared
// bins from the largest down), so that the kernels whose blocks each hold a
// long row start early and the many short blocks of the small bins fill the
// end, rather than a few long blocks running alone at the end of the phase.
inline int bin_order(const long long *sums, int *order) {
    int n = 0;
    for (int b = 1; b < kNumBins; ++b) order[n++] = b;
    auto key = [&](int b) { return sums[16 + b] > 0 ? (long long)b : -1ll; };
    for (int x = 1; x < n; ++x)
        for (int y = x; y > 0 && key(order[y]) > key(order[y - 1]); --y) {
            const int t = order[y];
            order[y] = order[y - 1];
            order[y - 1] = t;
        }
    return n;
}

inline int last_cuda_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMASH_OK : SMASH_ERR_CUDA;
}

// Resident blocks per SM of the numeric dense kernel.
inline int dense_blocks_of(const smash_handle *h, int dtype) {
    const int b = h->params.dense_blocks;
    return b > 0 ? b : (dtype ? 2 : 4);
}

// A thread-per-row bin pays only with enough rows to fill the GPU (its rows'
// dependent loads are hidden by other rows, not by other lanes of a row):
// fewer rows than one 128-thread block per SM take the warp-per-row hash.
inline int tiny_min_rows(const smash_handle *h) { return h->sms * 128; }

// The thread-per-row kernel keeps the 32-slot bins that have enough rows in
// both phases (measured faster there than row windows); row windows take the
// symbolic 64-slot bin before it.
inline bool tiny_first(const smash_handle *h, const BinRule &r, int bin, int count) {
    const int tb = tbits_of_bin(bin);
    return tb <= r.tiny_tbits && tb <= kTinyNumTBits && count >= tiny_min_rows(h);
}

inline BinRule sym_rule(const smash_handle *h, int64_t ncols) {
    BinRule r;
    r.inv_load = 1.0f / h->params.max_load;
    int mt = h->params.sym_max_tbits;
    // key-only table of 2^mt ints plus the staging of a 1024-thread group
    while (mt > kMinTBits && ((size_t)4 << mt) + 24 * 1024 > (size_t)max_smem_per_block()) --mt;
    r.max_tbits = mt;
    r.dense_ok = (h->params.sym_dense_ratio > 0 && ncols <= dense_bitmap_max_cols()) ? 1 : 0;
    r.dense_min = r.dense_ok ? (ncols + h->params.sym_dense_ratio - 1) / h->params.sym_dense_ratio : (1ll << 62);
    if (r.dense_min < 1) r.dense_min = 1;
    r.tiny_tbits = kTinySymTBits;
    return r;
}

inline BinRule num_rule(const smash_handle *h, int64_t ncols, int dtype) {
    BinRule r;
    r.inv_load = 1.0f / h->params.max_load;
    // dense rows need their columns counted in one bitmap (count pass) and a
    // column window that fits shared memory
    const bool dense_fits = ncols <= dense_bitmap_max_cols() && num_window_cols(dtype, dense_blocks_of(h, dtype), false) > 0;
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
    r.tiny_tbits = kTinyNumTBits;
    return r;
}

inline int group_threads(const HashLaunch &hl) {
    int t = 1 << (hl.tbits > hl.group_shift ? hl.tbits - hl.group_shift : 0);
    return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

// Whether a bin of tables of 2^hl.tbits slots runs the register-enumerating
// warp-row kernel (k_warp.cuh): one warp per row, and its shared memory fits.
// dtype < 0: the symbolic phase.
inline bool use_warp_rows(const smash_handle *h, const HashLaunch &hl, int dtype) {
    if (!h->params.warp_rows || group_threads(hl) != 32) return false;
    const size_t need = dtype < 0 ? sym_warp_smem(hl.tbits) : num_warp_smem(dtype, hl.tbits, 1.0f / h->params.max_load);
    return need <= (size_t)max_smem_per_block();
}

// Whether a bin runs the numeric group-row kernel (k_group.cuh): a block of
// 64 or more threads per row, and its shared memory fits.
inline bool use_group_rows(const smash_handle *h, const HashLaunch &hl, int dtype) {
    if (!h->params.group_rows || group_threads(hl) < 64) return false;
    return num_group_smem(dtype, hl.tbits, 1.0f / h->params.max_load, hl.group_shift) <=
           (size_t)max_smem_per_block();
}

// The row window of the bin of tables of 2^tbits slots (false: the bin takes
// another kernel). A row of the bin holds at most L = T / inv_load columns;
// a window takes W <= row_window rows with W * L <= 256 and tags of at most
// 31 bits. dtype < 0: the symbolic phase.
inline bool row_window_of(const smash_handle *h, int tbits, int64_t ncols, int dtype, RowWin &rw) {
    if (h->params.row_window < 2 || tbits > h->params.row_window_tbits) return false;
    const int T = 1 << tbits;
    const double inv = (double)(1.0f / h->params.max_load);
    int L = (int)((double)T / inv + 1e-9);
    L = L < 1 ? 1 : (L > T ? T : L);
    int W = h->params.row_window;
    if (W * L > 256) W = 256 / L;
    const int cb = colbits_of(ncols);
    if (cb > 30) return false;
    while (W > (1 << (31 - cb))) W >>= 1;
    if (W < 2) return false;
    int wbits = 0;
    while ((1 << wbits) < W) ++wbits;
    int tw = 0;
    while ((1 << tw) < W * T) ++tw;
    rw.W = W;
    rw.wbits = wbits;
    rw.cb = cb;
    rw.tbits = tw;
    rw.lcap = (W * L + 31) & ~31;
    rw.ts = (1 << tw) > 2 * rw.lcap ? (1 << tw) : 2 * rw.lcap;
    rw.nb = 1 << (tw - 1);
    rw.bsh = cb + wbits > tw - 1 ? cb + wbits - (tw - 1) : 0;
    const size_t need = dtype < 0 ? sym_rowwin_smem(rw) : num_rowwin_smem(rw, dtype);
    return need <= (size_t)max_smem_per_block();
}

inline HashLaunch hash_launch(const smash_handle *h, int tbits, int64_t ncols) {
    HashLaunch hl;
    hl.tbits = tbits;
    hl.group_shift = h->params.group_shift;
    hl.hash_kind = h->params.hash_kind;
    hl.colbits = colbits_of(ncols);
    hl.sms = h->sms;
    hl.blocks_per_sm = h->params.spill_blocks_per_sm > 0 ? h->params.spill_blocks_per_sm : 1;
    hl.dense_blocks = h->params.dense_blocks > 0 ? h->params.dense_blocks : 2;
    hl.sym_dense_blocks = h->params.sym_dense_blocks;
    return hl;
}

}  // namespace host
}  // namespace smash

namespace smash {
namespace host {

// Bin drivers (api.cu). They plan the rows of A (all rows, or the rows of
// row_list), scatter them into bins and launch one kernel per non-empty bin.
//   run_symbolic: writes the exact count of every planned row to nnz_out.
//   run_numeric:  fills the planned rows of `out` (exact or capacity mode);
//                 c_rp gives each planned row its size.
int run_symbolic(smash_handle *h, const RawOperands &op, int64_t n, Plan &pl, int *nnz_out, cudaStream_t s,
                 const int *row_list, int64_t list_n);
int run_numeric(smash_handle *h, const RawOperands &op, int64_t n, int dt, const NumOut &out, Plan &pl,
                cudaStream_t s, const int *row_list, int64_t list_n);
// The two halves of run_numeric: bins of the planned rows (fetched to the
// host), then one launch per bin. arena != nullptr: the dense bin runs in
// arena mode (capacity mode only).
struct BinPlan {
    int counts[16], offsets[17];
    long long maxsize[16], stats[4], sums[48];
};
// cap_rec (capacity mode): the rows' counts from the learned planning.
int run_bins(smash_handle *h, const RawOperands &op, int64_t n, int dt, const NumOut &out, Plan &pl,
             const BinPlan &bp, cudaStream_t s, const WinArena *arena, const RowGather *cap_rec = nullptr);
// Whether the dense bin (with `products` products) takes column windows, and
// their width and number.
// Whether the dense rows take column windows (cpc columns, nw windows, per
// slices of B per window: > 1 when each warp owns a slice).
bool dense_windows(const smash_handle *h, const RawOperands &op, int dt, long long products, int &cpc, int &nw,
                   int &per);

}  // namespace host
}  // namespace smash

namespace smash {
namespace host {
// Releases the batched path's per-handle state (batched.cu).
void batched_release(smash_handle *h);
}  // namespace host
}  // namespace smash
