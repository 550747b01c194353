// C ABI: handle, parameters, the symbolic and numeric phases.
#include "internal.h"

using namespace smash;
using namespace smash::host;

// ---------------------------------------------------------------------------
extern "C" {

int smash_default_params(smash_params *p) {
    if (!p) return SMASH_ERR_INVALID_ARG;
    memset(p, 0, sizeof(*p));
    p->hash_kind = 1;
    p->max_load = 0.5f;
    p->sym_max_tbits = 15;
    p->num_max_tbits = 14;
    p->group_shift = 4;
    p->dense_ratio = 4;
    p->bitmap_ratio = 4;
    p->spill_blocks_per_sm = 1;
    p->sym_dense_ratio = 64;
    p->dense_blocks = 0;
    p->sym_dense_blocks = 0;
    p->warp_rows = 1;
    p->bulk_copy = 0;
    p->group_rows = 0;
    p->row_window = 16;
    p->row_window_tbits = 7;
    p->dense_owner = 0;
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
    if (cudaHostAlloc((void **)&h->host, kHostWords * 8 * 8, cudaHostAllocMapped) != cudaSuccess) {
        delete h;
        return SMASH_ERR_ALLOC;
    }
    if (cudaHostGetDevicePointer((void **)&h->host_dev, h->host, 0) != cudaSuccess) {
        cudaFreeHost(h->host);
        delete h;
        return SMASH_ERR_CUDA;
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
        release(h, h->split);
        release(h, h->wslot);
        release(h, h->wcnt);
        release(h, h->stage);
        release(h, h->arena);
        release(h, h->learn);
        release(h, h->rcache);
        batched_release(h);
        release(h, h->err);
        destroy_streams(h);
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
    release(h, h->split);
    release(h, h->wslot);
    release(h, h->wcnt);
    release(h, h->stage);
    release(h, h->arena);
    release(h, h->learn);
    release(h, h->rcache);
    h->rkey.valid = false;
    h->wcache.valid = false;
    batched_release(h);
    // the error words move to the new allocator as well
    release(h, h->err);
    h->alloc = alloc ? alloc : default_alloc;
    h->free_fn = free_fn ? free_fn : default_free;
    h->ctx = alloc ? ctx : nullptr;
    int st = SMASH_OK;
    if (ensure(h, h->err, 256, 0) != SMASH_OK) {
        // the handle stays usable: back to cudaMalloc / cudaFree
        st = SMASH_ERR_ALLOC;
        h->alloc = default_alloc;
        h->free_fn = default_free;
        h->ctx = nullptr;
        if (ensure(h, h->err, 256, 0) != SMASH_OK) return SMASH_ERR_ALLOC;
    }
    if (cudaMemset(h->err.ptr, 0, h->err.bytes) != cudaSuccess) return SMASH_ERR_CUDA;
    return st;
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
    if ((st = run_symbolic(h, op, n, pl, pl.nnz, s, nullptr, 0))) return st;
    {
        LaunchTimer lt(h, s, "scan_rowptr", -1, 512, n, 0, 0, 0, 3);
        launch_scan_rowptr(pl.nnz, n, c_row_ptr, pl.total, pl.scan, s);
    }
    if ((st = last_cuda_status())) return st;
    if (read_small(h, 0, pl.total, sizeof(long long), s)) return SMASH_ERR_CUDA;
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
    h->plan_cache.valid = false;   // B's values may have changed since the last call
    if (n == 0 || C->nnz == 0) return SMASH_OK;
    Plan pl;
    if ((st = plan_buffers(h, n, false, s, pl))) return st;
    const RawOperands op = raw_ops(A, B);
    const int dt = dtype == SMASH_F64 ? 1 : 0;
    NumOut out;
    out.c_rp = C->row_ptr;
    out.c_ci = C->col_idx;
    out.c_val = C->val;
    out.c_nnz = C->nnz;
    if ((st = run_numeric(h, op, n, dt, out, pl, s, nullptr, 0))) return st;
    h->stats.c_nnz = C->nnz;
    return SMASH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
namespace smash {
namespace host {

int run_symbolic(smash_handle *h, const RawOperands &op, int64_t n, Plan &pl, int *nnz_out, cudaStream_t s,
                 const int *row_list, int64_t list_n) {
    int st;
    const BinRule rule = sym_rule(h, op.ncols);
    int *err = (int *)h->err.ptr;
    h->wcache.valid = false;
    if (row_list && cudaMemsetAsync(pl.bb.bin, 0, (size_t)n, s) != cudaSuccess) return SMASH_ERR_CUDA;
    // a full planning records the rows' counts for the numeric phase
    RowGather *keep = nullptr;
    if (!row_list) {
        h->rkey.valid = false;
        if ((st = ensure(h, h->rcache, sizeof(RowGather) * (size_t)n, s))) return st;
        keep = (RowGather *)h->rcache.ptr;
    }
    {
        LaunchTimer lt(h, s, "sym_rowinfo", -1, 256, row_list ? list_n : n, op.a_nnz, 0, 0, 2);
        launch_sym_rowinfo(op, rule, pl.bb, pl.bound, nnz_out, err, h->sms, s, row_list, list_n, keep);
    }
    if (keep) rcache_set(h, op);
    {
        LaunchTimer lt(h, s, "bin_scatter", -1, 256, n, 0, 0, 0);
        launch_bin_scatter(n, pl.bb, s);
    }
    if ((st = last_cuda_status())) return st;
    int counts[16], offsets[17];
    long long maxsize[16], stats[4], sums[48];
    if ((st = fetch_bins(h, pl, s, counts, offsets, maxsize, stats, sums))) return st;
    // buffers of the dense and spill bins, before the launches fork
    const int nsub = (int)((op.ncols + kSubCols - 1) / kSubCols);
    int spill_tb = 0;
    if (counts[kBinDense]) {
        if ((st = ensure(h, h->wslot, sizeof(int) * (size_t)n, s))) return st;
        if ((st = ensure(h, h->wcnt, sizeof(uint16_t) * (size_t)counts[kBinDense] * nsub, s))) return st;
        if (cudaMemsetAsync(h->wslot.ptr, 0xff, sizeof(int) * (size_t)n, s) != cudaSuccess) return SMASH_ERR_CUDA;
    }
    if (counts[kBinSpill]) {
        spill_tb = table_bits(maxsize[kBinSpill], rule.inv_load);
        const HashLaunch hl = hash_launch(h, spill_tb, op.ncols);
        if ((st = ensure(h, h->tables, ((size_t)sym_spill_grid(hl) << spill_tb) * sizeof(int), s))) return st;
    }
    int order[kNumBins];
    const int nb = bin_order(sums, order);
    Fork fk(h, s);
    int q = 0;
    for (int x = 0; x < nb; ++x) {
        const int b = order[x];
        if (!counts[b]) continue;
        cudaStream_t bs = fk.get(q++);
        const int *rows = pl.bb.rows + offsets[b];
        int *tok = pl.bb.tokens + b;
        if (b == kBinDense) {
            // the bitmap pass also counts each row's columns per block of
            // kSubCols columns, for the numeric dense kernel
            WinCount wc;
            wc.wslot = (int *)h->wslot.ptr;
            wc.wcnt = (uint16_t *)h->wcnt.ptr;
            wc.nsub = nsub;
            {
                const HashLaunch hl = hash_launch(h, 0, op.ncols);
                LaunchTimer lt(h, bs, "sym_dense", b, sym_dense_threads(hl, op.ncols), counts[b], sums[b], sums[16 + b],
                               sums[32 + b]);
                launch_sym_dense(op, rows, counts[b], tok, hl, wc, nnz_out, NumCheck{}, err, bs);
            }
            wcache_set(h, op, nsub, counts[b]);
        } else if (b == kBinSpill) {
            const HashLaunch hl = hash_launch(h, spill_tb, op.ncols);
            LaunchTimer lt(h, bs, "sym_spill", b, 1024, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_sym_spill(op, rows, counts[b], tok, hl, rule.inv_load, pl.bound, spill_tb, (int *)h->tables.ptr,
                             nnz_out, err, bs);
        } else if (RowWin rw; !tiny_first(h, rule, b, counts[b]) && row_window_of(h, tbits_of_bin(b), op.ncols, -1, rw)) {
            const HashLaunch hl = hash_launch(h, tbits_of_bin(b), op.ncols);
            LaunchTimer lt(h, bs, "sym_rowwin", b, 128, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_sym_rowwin(op, rows, counts[b], tok, rw, hl, nnz_out, err, bs);
        } else if (tbits_of_bin(b) <= rule.tiny_tbits && counts[b] >= tiny_min_rows(h)) {
            LaunchTimer lt(h, bs, "sym_tiny", b, 128, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_sym_tiny(op, rows, counts[b], tbits_of_bin(b), h->params.max_load, h->sms, nnz_out, err, bs);
        } else {
            const HashLaunch hl = hash_launch(h, tbits_of_bin(b), op.ncols);
            if (use_warp_rows(h, hl, -1)) {
                LaunchTimer lt(h, bs, "sym_warp", b, 128, counts[b], sums[b], sums[16 + b], sums[32 + b]);
                launch_sym_warp(op, rows, counts[b], tok, hl, nnz_out, err, bs);
            } else {
                LaunchTimer lt(h, bs, "sym_hash", b, group_threads(hl), counts[b], sums[b], sums[16 + b],
                               sums[32 + b]);
                launch_sym_hash(op, rows, counts[b], tok, hl, nnz_out, err, bs);
            }
        }
        if ((st = last_cuda_status())) return st;
    }
    return SMASH_OK;
}

int run_numeric(smash_handle *h, const RawOperands &op, int64_t n, int dt, const NumOut &out, Plan &pl,
                cudaStream_t s, const int *row_list, int64_t list_n) {
    const BinRule rule = num_rule(h, op.ncols, dt);
    int *err = (int *)h->err.ptr;
    if (row_list && cudaMemsetAsync(pl.bb.bin, 0, (size_t)n, s) != cudaSuccess) return SMASH_ERR_CUDA;
    // the rows' counts from the symbolic phase of the same operands, if kept
    const RowGather *kept = rcache_matches(h, op) ? (const RowGather *)h->rcache.ptr : nullptr;
    {
        LaunchTimer lt(h, s, "num_rowinfo", -1, 256, row_list ? list_n : n, op.a_nnz, 0, out.c_nnz, kept ? 1 : 2);
        launch_num_rowinfo(op, out.c_rp, out.c_nnz, rule, pl.bb, err, h->sms, s, row_list, list_n, kept);
    }
    {
        LaunchTimer lt(h, s, "bin_scatter", -1, 256, n, 0, 0, 0);
        launch_bin_scatter(n, pl.bb, s);
    }
    int st;
    if ((st = last_cuda_status())) return st;
    BinPlan bp;
    if ((st = fetch_bins(h, pl, s, bp.counts, bp.offsets, bp.maxsize, bp.stats, bp.sums))) return st;
    return run_bins(h, op, n, dt, out, pl, bp, s, nullptr, nullptr);
}

bool dense_windows(const smash_handle *h, const RawOperands &op, int dt, long long products, int &cpc, int &nw,
                   int &per) {
    per = 1;
    if (op.b_nnz >= INT_MAX) return false;   // window bounds are int32 positions in B
    const int bps = dense_blocks_of(h, dt);
    const double vsz = dt ? 8.0 : 4.0;
    // slicing B costs a pass over its rows (and a copy when they are unsorted)
    auto pays = [&](long long nsl) {
        if (nsl > window_plan_max_slices()) return false;
        const double plan =
            nsl > 1 ? 4.0 * (double)op.b_rows * (double)(nsl + 1) + 2.0 * (4 + vsz) * (double)op.b_nnz : 0.0;
        return 16.0 * (double)products >= plan;
    };
    if (h->params.dense_owner) {
        const int c = num_window_cols(dt, bps, true);
        const int S = window_warps(bps);
        if (c > 0) {
            const int n = (int)((op.ncols + c - 1) / c);
            if (pays((long long)n * S)) {
                cpc = c;
                nw = n;
                per = S;
                return true;
            }
        }
    }
    cpc = num_window_cols(dt, bps, false);
    if (cpc <= 0) return false;
    nw = (int)((op.ncols + cpc - 1) / cpc);
    return pays(nw);
}

int window_plan(smash_handle *h, const RawOperands &op, int dt, int cpc, int nw, int per, cudaStream_t s,
                BSlices &sl) {
    auto &pc = h->plan_cache;
    if (pc.valid && pc.b_rp == op.b_rp && pc.b_ci == op.b_ci && pc.b_val == op.b_val && pc.b_nnz == op.b_nnz &&
        pc.b_rows == op.b_rows && pc.ncols == op.ncols && pc.cpc == cpc && pc.nw == nw && pc.per == per &&
        pc.dt == dt) {
        sl = pc.sl;
        return SMASH_OK;
    }
    const size_t vsz = dt ? 8 : 4;
    const void *before = h->split.ptr;
    int st;
    if ((st = ensure(h, h->split, 256 + window_plan_bytes(op, nw * per, vsz), s))) return st;
    (void)before;
    {
        LaunchTimer lt(h, s, "dense_plan", -1, 256, op.b_rows, 0, 0, op.b_nnz, 0);
        lt.add_kernels(launch_window_plan(dt, op, nw, per, cpc, (char *)h->split.ptr + 256, sl, h->sms, s,
                                          (int *)((char *)h->host + 1536), (int *)((char *)h->host_dev + 1536)));
    }
    pc.valid = true;
    pc.b_rp = op.b_rp;
    pc.b_ci = op.b_ci;
    pc.b_val = op.b_val;
    pc.b_nnz = op.b_nnz;
    pc.b_rows = op.b_rows;
    pc.ncols = op.ncols;
    pc.cpc = cpc;
    pc.nw = nw;
    pc.per = per;
    pc.dt = dt;
    pc.sl = sl;
    return SMASH_OK;
}

int run_bins(smash_handle *h, const RawOperands &op, int64_t n, int dt, const NumOut &out, Plan &pl,
             const BinPlan &bp, cudaStream_t s, const WinArena *arena, const RowGather *cap_rec) {
    int st;
    const BinRule rule = num_rule(h, op.ncols, dt);
    int *err = (int *)h->err.ptr;
    const int *counts = bp.counts;
    const int *offsets = bp.offsets;
    const long long *maxsize = bp.maxsize;
    const long long *sums = bp.sums;
    const size_t vsz = dt ? 8 : 4;
    // the rows' product counts kept by the symbolic phase of these operands
    // (capacity mode: the counts of the learned planning)
    const RowGather *kept =
        out.row_nnz ? cap_rec : (rcache_matches(h, op) ? (const RowGather *)h->rcache.ptr : nullptr);
    // Dense rows take column windows when their products pay for slicing B
    // (a pass over B's rows and entries); otherwise the global hash. Their
    // counts and the slices of B are prepared on s before the bins fork.
    const int bd = kBinDense;
    int cpc = 0, nw = 0, per = 1;
    const bool windows = counts[bd] && dense_windows(h, op, dt, sums[16 + bd], cpc, nw, per);
    HashLaunch hld = hash_launch(h, 0, op.ncols);
    hld.dense_blocks = dense_blocks_of(h, dt);
    WinCount wc;
    BSlices sl;
    if (windows) {
        if (!arena) {
            // 1. per-block column counts of the dense rows: from the symbolic
            //    phase of the same operands, else counted here (and sizes checked)
            const int nsub = (int)((op.ncols + kSubCols - 1) / kSubCols);
            if (!wcache_matches(h, op) || h->wcache.nsub != nsub) {
                if ((st = ensure(h, h->wslot, sizeof(int) * (size_t)n, s))) return st;
                if (cudaMemsetAsync(h->wslot.ptr, 0xff, sizeof(int) * (size_t)n, s) != cudaSuccess)
                    return SMASH_ERR_CUDA;
                wcache_set(h, op, nsub, 0);
            }
            const int64_t base = h->wcache.slots;
            if ((st = ensure_keep(h, h->wcnt, sizeof(uint16_t) * (size_t)(base + counts[bd]) * nsub,
                                  sizeof(uint16_t) * (size_t)base * nsub, s)))
                return st;
            wc.wslot = (int *)h->wslot.ptr;
            wc.wcnt = (uint16_t *)h->wcnt.ptr;
            wc.nsub = nsub;
            wc.slot_base = base;
            wc.skip_slotted = 1;
            NumCheck nc;
            nc.c_rp = out.c_rp;
            nc.c_nnz = out.c_nnz;
            nc.row_nnz = out.row_nnz;
            {
                LaunchTimer lt(h, s, "num_dense_count", bd, sym_dense_threads(hld, op.ncols), counts[bd], sums[bd],
                               sums[16 + bd], sums[32 + bd]);
                launch_sym_dense(op, pl.bb.rows + offsets[bd], counts[bd], pl.bb.tokens + bd, hld, wc, nullptr, nc,
                                 err, s);
            }
            h->wcache.slots = base + counts[bd];
        }
        // 2. column windows: slices of B
        if ((st = window_plan(h, op, dt, cpc, nw, per, s, sl))) return st;
    }
    // global-memory tables of the spill bin (and of dense rows without windows)
    int spill_tb = 0;
    for (int b : {(int)kBinSpill, (int)kBinDense}) {
        if (!counts[b] || (b == kBinDense && windows)) continue;
        const int tb = table_bits(maxsize[b], rule.inv_load);
        spill_tb = tb > spill_tb ? tb : spill_tb;
    }
    if (spill_tb) {
        const HashLaunch hl = hash_launch(h, spill_tb, op.ncols);
        if ((st = ensure(h, h->tables, ((size_t)num_spill_grid(dt, hl) << spill_tb) * (4 + vsz), s))) return st;
    }
    // both spill launches (when there are two) share the tables: one stream
    cudaStream_t spill_stream = nullptr;
    int order[kNumBins];
    const int nb = bin_order(sums, order);
    Fork fk(h, s);
    int q = 0;
    for (int x = 0; x < nb; ++x) {
        const int b = order[x];
        if (!counts[b]) continue;
        const int *rows = pl.bb.rows + offsets[b];
        int *tok = pl.bb.tokens + b;
        if (b == kBinDense && windows) {
            cudaStream_t bs = fk.get(q++);
            // (row, window) items
            LaunchTimer lt(h, bs, "num_dense_window", b, 1024 / hld.dense_blocks, counts[b], sums[b], sums[16 + b],
                           sums[32 + b]);
            launch_num_window(dt, op, rows, counts[b], (unsigned long long *)h->split.ptr, hld, sl, wc,
                              arena ? *arena : WinArena{}, out, err, bs);
        } else if (b == kBinSpill || b == kBinDense) {
            if (!spill_stream) spill_stream = fk.get(q++);
            cudaStream_t bs = spill_stream;
            const HashLaunch hl = hash_launch(h, spill_tb, op.ncols);
            LaunchTimer lt(h, bs, "num_spill", b, 1024, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_num_spill(dt, op, rows, counts[b], tok, hl, rule.inv_load, spill_tb, h->tables.ptr, out, err, bs);
        } else if (tbits_of_bin(b) <= rule.tiny_tbits && counts[b] >= tiny_min_rows(h)) {
            cudaStream_t bs = fk.get(q++);
            LaunchTimer lt(h, bs, "num_tiny", b, 128, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_num_tiny(dt, op, rows, counts[b], tbits_of_bin(b), h->params.max_load, h->sms, out, err, bs);
        } else if (RowWin rw; row_window_of(h, tbits_of_bin(b), op.ncols, dt, rw)) {
            cudaStream_t bs = fk.get(q++);
            const HashLaunch hl = hash_launch(h, tbits_of_bin(b), op.ncols);
            LaunchTimer lt(h, bs, "num_rowwin", b, 128, counts[b], sums[b], sums[16 + b], sums[32 + b]);
            launch_num_rowwin(dt, op, rows, counts[b], tok, rw, hl, kept, out, err, bs);
        } else {
            cudaStream_t bs = fk.get(q++);
            const HashLaunch hl = hash_launch(h, tbits_of_bin(b), op.ncols);
            if (use_warp_rows(h, hl, dt)) {
                LaunchTimer lt(h, bs, "num_warp", b, 128, counts[b], sums[b], sums[16 + b], sums[32 + b]);
                launch_num_warp(dt, op, rows, counts[b], tok, hl, rule.inv_load, kept, h->params.bulk_copy, out, err,
                                bs);
            } else if (op.b_nnz < INT_MAX && use_group_rows(h, hl, dt)) {
                LaunchTimer lt(h, bs, "num_group", b, group_threads(hl), counts[b], sums[b], sums[16 + b],
                               sums[32 + b]);
                launch_num_group(dt, op, rows, counts[b], tok, hl, rule.inv_load, kept, out, err, bs);
            } else {
                LaunchTimer lt(h, bs, "num_hash", b, group_threads(hl), counts[b], sums[b], sums[16 + b],
                               sums[32 + b]);
                launch_num_hash(dt, op, rows, counts[b], tok, hl, rule.inv_load, h->params.bitmap_ratio, kept, out, err,
                                bs);
            }
        }
        if ((st = last_cuda_status())) return st;
    }
    return SMASH_OK;
}

}  // namespace host
}  // namespace smash
