// C ABI of the batched path: many C_m = A_m * B_m in one persistent launch,
// plus the autotuner of its table size.
#include <algorithm>
#include <cstdio>
#include <map>

#include "batch_types.h"
#include "internal.h"

using namespace smash;
using namespace smash::host;

namespace {

// Host-pinned staging and device workspace of the batched call, kept in a
// per-handle side table (the handle struct is shared with other files).
struct BatchState {
    DevBuf dev;
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
    int tw_bits = 10;
    int warp_less = 0;               // warp rows: tables up to 2^(tw_bits - warp_less) slots
    int block_more = 3;              // block rows: tables up to 2^(tw_bits + block_more) slots
    long long wait_spins = 4000000;  // grid-barrier polls (x ~256 ns: about one second)
    int missing = 0;                 // test hook: barrier arrivals that never come
    cudaStream_t cs = nullptr;       // private stream for graph recording
    cudaGraph_t graph = nullptr;     // the recorded launch, replayed while its key holds
    cudaGraphExec_t exec = nullptr;
    // what the recorded launch depends on: argument buffer, grid, type, table size
    const void *key_args = nullptr;
    int key_grid = 0, key_dt = -1, key_bits = 0;
};
std::map<smash_handle *, BatchState> g_batch;

BatchState &state_of(smash_handle *h) { return g_batch[h]; }

void drop_graph(BatchState &b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
}

// The persistent launch (with the reset of its work tokens and barrier words)
// is recorded once as a CUDA graph and replayed on s; its arguments are
// copied to p_dev before each replay (p_host: pinned). It is recorded again
// when the argument buffer, grid, type or table size changes; a direct launch
// is the fallback if recording is not possible.
int run_batched_graph(BatchState &b, int dt, const BatchArgs *p_host, BatchArgs *p_dev, int grid, cudaStream_t s) {
    if (cudaMemcpyAsync(p_dev, p_host, sizeof(BatchArgs), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    const bool same = b.exec && b.key_args == p_dev && b.key_grid == grid && b.key_dt == dt &&
                      b.key_bits == p_host->tw_bits;
    bool ok = true;
    if (!same) {
        drop_graph(b);
        if (!b.cs && cudaStreamCreateWithFlags(&b.cs, cudaStreamNonBlocking) != cudaSuccess) ok = false;
        if (ok && cudaStreamBeginCapture(b.cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) ok = false;
        if (ok) {
            const bool m = cudaMemsetAsync(p_host->counters + 2, 0, sizeof(int) * 10, b.cs) == cudaSuccess;
            const int e = launch_batched(dt, p_dev, p_host->tw_bits, grid, b.cs);
            const bool endok = cudaStreamEndCapture(b.cs, &b.graph) == cudaSuccess;
            ok = m && e == 0 && endok && b.graph;
        }
        if (ok) ok = cudaGraphInstantiate(&b.exec, b.graph, 0) == cudaSuccess;
        if (ok) {
            b.key_args = p_dev;
            b.key_grid = grid;
            b.key_dt = dt;
            b.key_bits = p_host->tw_bits;
        }
    }
    if (ok) ok = cudaGraphLaunch(b.exec, s) == cudaSuccess;
    if (ok) return SMASH_OK;
    cudaGetLastError();
    drop_graph(b);
    if (cudaMemsetAsync(p_host->counters + 2, 0, sizeof(int) * 10, s) != cudaSuccess) return SMASH_ERR_CUDA;
    if (launch_batched(dt, p_dev, p_host->tw_bits, grid, s) != 0) {
        cudaGetLastError();
        return SMASH_ERR_CUDA;
    }
    return SMASH_OK;
}

int ensure_pinned(BatchState &b, size_t need) {
    if (b.pinned_bytes >= need) return SMASH_OK;
    if (b.pinned) cudaFreeHost(b.pinned);
    b.pinned = nullptr;
    b.pinned_bytes = 0;
    if (cudaMallocHost(&b.pinned, need) != cudaSuccess) return SMASH_ERR_ALLOC;
    b.pinned_bytes = need;
    return SMASH_OK;
}

struct Layout {
    BatchMat *mats;
    int64_t *row_start, *tile_start;
    uint8_t *cls;
    int *ub, *nnz, *big, *huge, *counters;
    unsigned long long *sums;
    int64_t *base, *totals;
};

}  // namespace

namespace smash {
namespace host {
void batched_release(smash_handle *h) {
    auto it = g_batch.find(h);
    if (it == g_batch.end()) return;
    BatchState &b = it->second;
    drop_graph(b);
    if (b.cs) cudaStreamDestroy(b.cs);
    if (b.pinned) cudaFreeHost(b.pinned);
    release(h, b.dev);
    g_batch.erase(it);
}
}  // namespace host
}  // namespace smash

extern "C" {

int smash_batched_set_table_bits(smash_handle *h, int bits) {
    if (!h || bits < 6 || bits > 12) return SMASH_ERR_INVALID_ARG;
    state_of(h).tw_bits = bits;
    return SMASH_OK;
}

int smash_batched_set_wait(smash_handle *h, int64_t wait_spins, int missing_arrivals) {
    if (!h || wait_spins < 0 || missing_arrivals < 0 || missing_arrivals > 1) return SMASH_ERR_INVALID_ARG;
    BatchState &b = state_of(h);
    b.wait_spins = wait_spins > 0 ? wait_spins : 4000000;
    b.missing = missing_arrivals;
    return SMASH_OK;
}

int smash_batched_set_row_cutoffs(smash_handle *h, int warp_less, int block_more) {
    if (!h || warp_less < 0 || warp_less > 3 || block_more < 0 || block_more > 3) return SMASH_ERR_INVALID_ARG;
    state_of(h).warp_less = warp_less;
    state_of(h).block_more = block_more;
    return SMASH_OK;
}

int smash_batched_get_row_cutoffs(smash_handle *h, int *warp_less, int *block_more) {
    if (!h || !warp_less || !block_more) return SMASH_ERR_INVALID_ARG;
    *warp_less = state_of(h).warp_less;
    *block_more = state_of(h).block_more;
    return SMASH_OK;
}

int smash_batched_get_table_bits(smash_handle *h, int *bits) {
    if (!h || !bits) return SMASH_ERR_INVALID_ARG;
    *bits = state_of(h).tw_bits;
    return SMASH_OK;
}

int spgemm_batched(smash_handle *h, int count, const smash_csr *A, const smash_csr *B, smash_dtype dtype,
                   smash_csr *C, smash_batched_stats *stats, void *stream) {
    if (!h || count < 0 || (count > 0 && (!A || !B || !C))) return SMASH_ERR_INVALID_ARG;
    if (dtype != SMASH_F32 && dtype != SMASH_F64) return SMASH_ERR_UNSUPPORTED;
    int st;
    int64_t nrows = 0, ntiles = 0;
    for (int m = 0; m < count; ++m) {
        if ((st = check_csr(&A[m], true))) return st;
        if ((st = check_csr(&B[m], true))) return st;
        if (A[m].cols != B[m].rows) return SMASH_ERR_SHAPE_MISMATCH;
        nrows += A[m].rows;
        ntiles += (A[m].rows + kBW - 1) / kBW;
    }
    if (nrows >= (1ll << 31)) return SMASH_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    BatchState &bs = state_of(h);
    const int dt = dtype == SMASH_F64 ? 1 : 0;
    const size_t vsz = dt ? 8 : 4;
    smash_batched_stats ls;
    memset(&ls, 0, sizeof(ls));
    ls.products = count;
    ls.rows = nrows;
    for (int m = 0; m < count; ++m) {
        C[m].rows = A[m].rows;
        C[m].cols = B[m].cols;
        C[m].nnz = 0;
        C[m].row_ptr = nullptr;
        C[m].col_idx = nullptr;
        C[m].val = nullptr;
    }
    if (count == 0) {
        if (stats) *stats = ls;
        return SMASH_OK;
    }
    // device workspace
    size_t need = 0;
    carve_size<BatchMat>(need, count);
    carve_size<int64_t>(need, count + 1);
    carve_size<int64_t>(need, count + 1);
    carve_size<uint8_t>(need, nrows);
    carve_size<int>(need, nrows);
    carve_size<int>(need, nrows);
    carve_size<int>(need, nrows);
    carve_size<int>(need, nrows);
    carve_size<int>(need, 12);
    carve_size<unsigned long long>(need, 4);
    carve_size<int64_t>(need, count + 1);
    carve_size<int64_t>(need, count);
    carve_size<BatchArgs>(need, 1);
    if ((st = ensure(h, bs.dev, need, s))) return st;
    Carver c(bs.dev.ptr);
    Layout L;
    L.mats = c.take<BatchMat>(count);
    L.row_start = c.take<int64_t>(count + 1);
    L.tile_start = c.take<int64_t>(count + 1);
    L.cls = c.take<uint8_t>(nrows);
    L.ub = c.take<int>(nrows);
    L.nnz = c.take<int>(nrows);
    L.big = c.take<int>(nrows);
    L.huge = c.take<int>(nrows);
    L.counters = c.take<int>(12);
    L.sums = c.take<unsigned long long>(4);
    L.base = c.take<int64_t>(count + 1);
    L.totals = c.take<int64_t>(count);
    BatchArgs *args_dev = c.take<BatchArgs>(1);
    // descriptors (pinned host -> device)
    const size_t hbytes = sizeof(BatchMat) * count + 2 * sizeof(int64_t) * (count + 1) + sizeof(BatchArgs) + 64;
    if ((st = ensure_pinned(bs, hbytes + 4096))) return st;
    cudaStreamSynchronize(s);   // the pinned staging may still feed a previous copy
    BatchMat *hm = (BatchMat *)bs.pinned;
    int64_t *hrs = (int64_t *)(hm + count);
    int64_t *hts = hrs + count + 1;
    int64_t ro = 0, to = 0;
    for (int m = 0; m < count; ++m) {
        BatchMat &d = hm[m];
        d.a_rp = A[m].row_ptr;
        d.a_ci = A[m].col_idx;
        d.a_val = A[m].val;
        d.b_rp = B[m].row_ptr;
        d.b_ci = B[m].col_idx;
        d.b_val = B[m].val;
        d.a_nnz = A[m].nnz;
        d.b_nnz = B[m].nnz;
        d.a_rows = (int32_t)A[m].rows;
        d.b_rows = (int32_t)B[m].rows;
        d.ncols = (int32_t)B[m].cols;
        d.pad = 0;
        d.row_off = ro;
        d.tile_off = to;
        hrs[m] = ro;
        hts[m] = to;
        ro += A[m].rows;
        to += (A[m].rows + kBW - 1) / kBW;
    }
    hrs[count] = ro;
    hts[count] = to;
    if (cudaMemcpyAsync(L.mats, hm, sizeof(BatchMat) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(L.row_start, hrs, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(L.tile_start, hts, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(L.counters, 0, sizeof(int) * 12, s) != cudaSuccess ||
        cudaMemsetAsync(L.sums, 0, sizeof(unsigned long long) * 4, s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    BatchArgs p;
    memset(&p, 0, sizeof(p));
    p.mats = L.mats;
    p.nmat = count;
    p.nrows = nrows;
    p.ntiles = ntiles;
    p.row_start = L.row_start;
    p.tile_start = L.tile_start;
    p.cls = L.cls;
    p.ub = L.ub;
    p.nnz = L.nnz;
    p.big = L.big;
    p.huge = L.huge;
    p.counters = L.counters;
    p.sums = L.sums;
    p.base = L.base;
    p.totals = L.totals;
    p.err = (int *)h->err.ptr;
    p.tw_bits = bs.tw_bits;
    p.warp_bits = bs.tw_bits - bs.warp_less;
    p.block_bits = bs.tw_bits + bs.block_more;
    p.wait_spins = bs.wait_spins;
    p.missing = bs.missing;
    p.dense_max = batched_dense_max(dt, bs.tw_bits);
    p.hc = HashCfg{h->params.hash_kind, 0};
    p.inv_load = 1.0f / h->params.max_load;
    {
        LaunchTimer lt(h, s, "batch_rowinfo", -1, 256, nrows, 0, 0, 0);
        launch_batch_rowinfo(p, h->sms, s);
    }
    if ((st = last_cuda_status())) return st;
    // sizes for the pools
    char *hb = (char *)h->host;
    if (cudaMemcpyAsync(hb, L.counters, sizeof(int) * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hb + 64, L.sums, sizeof(unsigned long long) * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    int nbig, nhuge;
    unsigned long long sum_ub, sum_f;
    memcpy(&nbig, hb, 4);
    memcpy(&nhuge, hb + 4, 4);
    memcpy(&sum_ub, hb + 64, 8);
    memcpy(&sum_f, hb + 72, 8);
    ls.big_rows = nbig;
    ls.huge_rows = nhuge;
    ls.flop = (int64_t)sum_f;
    // pools (owned by the caller after the call): row pointers, columns, values
    int64_t *rp_pool = (int64_t *)h->alloc(sizeof(int64_t) * (size_t)(nrows + count), h->ctx);
    int32_t *ci_pool = (int32_t *)h->alloc(sizeof(int32_t) * (size_t)(sum_ub > 0 ? sum_ub : 1), h->ctx);
    void *val_pool = h->alloc(vsz * (size_t)(sum_ub > 0 ? sum_ub : 1), h->ctx);
    if (!rp_pool || !ci_pool || !val_pool) {
        if (rp_pool) h->free_fn(rp_pool, h->ctx);
        if (ci_pool) h->free_fn(ci_pool, h->ctx);
        if (val_pool) h->free_fn(val_pool, h->ctx);
        return SMASH_ERR_ALLOC;
    }
    p.rp_pool = rp_pool;
    p.ci_pool = ci_pool;
    p.val_pool = val_pool;
    // staging of the one-pass (dense-accumulator) rows: room min(flop, cols)
    // per row at the exclusive prefix of those rooms
    p.stage_off = nullptr;
    p.stage_ci = nullptr;
    p.stage_val = nullptr;
    {
        size_t need = 0;
        carve_size<int64_t>(need, (size_t)nrows + 1);
        carve_size<long long>(need, 1);
        carve_size<char>(need, scan_scratch_bytes(nrows));
        carve_size<int32_t>(need, (size_t)(sum_ub > 0 ? sum_ub : 1));
        carve_size<char>(need, vsz * (size_t)(sum_ub > 0 ? sum_ub : 1));
        if ((st = ensure(h, h->stage, need, s))) {
            h->free_fn(rp_pool, h->ctx);
            h->free_fn(ci_pool, h->ctx);
            h->free_fn(val_pool, h->ctx);
            return st;
        }
        Carver sc(h->stage.ptr);
        int64_t *so = sc.take<int64_t>((size_t)nrows + 1);
        long long *tot = sc.take<long long>(1);
        void *scr = sc.take<char>(scan_scratch_bytes(nrows));
        p.stage_ci = sc.take<int32_t>((size_t)(sum_ub > 0 ? sum_ub : 1));
        p.stage_val = sc.take<char>(vsz * (size_t)(sum_ub > 0 ? sum_ub : 1));
        p.stage_off = so;
        launch_scan_rowptr(L.ub, nrows, so, tot, scr, s);
    }
    // on any failure from here on the pools go back to the allocator and C
    // is left empty (nothing to release for the caller)
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        h->free_fn(rp_pool, h->ctx);
        h->free_fn(ci_pool, h->ctx);
        h->free_fn(val_pool, h->ctx);
        for (int m = 0; m < count; ++m) {
            C[m].nnz = 0;
            C[m].row_ptr = nullptr;
            C[m].col_idx = nullptr;
            C[m].val = nullptr;
        }
        return code;
    };
    // rows too large for one block: exact symbolic by the regular path, per product
    std::vector<int> huge;
    std::vector<std::pair<int, std::vector<int>>> huge_by_mat;
    if (nhuge > 0) {
        huge.resize(nhuge);
        if (cudaMemcpyAsync(huge.data(), L.huge, sizeof(int) * nhuge, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(SMASH_ERR_CUDA);
        std::map<int, std::vector<int>> by;
        for (int g2 : huge) {
            int m = (int)(std::upper_bound(hrs, hrs + count + 1, (int64_t)g2) - hrs) - 1;
            while (m + 1 < count && hrs[m + 1] <= g2) ++m;
            by[m].push_back((int)(g2 - hrs[m]));
        }
        for (auto &kv : by) huge_by_mat.push_back(kv);
        for (auto &kv : huge_by_mat) {
            const int m = kv.first;
            const RawOperands op = raw_ops(&A[m], &B[m]);
            Plan pl;
            if ((st = plan_buffers(h, A[m].rows, true, s, pl))) return fail(st);
            int *list = (int *)h->host;   // staged through pinned memory
            if (ensure(h, h->learn, sizeof(int) * kv.second.size() + 256, s)) return fail(SMASH_ERR_ALLOC);
            if (cudaMemcpyAsync(h->learn.ptr, kv.second.data(), sizeof(int) * kv.second.size(),
                                cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return fail(SMASH_ERR_CUDA);
            (void)list;
            if ((st = run_symbolic(h, op, A[m].rows, pl, L.nnz + hrs[m], s, (const int *)h->learn.ptr,
                                   (int64_t)kv.second.size())))
                return fail(st);
        }
    }
    // the persistent launch
    const int grid_max = batched_grid(dt, bs.tw_bits, h->sms);
    const long long items = (long long)nbig + ntiles;
    int grid = (int)(items < grid_max ? items : grid_max);
    if (grid < 1) grid = 1;
    {
        LaunchTimer lt(h, s, "batched_persistent", -1, 256, nrows, 0, (long long)sum_f, 0);
        // the arguments through pinned memory, after the descriptors
        BatchArgs *p_pin = (BatchArgs *)(((uintptr_t)(hts + count + 1) + 63) & ~(uintptr_t)63);
        *p_pin = p;
        if ((st = run_batched_graph(bs, dt, p_pin, args_dev, grid, s))) return fail(st);
    }
    // a barrier that ran out of time (or any failed check) leaves the row
    // pointers incomplete: stop before anything reads them
    if ((st = read_flags(h, s, true))) return fail(st);
    // base offsets and totals
    std::vector<int64_t> base(count + 1), totals(count);
    if (cudaMemcpyAsync(base.data(), L.base, sizeof(int64_t) * (count + 1), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(totals.data(), L.totals, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SMASH_ERR_CUDA);
    for (int m = 0; m < count; ++m) {
        C[m].nnz = totals[m];
        C[m].row_ptr = rp_pool + hrs[m] + m;
        C[m].col_idx = ci_pool + base[m];
        C[m].val = (char *)val_pool + vsz * (size_t)base[m];
    }
    ls.c_nnz = base[count];
    // values of the huge rows by the regular path
    for (auto &kv : huge_by_mat) {
        const int m = kv.first;
        const RawOperands op = raw_ops(&A[m], &B[m]);
        Plan pl;
        if ((st = plan_buffers(h, A[m].rows, false, s, pl))) return fail(st);
        if (ensure(h, h->learn, sizeof(int) * kv.second.size() + 256, s)) return fail(SMASH_ERR_ALLOC);
        if (cudaMemcpyAsync(h->learn.ptr, kv.second.data(), sizeof(int) * kv.second.size(), cudaMemcpyHostToDevice,
                            s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(SMASH_ERR_CUDA);
        NumOut o;
        o.c_rp = C[m].row_ptr;
        o.c_ci = C[m].col_idx;
        o.c_val = C[m].val;
        o.c_nnz = C[m].nnz;
        if ((st = run_numeric(h, op, A[m].rows, dt, o, pl, s, (const int *)h->learn.ptr, (int64_t)kv.second.size())))
            return fail(st);
    }
    if ((st = read_flags(h, s, true))) return fail(st);
    if (stats) *stats = ls;
    return SMASH_OK;
}

int smash_batched_autotune(smash_handle *h, int count, const smash_csr *A, const smash_csr *B, smash_dtype dtype,
                           int *best_bits, float *best_ms, void *stream) {
    if (!h || !best_bits) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<smash_csr> C((size_t)(count > 0 ? count : 1));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1, best_wl = 0, best_bm = 3;
    float bms = 1e30f;
    BatchState &bst = state_of(h);
    const int keep = bst.tw_bits, keep_wl = bst.warp_less, keep_bm = bst.block_more;
    // the per-warp table size, and the row sizes served by one warp (32
    // threads per row) and by the whole block (256 threads per row)
    for (int cand = 0; cand < 4 * 2 * 2; ++cand) {
        const int bits = 8 + cand / 4, wl = (cand >> 1) & 1, bm = 2 + (cand & 1);
        if (batched_smem(dtype == SMASH_F64, bits) > (size_t)max_smem_per_block()) continue;
        bst.tw_bits = bits;
        bst.warp_less = wl;
        bst.block_more = bm;
        float tot = 0.f;
        int st = SMASH_OK;
        for (int rep = 0; rep < 3 && st == SMASH_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = spgemm_batched(h, count, A, B, dtype, C.data(), nullptr, stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;
            if (count > 0) smash_free_csr(h, &C[0]);
        }
        if (st != SMASH_OK) continue;
        if (tot < bms) {
            bms = tot;
            best = bits;
            best_wl = wl;
            best_bm = bm;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) {
        bst.tw_bits = keep;
        bst.warp_less = keep_wl;
        bst.block_more = keep_bm;
        return SMASH_ERR_INTERNAL;
    }
    bst.tw_bits = best;
    bst.warp_less = best_wl;
    bst.block_more = best_bm;
    *best_bits = best;
    if (best_ms) *best_ms = bms / 2.f;
    return SMASH_OK;
}

}  // extern "C"
