// Column windows of the dense rows: slices of B.
//
// A dense row's accumulator (one slot per column of B) is cut into windows of
// cpc consecutive columns, window w = [w*cpc, (w+1)*cpc), and each (row,
// window) pair is an independent work item of the numeric dense kernel, whose
// accumulator is the window only. So that an item enumerates only the
// products that land in its window, woff[k][0..nw] records where each
// window's entries start in row k of B (absolute positions; B has fewer than
// 2^31 entries when windows are used). When
// every row of B is sorted by column the windows are contiguous already and
// their bounds come from binary searches (B itself is the sliced copy);
// otherwise the entries of each row are regrouped by window into a copy
// (stable within a window). For the owner-computes dense kernel each window
// is cut further into one slice per warp, slice q holding the columns of
// every per-th group of 32 columns from group q on; those slices are always
// regrouped into a copy.
#include "device_common.cuh"
#include "kernels.h"

namespace smash {

constexpr int kSplitNT = 256;
constexpr int kSplitWarps = kSplitNT / 32;

__device__ __forceinline__ bool b_row_ok(const int64_t *b_rp, int64_t k, int64_t b_nnz, int64_t &s, int64_t &t) {
    s = b_rp[k];
    t = b_rp[k + 1];
    if (s < 0 || t < s || t > b_nnz || t - s >= kMaxBRow) {
        s = t = 0;
        return false;
    }
    return true;
}

// Window of column j (bad indices go to window 0; the enumeration reports them).
__device__ __forceinline__ int window_of(int j, int cpc, int nw) {
    const int w = j >= 0 ? j / cpc : 0;
    return w < nw ? w : nw - 1;
}

// Slice of column j: its window when per == 1; else one of the window's per
// slices, each owning every per-th group of 32 columns of the window (so
// that columns crowded at one end of a window spread over all slices).
__device__ __forceinline__ int slice_of(int j, int cpc, int nw, int per) {
    const int w = window_of(j, cpc, nw);
    if (per == 1) return w;
    const int off = j >= 0 ? j - w * cpc : 0;
    return w * per + (((unsigned)off >> 5) % (unsigned)per);
}

// One warp per row of B: entries per window (shared counters per warp), then
// their exclusive prefix -> woff[k][0..nw].
__global__ void __launch_bounds__(kSplitNT) k_split_count(const int64_t *b_rp, const int32_t *b_ci, int64_t b_rows,
                                                          int64_t b_nnz, int cpc, int nwin, int per, int32_t *woff) {
    const int nw = nwin * per;   // slices
    extern __shared__ int s_cnt[];   // [kSplitWarps][nw]
    const int lane = lane_id();
    int *cnt = s_cnt + (threadIdx.x >> 5) * nw;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < b_rows; k += warps) {
        for (int q = lane; q < nw; q += 32) cnt[q] = 0;
        __syncwarp();
        int64_t s, t;
        b_row_ok(b_rp, k, b_nnz, s, t);
        for (int64_t e0 = s; e0 < t; e0 += 32) {
            const int64_t e = e0 + lane;
            const int q = e < t ? slice_of(__ldg(b_ci + e), cpc, nwin, per) : -1;
            const unsigned peers = __match_any_sync(kFull, q);
            if (e < t && (peers & lanemask_lt()) == 0) atomicAdd(cnt + q, __popc(peers));
        }
        __syncwarp();
        int run = 0;
        for (int q0 = 0; q0 < nw; q0 += 32) {
            const int q = q0 + lane;
            const int c = q < nw ? cnt[q] : 0;
            const int incl = warp_incl_scan(c);
            if (q < nw) woff[k * (nw + 1) + q] = (int32_t)(s + run + incl - c);
            run += __shfl_sync(kFull, incl, 31);
        }
        if (lane == 0) woff[k * (nw + 1) + nw] = (int32_t)(s + run);
        __syncwarp();
    }
}

// One warp per row of B: stable regrouping of the row's entries by window.
template <typename V>
__global__ void __launch_bounds__(kSplitNT) k_split_scatter(const int64_t *b_rp, const int32_t *b_ci, const V *b_val,
                                                            int64_t b_rows, int64_t b_nnz, int cpc, int nwin,
                                                            int per, const int32_t *woff, int32_t *out_ci,
                                                            V *out_val) {
    const int nw = nwin * per;   // slices
    extern __shared__ int s_cur[];   // [kSplitWarps][nw]
    const int lane = lane_id();
    int *cur = s_cur + (threadIdx.x >> 5) * nw;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < b_rows; k += warps) {
        for (int q = lane; q < nw; q += 32) cur[q] = woff[k * (nw + 1) + q];
        __syncwarp();
        int64_t s, t;
        b_row_ok(b_rp, k, b_nnz, s, t);
        for (int64_t e0 = s; e0 < t; e0 += 32) {
            const int64_t e = e0 + lane;
            const bool valid = e < t;
            int j = 0, q = -1;
            V v = V(0);
            if (valid) {
                j = __ldg(b_ci + e);
                v = b_val[e];
                q = slice_of(j, cpc, nwin, per);
            }
            const unsigned peers = __match_any_sync(kFull, q);
            const int base = valid ? cur[q] : 0;
            __syncwarp();
            if (valid) {
                const int pos = base + __popc(peers & lanemask_lt());
                out_ci[pos] = j;
                out_val[pos] = v;
                if ((peers & lanemask_lt()) == 0) cur[q] = base + __popc(peers);
            }
            __syncwarp();
        }
    }
}

// Any row of B with a column smaller than its predecessor sets *unsorted.
__global__ void __launch_bounds__(256) k_check_sorted(const int64_t *b_rp, const int32_t *b_ci, int64_t b_rows,
                                                      int64_t b_nnz, int *unsorted) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < b_rows; k += warps) {
        int64_t s, t;
        b_row_ok(b_rp, k, b_nnz, s, t);
        for (int64_t e = s + lane; e + 1 < t; e += 32) bad |= __ldg(b_ci + e) > __ldg(b_ci + e + 1);
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(unsorted, 1);
}

// Sorted rows: woff[k][w] = first entry of row k with column >= w*cpc
// (binary search); window 0 starts at the row's start and the last window
// ends at its end, so that out-of-range columns stay enumerated (and are
// reported). One thread per (row, window bound).
__global__ void __launch_bounds__(256) k_split_bsearch(const int64_t *b_rp, const int32_t *b_ci, int64_t b_rows,
                                                       int64_t b_nnz, int cpc, int nw, int32_t *woff) {
    const int64_t total = b_rows * (int64_t)(nw + 1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
        const int64_t k = x / (nw + 1);
        const int w = (int)(x - k * (nw + 1));
        int64_t s, t;
        b_row_ok(b_rp, k, b_nnz, s, t);
        int64_t pos;
        if (w == 0) pos = s;
        else if (w == nw) pos = t;
        else {
            const int key = w * cpc;
            int64_t lo = s, hi = t;   // first entry >= key
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (__ldg(b_ci + mid) < key) lo = mid + 1;
                else hi = mid;
            }
            pos = lo;
        }
        woff[x] = (int32_t)pos;
    }
}

// The counting pass keeps one counter per slice and warp in shared memory.
int window_plan_max_slices() { return (int)((size_t)max_smem_per_block() / (4 * kSplitWarps)) - 1; }

size_t window_plan_bytes(const RawOperands &op, int nw, size_t vsz) {
    size_t b = 0;
    auto add = [&](size_t n) { b = ((b + 255) & ~size_t(255)) + n; };
    if (nw > 1) {
        add(sizeof(int));                       // unsorted flag
        add(4 * (size_t)op.b_rows * (nw + 1));  // woff
        add(4 * (size_t)op.b_nnz);              // ci
        add(vsz * (size_t)op.b_nnz);            // val
    }
    return b + 256;
}

int launch_window_plan(int dtype, const RawOperands &op, int nwin, int per, int cpc, void *ws, BSlices &sl,
                       int sms, cudaStream_t s, int *host_word, int *host_word_dev) {
    const int nw = nwin * per;   // slices
    sl.nslices = nw;
    sl.cpc = cpc;
    sl.per_win = per;
    sl.woff = nullptr;
    sl.ci = nullptr;
    sl.val = nullptr;
    if (nw <= 1 || op.b_rows <= 0) return 0;
    const size_t vsz = dtype ? 8 : 4;
    char *p = (char *)ws;
    size_t off = 0;
    auto take = [&](size_t n) -> void * {
        off = (off + 255) & ~size_t(255);
        void *r = p + off;
        off += n;
        return r;
    };
    int *unsorted = (int *)take(sizeof(int));
    int32_t *woff = (int32_t *)take(4 * (size_t)op.b_rows * (nw + 1));
    int32_t *sci = (int32_t *)take(4 * (size_t)op.b_nnz);
    void *sval = take(vsz * (size_t)op.b_nnz);
    const int64_t cap_blocks = (int64_t)sms * 8;
    const int64_t blocks = (op.b_rows + kSplitWarps - 1) / kSplitWarps;
    const int grid = (int)(blocks < cap_blocks ? blocks : cap_blocks);
    // sorted rows of B need no copy when each window is one slice
    sl.woff = woff;
    int sorted = 0;
    if (per == 1) {
        cudaMemsetAsync(unsorted, 0, sizeof(int), s);
        k_check_sorted<<<grid, kSplitNT, 0, s>>>(op.b_rp, op.b_ci, op.b_rows, op.b_nnz, unsorted);
        launch_read_small(unsorted, host_word_dev, sizeof(int), s);
        cudaStreamSynchronize(s);
        sorted = *host_word == 0;
    }
    if (sorted) {
        const int64_t pairs = op.b_rows * (int64_t)(nw + 1);
        const int64_t bb = (pairs + 255) / 256;
        k_split_bsearch<<<(int)(bb < cap_blocks ? bb : cap_blocks), 256, 0, s>>>(op.b_rp, op.b_ci, op.b_rows,
                                                                                 op.b_nnz, cpc, nw, woff);
        sl.ci = op.b_ci;
        sl.val = op.b_val;
        return 2;
    }
    const size_t smem = (size_t)kSplitWarps * nw * sizeof(int);
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_split_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_split_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_split_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    k_split_count<<<grid, kSplitNT, smem, s>>>(op.b_rp, op.b_ci, op.b_rows, op.b_nnz, cpc, nwin, per, woff);
    if (dtype)
        k_split_scatter<double><<<grid, kSplitNT, smem, s>>>(op.b_rp, op.b_ci, (const double *)op.b_val, op.b_rows,
                                                              op.b_nnz, cpc, nwin, per, woff, sci, (double *)sval);
    else
        k_split_scatter<float><<<grid, kSplitNT, smem, s>>>(op.b_rp, op.b_ci, (const float *)op.b_val, op.b_rows,
                                                             op.b_nnz, cpc, nwin, per, woff, sci, (float *)sval);
    sl.ci = sci;
    sl.val = sval;
    return per == 1 ? 3 : 2;
}

}  // namespace smash
