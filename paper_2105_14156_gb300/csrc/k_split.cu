// Column windows of the dense rows: slices of B.
//
// A dense row's accumulator (one slot per column of B) is cut into windows of
// cpc consecutive columns, window w = [w*cpc, (w+1)*cpc), and each (row,
// window) pair is an independent work item of the numeric dense kernel, whose
// accumulator is the window only. So that an item enumerates only the
// products that land in its window, the entries of each row of B are
// regrouped by window (stable within a window; a no-op reordering when the
// row is sorted) and woff[k][0..nw] records where each window's entries
// start, relative to the row's start.
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

// One warp per row of B: entries per window (shared counters per warp), then
// their exclusive prefix -> woff[k][0..nw].
__global__ void __launch_bounds__(kSplitNT) k_split_count(const int64_t *b_rp, const int32_t *b_ci, int64_t b_rows,
                                                          int64_t b_nnz, int cpc, int nw, int32_t *woff) {
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
            const int q = e < t ? window_of(__ldg(b_ci + e), cpc, nw) : -1;
            const unsigned peers = __match_any_sync(kFull, q);
            if (e < t && (peers & lanemask_lt()) == 0) atomicAdd(cnt + q, __popc(peers));
        }
        __syncwarp();
        int run = 0;
        for (int q0 = 0; q0 < nw; q0 += 32) {
            const int q = q0 + lane;
            const int c = q < nw ? cnt[q] : 0;
            const int incl = warp_incl_scan(c);
            if (q < nw) woff[k * (nw + 1) + q] = run + incl - c;
            run += __shfl_sync(kFull, incl, 31);
        }
        if (lane == 0) woff[k * (nw + 1) + nw] = run;
        __syncwarp();
    }
}

// One warp per row of B: stable regrouping of the row's entries by window.
template <typename V>
__global__ void __launch_bounds__(kSplitNT) k_split_scatter(const int64_t *b_rp, const int32_t *b_ci, const V *b_val,
                                                            int64_t b_rows, int64_t b_nnz, int cpc, int nw,
                                                            const int32_t *woff, int32_t *out_ci, V *out_val) {
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
                q = window_of(j, cpc, nw);
            }
            const unsigned peers = __match_any_sync(kFull, q);
            const int base = valid ? cur[q] : 0;
            __syncwarp();
            if (valid) {
                const int pos = base + __popc(peers & lanemask_lt());
                out_ci[s + pos] = j;
                out_val[s + pos] = v;
                if ((peers & lanemask_lt()) == 0) cur[q] = base + __popc(peers);
            }
            __syncwarp();
        }
    }
}

size_t window_plan_bytes(const RawOperands &op, int nw, size_t vsz) {
    size_t b = 0;
    auto add = [&](size_t n) { b = ((b + 255) & ~size_t(255)) + n; };
    if (nw > 1) {
        add(4 * (size_t)op.b_rows * (nw + 1));  // woff
        add(4 * (size_t)op.b_nnz);              // ci
        add(vsz * (size_t)op.b_nnz);            // val
    }
    return b + 256;
}

void launch_window_plan(int dtype, const RawOperands &op, int nw, int cpc, void *ws, BSlices &sl, int sms,
                        cudaStream_t s) {
    sl.nslices = nw;
    sl.cpc = cpc;
    sl.woff = nullptr;
    sl.ci = nullptr;
    sl.val = nullptr;
    if (nw <= 1 || op.b_rows <= 0) return;
    const size_t vsz = dtype ? 8 : 4;
    char *p = (char *)ws;
    size_t off = 0;
    auto take = [&](size_t n) -> void * {
        off = (off + 255) & ~size_t(255);
        void *r = p + off;
        off += n;
        return r;
    };
    int32_t *woff = (int32_t *)take(4 * (size_t)op.b_rows * (nw + 1));
    int32_t *sci = (int32_t *)take(4 * (size_t)op.b_nnz);
    void *sval = take(vsz * (size_t)op.b_nnz);
    const int64_t cap_blocks = (int64_t)sms * 8;
    const int64_t blocks = (op.b_rows + kSplitWarps - 1) / kSplitWarps;
    const int grid = (int)(blocks < cap_blocks ? blocks : cap_blocks);
    const size_t smem = (size_t)kSplitWarps * nw * sizeof(int);
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_split_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_split_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_split_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    k_split_count<<<grid, kSplitNT, smem, s>>>(op.b_rp, op.b_ci, op.b_rows, op.b_nnz, cpc, nw, woff);
    if (dtype)
        k_split_scatter<double><<<grid, kSplitNT, smem, s>>>(op.b_rp, op.b_ci, (const double *)op.b_val, op.b_rows,
                                                              op.b_nnz, cpc, nw, woff, sci, (double *)sval);
    else
        k_split_scatter<float><<<grid, kSplitNT, smem, s>>>(op.b_rp, op.b_ci, (const float *)op.b_val, op.b_rows,
                                                             op.b_nnz, cpc, nw, woff, sci, (float *)sval);
    sl.woff = woff;
    sl.ci = sci;
    sl.val = sval;
}

}  // namespace smash
