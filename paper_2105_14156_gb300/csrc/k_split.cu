// Planning of the dense-row cluster kernel: column windows, slices of B and
// hot columns.
//
// A dense row's accumulator (one slot per column of B) is spread over the ns
// blocks of a cluster, block q owning the contiguous window of columns
// [split[q], split[q+1]). Windows are chosen so that each receives about the
// same number of products: the weight of column j is the number of products
// that land on it over the whole product, w_j = sum over entries B[k, j] of
// the number of entries of A in column k. Split points sit at the ns-quantiles
// of the cumulative weight, moved where needed so that no window is wider than
// `cap` columns (the shared memory of one block).
//
// Slices: the entries of each row of B are regrouped by window (stable within
// a window) and woff[k][0..ns] records where each window's entries start,
// relative to the row's start, so every block enumerates only its own
// products.
//
// Hot columns: within each window, the first H columns (by index) whose
// weight reaches `thresh` get private per-warp accumulator slots in the
// kernel. Outputs per window q: hot_bm[q][cpc/32] over window-local columns,
// hot_col[q][H] (window-local column of each slot), hot_n[q].
#include "device_common.cuh"
#include "kernels.h"

namespace smash {

constexpr int kMaxSlices = 8;
constexpr int kTile = 4096;

__device__ __forceinline__ bool b_row_ok(const int64_t *b_rp, int64_t k, int64_t b_nnz, int64_t &s, int64_t &t) {
    s = b_rp[k];
    t = b_rp[k + 1];
    if (s < 0 || t < s || t > b_nnz || t - s >= kMaxBRow) {
        s = t = 0;
        return false;
    }
    return true;
}

// Window of column j given split points sp[0..ns] (bad indices go to window 0;
// the enumeration reports them).
__device__ __forceinline__ int window_of(int j, const int *sp, int ns) {
    int q = 0;
    for (int k = 1; k < ns; ++k) q += (j >= sp[k]) ? 1 : 0;
    return q;
}

// Entries of A per column of A (= per row of B).
__global__ void __launch_bounds__(256) k_colcount_a(const int32_t *a_ci, int64_t a_nnz, int b_rows, int *ca) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a_nnz; e += stride) {
        const int k = __ldg(a_ci + e);
        if ((unsigned)k < (unsigned)b_rows) atomicAdd(ca + k, 1);
    }
}

// Product weight per column of B: one warp per row k adds ca[k] to its columns.
__global__ void __launch_bounds__(256) k_colweight(const int64_t *b_rp, const int32_t *b_ci, int64_t b_rows,
                                                   int64_t b_nnz, int ncols, const int *ca,
                                                   unsigned long long *w) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < b_rows; k += warps) {
        const int c = ca[k];
        if (c == 0) continue;
        int64_t s, t;
        b_row_ok(b_rp, k, b_nnz, s, t);
        for (int64_t e = s + lane; e < t; e += 32) {
            const int j = __ldg(b_ci + e);
            if ((unsigned)j < (unsigned)ncols) atomicAdd(w + j, (unsigned long long)c);
        }
    }
}

// Per-tile sums of the weights.
__global__ void __launch_bounds__(1024) k_tile_sums(const unsigned long long *w, int ncols,
                                                    unsigned long long *part) {
    __shared__ unsigned long long s_w[32];
    const int base = blockIdx.x * kTile;
    unsigned long long v = 0;
    for (int j = base + threadIdx.x; j < base + kTile && j < ncols; j += blockDim.x) v += w[j];
    v = warp_sum(v);
    if (lane_id() == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < 32; ++k) t += s_w[k];
        part[blockIdx.x] = t;
    }
}

// One block of 1024 threads: balanced split points under the width cap.
__global__ void __launch_bounds__(1024) k_pick_splits(const unsigned long long *w, const unsigned long long *part,
                                                      int ntiles, int ncols, int ns, int cap, int *sp) {
    __shared__ int s_want[kMaxSlices + 1];
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_run;
    __shared__ int s_tile, s_found;
    if (threadIdx.x == 0) {
        s_want[0] = 0;
        s_want[ns] = ncols;
    }
    unsigned long long total = 0;
    for (int b = 0; b < ntiles; ++b) total += part[b];
    for (int q = 1; q < ns; ++q) {
        const unsigned long long target = (total * (unsigned long long)q) / (unsigned long long)ns;
        // tile holding the target (tiles are few: serial on one thread)
        if (threadIdx.x == 0) {
            unsigned long long run = 0;
            int b = 0;
            while (b < ntiles - 1 && run + part[b] <= target) run += part[b++];
            s_tile = b;
            s_run = run;
            s_found = ncols;
        }
        __syncthreads();
        // first column j of the tile whose cumulative weight exceeds the target
        const int j0 = s_tile * kTile + threadIdx.x * (kTile / 1024);
        unsigned long long loc = 0;
        for (int k = 0; k < kTile / 1024; ++k)
            if (j0 + k < ncols) loc += w[j0 + k];
        unsigned long long incl = loc;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, incl, o);
            if (lane_id() >= o) incl += t;
        }
        if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
        __syncthreads();
        unsigned long long run = s_run;
        for (int k = 0; k < (int)(threadIdx.x >> 5); ++k) run += s_w[k];
        run += incl - loc;
        for (int k = 0; k < kTile / 1024; ++k) {
            const int j = j0 + k;
            if (j < ncols) {
                run += w[j];
                if (run > target) {
                    atomicMin(&s_found, j);
                    break;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_want[q] = s_found;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // enforce widths in [1, cap]: s_q in [ncols - (ns-q)*cap, s_{q-1} + cap]
        int prev = 0;
        sp[0] = 0;
        for (int q = 1; q < ns; ++q) {
            int v = s_want[q];
            const long long lo_bound = (long long)ncols - (long long)(ns - q) * cap;
            const long long hi_bound = (long long)prev + cap;
            if (v < lo_bound) v = (int)lo_bound;
            if (v > hi_bound) v = (int)hi_bound;
            if (v < prev) v = prev;
            sp[q] = v;
            prev = v;
        }
        sp[ns] = ncols;
    }
}

__global__ void __launch_bounds__(1024) k_hot_select(const unsigned long long *w, const int *sp, int cpc, int H,
                                                     unsigned long long thresh, unsigned *hot_bm, int *hot_col,
                                                     int *hot_n) {
    __shared__ int s_w[32];
    __shared__ int s_base;
    const int q = blockIdx.x;
    const int lo = sp[q], hi = sp[q + 1];
    const int words = cpc >> 5;
    unsigned *bm = hot_bm + (size_t)q * words;
    int *cols = hot_col + (size_t)q * H;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int w0 = 0; w0 < words; w0 += blockDim.x) {
        const int wd = w0 + threadIdx.x;
        unsigned bits = 0u;
        if (wd < words)
            for (int b = 0; b < 32; ++b) {
                const int j = lo + wd * 32 + b;
                if (j < hi && w[j] >= thresh) bits |= 1u << b;
            }
        const int c = __popc(bits);
        const int incl = warp_incl_scan(c);
        if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
        __syncthreads();
        int off = s_base;
        for (int k = 0; k < (int)(threadIdx.x >> 5); ++k) off += s_w[k];
        int r = off + incl - c;
        unsigned kept = 0u;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1u;
            if (r < H) {
                kept |= 1u << b;
                cols[r] = wd * 32 + b;
            }
            ++r;
        }
        if (wd < words) bm[wd] = kept;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += s_w[k];
            s_base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) hot_n[q] = s_base < H ? s_base : H;
}

// One warp per row of B: entries per window -> woff (row-relative offsets).
__global__ void __launch_bounds__(256) k_split_count(const int64_t *b_rp, const int32_t *b_ci, int64_t b_rows,
                                                     int64_t b_nnz, const int *sp_g, int ns, int32_t *woff) {
    __shared__ int sp[kMaxSlices + 1];
    if (threadIdx.x <= ns) sp[threadIdx.x] = sp_g[threadIdx.x];
    __syncthreads();
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < b_rows; k += warps) {
        int64_t s, t;
        b_row_ok(b_rp, k, b_nnz, s, t);
        int c[kMaxSlices];
#pragma unroll
        for (int q = 0; q < kMaxSlices; ++q) c[q] = 0;
        for (int64_t e = s + lane; e < t; e += 32) {
            const int q = window_of(__ldg(b_ci + e), sp, ns);
#pragma unroll
            for (int qq = 0; qq < kMaxSlices; ++qq) c[qq] += (qq == q) ? 1 : 0;
        }
        int run = 0;
#pragma unroll
        for (int q = 0; q < kMaxSlices; ++q) {
            const int tot = warp_sum(c[q]);
            if (q < ns) {
                if (lane == 0) woff[k * (ns + 1) + q] = run;
                run += tot;
            }
        }
        if (lane == 0) woff[k * (ns + 1) + ns] = run;
    }
}

// One warp per row of B: stable regrouping of the row's entries by window.
template <typename V>
__global__ void __launch_bounds__(256) k_split_scatter(const int64_t *b_rp, const int32_t *b_ci, const V *b_val,
                                                       int64_t b_rows, int64_t b_nnz, const int *sp_g, int ns,
                                                       const int32_t *woff, int32_t *out_ci, V *out_val) {
    __shared__ int sp[kMaxSlices + 1];
    if (threadIdx.x <= ns) sp[threadIdx.x] = sp_g[threadIdx.x];
    __syncthreads();
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < b_rows; k += warps) {
        int64_t s, t;
        b_row_ok(b_rp, k, b_nnz, s, t);
        int cur[kMaxSlices];
#pragma unroll
        for (int q = 0; q < kMaxSlices; ++q) cur[q] = q < ns ? woff[k * (ns + 1) + q] : 0;
        for (int64_t e0 = s; e0 < t; e0 += 32) {
            const int64_t e = e0 + lane;
            const bool valid = e < t;
            int j = 0, q = -1;
            V v = V(0);
            if (valid) {
                j = __ldg(b_ci + e);
                v = b_val[e];
                q = window_of(j, sp, ns);
            }
            int pos = 0;
#pragma unroll
            for (int qq = 0; qq < kMaxSlices; ++qq) {
                const unsigned m = __ballot_sync(kFull, q == qq);
                if (q == qq) pos = cur[qq] + __popc(m & lanemask_lt());
                cur[qq] += __popc(m);
            }
            if (valid) {
                out_ci[s + pos] = j;
                out_val[s + pos] = v;
            }
        }
    }
}

size_t dense_plan_bytes(const RawOperands &op, int ns, int cpc, int H, size_t vsz) {
    const size_t ntiles = ((size_t)op.ncols + kTile - 1) / kTile;
    size_t b = 0;
    auto add = [&](size_t n) { b = ((b + 255) & ~size_t(255)) + n; };
    add(4 * (size_t)op.b_rows);           // ca
    add(8 * (size_t)op.ncols);            // w
    add(8 * ntiles);                      // part
    add(4 * (kMaxSlices + 1));            // splits
    add(4 * (size_t)ns * (cpc / 32));     // hot_bm
    add(4 * (size_t)ns * (H > 0 ? H : 1));  // hot_col
    add(4 * (size_t)ns);                  // hot_n
    if (ns > 1) {
        add(4 * (size_t)op.b_rows * (ns + 1));  // woff
        add(4 * (size_t)op.b_nnz);              // ci
        add(vsz * (size_t)op.b_nnz);            // val
    }
    return b + 256;
}

void launch_dense_plan(int dtype, const RawOperands &op, int ns, int cap, int cpc, int H, int hot_factor,
                       void *ws, BSlices &sl, int sms, cudaStream_t s) {
    const size_t vsz = dtype ? 8 : 4;
    const int ntiles = (int)(((int64_t)op.ncols + kTile - 1) / kTile);
    char *p = (char *)ws;
    size_t off = 0;
    auto take = [&](size_t n) -> void * {
        off = (off + 255) & ~size_t(255);
        void *r = p + off;
        off += n;
        return r;
    };
    int *ca = (int *)take(4 * (size_t)op.b_rows);
    unsigned long long *w = (unsigned long long *)take(8 * (size_t)op.ncols);
    unsigned long long *part = (unsigned long long *)take(8 * (size_t)ntiles);
    int *sp = (int *)take(4 * (kMaxSlices + 1));
    unsigned *hot_bm = (unsigned *)take(4 * (size_t)ns * (cpc / 32));
    int *hot_col = (int *)take(4 * (size_t)ns * (H > 0 ? H : 1));
    int *hot_n = (int *)take(4 * (size_t)ns);
    const int64_t cap_blocks = (int64_t)sms * 8;
    cudaMemsetAsync(ca, 0, 4 * (size_t)op.b_rows, s);
    cudaMemsetAsync(w, 0, 8 * (size_t)op.ncols, s);
    if (op.a_nnz > 0) {
        const int64_t blocks = (op.a_nnz + 255) / 256;
        k_colcount_a<<<(int)(blocks < cap_blocks ? blocks : cap_blocks), 256, 0, s>>>(op.a_ci, op.a_nnz, op.b_rows,
                                                                                       ca);
    }
    if (op.b_rows > 0) {
        const int64_t blocks = (op.b_rows + 7) / 8;
        k_colweight<<<(int)(blocks < cap_blocks ? blocks : cap_blocks), 256, 0, s>>>(op.b_rp, op.b_ci, op.b_rows,
                                                                                      op.b_nnz, op.ncols, ca, w);
    }
    if (ntiles > 0) k_tile_sums<<<ntiles, 1024, 0, s>>>(w, op.ncols, part);
    k_pick_splits<<<1, 1024, 0, s>>>(w, part, ntiles, op.ncols, ns, cap, sp);
    sl.splits = sp;
    sl.hot_h = 0;
    if (H > 0) {
        // threshold: hot_factor times the average product weight per column
        // (computed on the device would need a sync; the bound below uses the
        // exact total through nnz(A) * average row length of B)
        const double avg_b = op.b_rows > 0 ? (double)op.b_nnz / (double)op.b_rows : 0.0;
        const double avg_w = op.ncols > 0 ? (double)op.a_nnz * avg_b / (double)op.ncols : 0.0;
        double th = avg_w * hot_factor;
        if (th < 2.0) th = 2.0;
        k_hot_select<<<ns, 1024, 0, s>>>(w, sp, cpc, H, (unsigned long long)th, hot_bm, hot_col, hot_n);
        sl.hot_bm = hot_bm;
        sl.hot_col = hot_col;
        sl.hot_n = hot_n;
        sl.hot_h = H;
    }
    if (ns > 1) {
        int32_t *woff = (int32_t *)take(4 * (size_t)op.b_rows * (ns + 1));
        int32_t *sci = (int32_t *)take(4 * (size_t)op.b_nnz);
        void *sval = take(vsz * (size_t)op.b_nnz);
        if (op.b_rows > 0) {
            const int64_t blocks = (op.b_rows + 7) / 8;
            const int grid = (int)(blocks < cap_blocks ? blocks : cap_blocks);
            k_split_count<<<grid, 256, 0, s>>>(op.b_rp, op.b_ci, op.b_rows, op.b_nnz, sp, ns, woff);
            if (dtype)
                k_split_scatter<double><<<grid, 256, 0, s>>>(op.b_rp, op.b_ci, (const double *)op.b_val, op.b_rows,
                                                             op.b_nnz, sp, ns, woff, sci, (double *)sval);
            else
                k_split_scatter<float><<<grid, 256, 0, s>>>(op.b_rp, op.b_ci, (const float *)op.b_val, op.b_rows,
                                                            op.b_nnz, sp, ns, woff, sci, (float *)sval);
        }
        sl.woff = woff;
        sl.ci = sci;
        sl.val = sval;
    }
    (void)cap;
}

}  // namespace smash
