// Row planning kernels: per-row product counts, binning, row-pointer scan.
//
// Window Distribution Phase: the number of FMAs of every row is counted from
// the row pointers alone (Gustavson's first pass: flop_i = sum_{k in A_i} |B_k|),
// and each row is assigned to a dense or a sparse (hashed) path by a threshold
// on that count. Rows are then grouped by the table size they need, so that one
// kernel launch serves rows of similar cost (the GPU counterpart of packing
// rows into windows sized to the scratchpad).
#include <climits>

#include "device_common.cuh"
#include "kernels.h"
#include "mlp.cuh"

namespace smash {

__device__ __forceinline__ int bin_for(long long size, long long f, const BinRule &r) {
    if (size <= 0) return kBinEmpty;
    if (r.dense_ok && size >= r.dense_min) return kBinDense;
    int tb = table_bits(size, r.inv_load);
    // the thread-per-row bins (k_tiny.cu) take rows of at most
    // kTinyFlopPerSlot * T products; a row with more goes to the first bin
    // above them
    if (tb <= r.tiny_tbits && f > ((long long)kTinyFlopPerSlot << tb) && r.tiny_tbits + 1 <= r.max_tbits)
        tb = r.tiny_tbits + 1;
    if (tb <= r.max_tbits) return bin_of_tbits(tb);
    return r.dense_ok ? kBinDense : kBinSpill;
}

// flop_i and nnz(A_i) of every planned row. k_rowinfo: one thread per row;
// rows longer than kLongRow entries go to a list (the long rows of R-MAT sit
// together at small row ids) that k_rowinfo_long spreads over all warps, one
// warp per row. The size that bins the row is the bound min(flop_i, cols(B))
// in the symbolic phase (c_rp == nullptr) and the exact length
// c_rp[i+1] - c_rp[i] in the numeric phase. Per-bin statistics are combined
// over each warp's rows of the same bin before they reach the block's shared
// counters, and the blocks' counters reach the global ones once per block.
constexpr int kLongRow = 64;

__device__ __forceinline__ long long b_row_len(const RawOperands &op, int k, int *err) {
    if ((unsigned)k >= (unsigned)op.b_rows) {
        raise_err(err, kErrBadIndex);
        return 0;
    }
    const int64_t s = __ldg(op.b_rp + k), t = __ldg(op.b_rp + k + 1);
    if (s >= 0 && t >= s && t <= op.b_nnz) return t - s;
    raise_err(err, kErrBadRowPtr);
    return 0;
}

struct RowStats {
    int cnt[kNumBins];
    long long max[kNumBins];
    long long sum[3][kNumBins];
    long long prod, maxrow;

    __device__ __forceinline__ void init() {
        if (threadIdx.x < kNumBins) {
            cnt[threadIdx.x] = 0;
            max[threadIdx.x] = 0;
            sum[0][threadIdx.x] = sum[1][threadIdx.x] = sum[2][threadIdx.x] = 0;
        }
        if (threadIdx.x == 0) {
            prod = 0;
            maxrow = 0;
        }
    }
    __device__ __forceinline__ void flush(BinBuffers &bb) {
        if (threadIdx.x < kNumBins && cnt[threadIdx.x]) {
            const int b = threadIdx.x;
            atomicAdd(bb.counts + b, cnt[b]);
            atomicMax(bb.maxsize + b, max[b]);
            for (int q = 0; q < 3; ++q)
                atomicAdd((unsigned long long *)(bb.sums + q * 16 + b), (unsigned long long)sum[q][b]);
        }
        if (threadIdx.x == 0) {
            atomicAdd((unsigned long long *)bb.stats, (unsigned long long)prod);
            atomicMax(bb.stats + 1, maxrow);
        }
    }
};

// Bins the warp's valid rows (one per lane) by `size` and adds them to the
// block's statistics. Called by all 32 lanes.
__device__ __forceinline__ void bin_rows(bool valid, int64_t i, int64_t len, long long f, long long size,
                                         const BinRule &rule, BinBuffers &bb, int *nnz_out, RowStats &st) {
    const int lane = lane_id();
    int b = kBinEmpty;
    if (valid) {
        b = bin_for(size, f, rule);
        bb.bin[i] = (uint8_t)b;
        if (nnz_out && b == kBinEmpty) nnz_out[i] = 0;
    }
    // warps whose values all fit 26 bits reduce with the 32-bit warp
    // reductions (sums of 32 of them fit 31 bits), the others with shuffles
    const bool small = __all_sync(kFull, !valid || (len < (1 << 26) && f < (1ll << 26) && size < (1ll << 26)));
    auto wsum = [&](long long v) -> long long {
        return small ? (long long)__reduce_add_sync(kFull, (unsigned)v) : warp_sum(v);
    };
    auto wmax = [&](long long v) -> long long {
        return small ? (long long)__reduce_max_sync(kFull, (unsigned)v) : warp_max(v);
    };
    const long long wp = wsum(valid ? f : 0ll);
    const long long wm = wmax(valid ? f : 0ll);
    if (lane == 0) {
        atomicAdd((unsigned long long *)&st.prod, (unsigned long long)wp);
        atomicMax(&st.maxrow, wm);
    }
    for (unsigned todo = __ballot_sync(kFull, valid); todo;) {
        const int b0 = __shfl_sync(kFull, b, __ffs(todo) - 1);
        const bool mine = valid && b == b0;
        const unsigned m = __ballot_sync(kFull, mine);
        todo &= ~m;
        const long long s0 = wsum(mine ? (long long)len : 0ll);
        const long long s1 = wsum(mine ? f : 0ll);
        const long long s2 = wsum(mine ? size : 0ll);
        const long long mx = wmax(mine ? size : 0ll);
        if (lane == 0) {
            atomicAdd(&st.cnt[b0], __popc(m));
            atomicMax(&st.max[b0], mx);
            atomicAdd((unsigned long long *)&st.sum[0][b0], (unsigned long long)s0);
            atomicAdd((unsigned long long *)&st.sum[1][b0], (unsigned long long)s1);
            atomicAdd((unsigned long long *)&st.sum[2][b0], (unsigned long long)s2);
        }
    }
}

// Size that bins row i: symbolic phase: the bound min(flop_i, cols(B))
// (written to bound_out); numeric phase: c_rp's row length.
__device__ __forceinline__ long long row_size(int64_t i, long long f, const RawOperands &op, const int64_t *c_rp,
                                              int64_t c_nnz, long long *bound_out, int *err) {
    if (c_rp) {
        const int64_t s = c_rp[i], t = c_rp[i + 1];
        if (s < 0 || t < s || t > c_nnz) {
            raise_err(err, kErrBadRowPtr);
            return 0;
        }
        return t - s;
    }
    const long long ub = f < (long long)op.ncols ? f : (long long)op.ncols;
    bound_out[i] = ub;
    return ub;
}

// Learned planning, second pass: one warp per 32 rows through the predictor
// (mlp_forward_warp), capacity cap_i = cap_of(y_i, margin, min(flop_i,
// cols(B))), bin of the row by cap_i.
__global__ void __launch_bounds__(256, 4) k_learned_bin(RawOperands op, BinRule rule, BinBuffers bb, LearnArgs la,
                                                     int64_t nrows) {
    __shared__ RowStats st;
    extern __shared__ __align__(16) float s_mlp[];   // the predictor's weights (mlp.cuh)
    st.init();
    // without weights every row is sized by its bound min(flop_i, cols(B))
    const bool model = la.wb != nullptr;
    if (model) load_mlp_tc(s_mlp, (const __nv_bfloat16 *)la.wb, la.norm);
    __syncthreads();
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (int64_t base = gw * 32; base < nrows; base += warps * 32) {
        const int64_t i = base + lane;
        const bool valid = i < nrows;
        RowGather rg{0, 0, 0};
        if (valid) rg = la.gather[i];
        float y = 0.f;
        if (model) {
            float x[kFeat];
            row_features(rg.na, rg.f, rg.mx, op.ncols, x);
            y = mlp_forward_warp(s_mlp, x, (uint32_t *)(s_mlp + kSmH1) + (threadIdx.x >> 5) * kH1Words);
        }
        long long size = 0;
        if (valid) {
            const long long ub = rg.f < (long long)op.ncols ? rg.f : (long long)op.ncols;
            size = model ? cap_of(y, la.margin, ub) : ub;
            la.cap[i] = (int)size;
        }
        bin_rows(valid, i, rg.na, rg.f, size, rule, bb, nullptr, st);
    }
    __syncthreads();
    st.flush(bb);
}

// Numeric planning from the counts the symbolic phase kept (one RowGather
// per row): a streaming pass, no gathers from B.
__global__ void __launch_bounds__(256) k_rowinfo_cached(RawOperands op, const int64_t *c_rp, int64_t c_nnz,
                                                        BinRule rule, BinBuffers bb, const RowGather *rec,
                                                        int *err, const int *row_list, int64_t nrows) {
    __shared__ RowStats st;
    st.init();
    __syncthreads();
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (int64_t base = gw * 32; base < nrows; base += warps * 32) {
        const int64_t r = base + lane;
        const bool valid = r < nrows;
        int64_t i = 0;
        RowGather rg{0, 0, 0};
        long long size = 0;
        if (valid) {
            i = row_list ? row_list[r] : r;
            rg = rec[i];
            size = row_size(i, rg.f, op, c_rp, c_nnz, nullptr, err);
        }
        bin_rows(valid, i, rg.na, rg.f, size, rule, bb, nullptr, st);
    }
    __syncthreads();
    st.flush(bb);
}

// Small reads for the host: device words into mapped host memory.
__global__ void __launch_bounds__(256) k_read_small(const unsigned *src, unsigned *dst, int words) {
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
}

void launch_read_small(const void *src, void *dst_mapped, size_t bytes, cudaStream_t s) {
    const int words = (int)(bytes / 4);
    if (words > 0) k_read_small<<<1, 256, 0, s>>>((const unsigned *)src, (unsigned *)dst_mapped, words);
}

// Short rows: one thread per row. Long rows: appended to long_list.
template <bool LEARN>
__global__ void __launch_bounds__(256) k_rowinfo(RawOperands op, const int64_t *c_rp, int64_t c_nnz, BinRule rule,
                                                 BinBuffers bb, long long *bound_out, int *nnz_out, int *err,
                                                 const int *row_list, int64_t nrows, int *long_list,
                                                 unsigned long long *long_count, LearnArgs la) {
    __shared__ RowStats st;
    st.init();
    __syncthreads();
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (int64_t base = gw * 32; base < nrows; base += warps * 32) {
        const int64_t r = base + lane;
        bool valid = r < nrows;
        int64_t i = 0, ab = 0, ae = 0;
        if (valid) {
            i = row_list ? row_list[r] : r;
            ab = __ldg(op.a_rp + i);
            ae = __ldg(op.a_rp + i + 1);
            if (ab < 0 || ae < ab || ae > op.a_nnz) {
                raise_err(err, kErrBadRowPtr);
                ab = ae = 0;
            }
        }
        const bool longrow = ae - ab > kLongRow;
        const unsigned lm = __ballot_sync(kFull, longrow);
        if (lm) {
            unsigned long long at = 0;
            if (lane == 0) at = atomicAdd(long_count, (unsigned long long)__popc(lm));
            at = __shfl_sync(kFull, at, 0);
            if (longrow) long_list[at + __popc(lm & lanemask_lt())] = (int)i;
        }
        valid = valid && !longrow;
        long long f = 0, mx = 0;
#pragma unroll 4
        for (int64_t e = ab; e < (longrow ? ab : ae); ++e) {
            const long long l = b_row_len(op, __ldg(op.a_ci + e), err);
            f += l;
            mx = l > mx ? l : mx;
        }
        if constexpr (LEARN) {
            // learned planning: only the row's flop count and longest row of B
            // here; k_learned_bin runs the predictor and bins the rows
            if (valid) la.gather[i] = RowGather{f, (int)(ae - ab), (int)(mx < INT_MAX ? mx : INT_MAX)};
        } else {
            long long size = 0;
            if (valid) size = row_size(i, f, op, c_rp, c_nnz, bound_out, err);
            // the symbolic phase keeps each row's counts for the numeric phase
            if (valid && la.gather) la.gather[i] = RowGather{f, (int)(ae - ab), (int)(mx < INT_MAX ? mx : INT_MAX)};
            bin_rows(valid, i, ae - ab, f, size, rule, bb, c_rp ? nullptr : nnz_out, st);
        }
    }
    __syncthreads();
    st.flush(bb);
}

// The long rows: one block per row (the longest rows of R-MAT hold tens of
// thousands of entries; a block spreads them over 256 threads).
template <bool LEARN>
__global__ void __launch_bounds__(256) k_rowinfo_long(RawOperands op, const int64_t *c_rp, int64_t c_nnz,
                                                      BinRule rule, BinBuffers bb, long long *bound_out, int *nnz_out,
                                                      int *err, const int *long_list,
                                                      const unsigned long long *long_count, LearnArgs la) {
    __shared__ RowStats st;
    __shared__ long long s_f[8], s_mx[8];
    st.init();
    __syncthreads();
    const int lane = lane_id();
    const int wp = threadIdx.x >> 5;
    const int64_t n = (int64_t)*long_count;
    for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
        const int64_t i = long_list[q];
        const int64_t ab = __ldg(op.a_rp + i), ae = __ldg(op.a_rp + i + 1);   // checked by k_rowinfo
        long long f = 0, mx = 0;
#pragma unroll 4
        for (int64_t e = ab + threadIdx.x; e < ae; e += 256) {
            const long long l = b_row_len(op, __ldg(op.a_ci + e), err);
            f += l;
            mx = l > mx ? l : mx;
        }
        f = warp_sum(f);
        mx = warp_max(mx);
        if (lane == 0) {
            s_f[wp] = f;
            s_mx[wp] = mx;
        }
        __syncthreads();
        if (wp == 0) {
            f = lane < 8 ? s_f[lane] : 0;
            mx = lane < 8 ? s_mx[lane] : 0;
            f = warp_sum(f);
            mx = warp_max(mx);
            if constexpr (LEARN) {
                if (lane == 0) la.gather[i] = RowGather{f, (int)(ae - ab), (int)(mx < INT_MAX ? mx : INT_MAX)};
            } else {
                long long size = 0;
                if (lane == 0) size = row_size(i, f, op, c_rp, c_nnz, bound_out, err);
                if (lane == 0 && la.gather)
                    la.gather[i] = RowGather{f, (int)(ae - ab), (int)(mx < INT_MAX ? mx : INT_MAX)};
                bin_rows(lane == 0, i, ae - ab, f, size, rule, bb, c_rp ? nullptr : nnz_out, st);
            }
        }
        __syncthreads();
    }
    __syncthreads();
    st.flush(bb);
}

// Scatter row ids into their bins. Each block reserves one range per bin.
constexpr int kScatNT = 256, kScatItems = 8;
__global__ void __launch_bounds__(kScatNT) k_bin_scatter(int64_t n, BinBuffers bb) {
    __shared__ int s_off[kNumBins + 1], s_cnt[kNumBins], s_base[kNumBins];
    if (threadIdx.x < kNumBins) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < kNumBins; ++b) {
            s_off[b] = acc;
            if (b != kBinEmpty) acc += bb.counts[b];
        }
        s_off[kNumBins] = acc;
        if (blockIdx.x == 0)
            for (int b = 0; b <= kNumBins; ++b) bb.offsets[b] = s_off[b];
    }
    __syncthreads();
    int loc[kScatItems];
    int bins[kScatItems];
    const int64_t base = (int64_t)blockIdx.x * kScatNT * kScatItems;
#pragma unroll
    for (int it = 0; it < kScatItems; ++it) {
        const int64_t i = base + it * kScatNT + threadIdx.x;
        bins[it] = -1;
        if (i < n) {
            const int b = bb.bin[i];
            if (b != kBinEmpty) {
                bins[it] = b;
                loc[it] = atomicAdd(&s_cnt[b], 1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < kNumBins && s_cnt[threadIdx.x])
        s_base[threadIdx.x] = atomicAdd(bb.cursor + threadIdx.x, s_cnt[threadIdx.x]);
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kScatItems; ++it) {
        if (bins[it] >= 0) {
            const int b = bins[it];
            bb.rows[s_off[b] + s_base[b] + loc[it]] = (int)(base + it * kScatNT + threadIdx.x);
        }
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 row counts into the int64 row pointer of C.
constexpr int kScanNT = 512, kScanItems = 8, kScanTile = kScanNT * kScanItems;

__device__ __forceinline__ long long block_excl_scan64(long long v, long long *s_w, long long *total) {
    const long long incl = warp_incl_scan64(v);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 31) s_w[w] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long x = threadIdx.x < (blockDim.x >> 5) ? s_w[threadIdx.x] : 0;
        long long xi = warp_incl_scan64(x);
        s_w[threadIdx.x] = xi - x;
        if (threadIdx.x == 31) s_w[32] = xi;
    }
    __syncthreads();
    const long long r = s_w[w] + incl - v;
    *total = s_w[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanNT) k_scan_reduce(const int *nnz, int64_t n, long long *part) {
    __shared__ long long s_w[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        const int64_t i = base + it * kScanNT + threadIdx.x;
        if (i < n) s += nnz[i];
    }
    long long tot;
    block_excl_scan64(s, s_w, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(long long *part, int64_t nparts, int64_t n,
                                                   int64_t *c_rp, long long *total) {
    __shared__ long long s_w[33];
    long long carry = 0;
    for (int64_t b0 = 0; b0 < nparts; b0 += blockDim.x) {
        const int64_t b = b0 + threadIdx.x;
        const long long v = b < nparts ? part[b] : 0;
        long long tot;
        const long long ex = block_excl_scan64(v, s_w, &tot);
        if (b < nparts) part[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        c_rp[n] = carry;
        *total = carry;
    }
}

__global__ void __launch_bounds__(kScanNT) k_scan_down(const int *nnz, int64_t n, const long long *part,
                                                       int64_t *c_rp) {
    __shared__ long long s_w[33];
    __shared__ int s_v[kScanTile];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        const int64_t i = base + it * kScanNT + threadIdx.x;
        s_v[it * kScanNT + threadIdx.x] = i < n ? nnz[i] : 0;
    }
    __syncthreads();
    long long loc = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) loc += s_v[threadIdx.x * kScanItems + it];
    long long tot;
    long long run = part[blockIdx.x] + block_excl_scan64(loc, s_w, &tot);
    long long outv[kScanItems];
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        outv[it] = run;
        run += s_v[threadIdx.x * kScanItems + it];
    }
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        const int64_t i = base + threadIdx.x * kScanItems + it;
        if (i < n) c_rp[i] = outv[it];
    }
}

// ---------------------------------------------------------------------------
static int rowinfo_grid(int64_t rows, int sms) {
    const int64_t blocks = (rows + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    return (int)(blocks < cap ? blocks : cap);
}

// bb.rows (filled later by the bin scatter) holds the long-row list meanwhile;
// bb.stats[2] counts it.
template <bool LEARN>
static void rowinfo(const RawOperands &op, const int64_t *c_rp, int64_t c_nnz, const BinRule &rule, BinBuffers bb,
                    long long *bound_out, int *nnz_out, int *err, int sms, cudaStream_t s, const int *row_list,
                    int64_t n, const LearnArgs &la = LearnArgs{}) {
    unsigned long long *lc = (unsigned long long *)(bb.stats + 2);
    k_rowinfo<LEARN><<<rowinfo_grid(n, sms), 256, 0, s>>>(op, c_rp, c_nnz, rule, bb, bound_out, nnz_out, err,
                                                             row_list, n, bb.rows, lc, la);
    // at most min(n, nnz(A) / (kLongRow + 1)) long rows, one per block
    int64_t most = op.a_nnz / (kLongRow + 1) + 1;
    if (most > n) most = n;
    const int64_t blocks = most;
    const int64_t cap = (int64_t)sms * 8;
    k_rowinfo_long<LEARN><<<(int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap), 256, 0, s>>>(
        op, c_rp, c_nnz, rule, bb, bound_out, nnz_out, err, bb.rows, lc, la);
}

void launch_learned_gather(const RawOperands &op, const BinRule &rule, BinBuffers bb, const LearnArgs &la,
                           int *err, int sms, cudaStream_t s) {
    if (op.a_rows == 0) return;
    rowinfo<true>(op, nullptr, 0, rule, bb, nullptr, nullptr, err, sms, s, nullptr, op.a_rows, la);
}

void launch_learned_bin(const RawOperands &op, const BinRule &rule, BinBuffers bb, const LearnArgs &la, int sms,
                        cudaStream_t s) {
    if (op.a_rows == 0) return;
    const int64_t blocks = (op.a_rows + 255) / 256;
    const int64_t cap = (int64_t)sms * 4;
    static bool attr = false;
    const size_t smem = (size_t)mlp_tc_words(256 / 32) * 4;
    if (!attr) {
        cudaFuncSetAttribute(k_learned_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    k_learned_bin<<<(int)(blocks < cap ? blocks : cap), 256, smem, s>>>(
        op, rule, bb, la, op.a_rows);
}

void launch_sym_rowinfo(const RawOperands &op, const BinRule &rule, BinBuffers bb, long long *bound_out,
                        int *nnz_out, int *err, int sms, cudaStream_t s, const int *row_list, int64_t list_n,
                        RowGather *keep) {
    const int64_t n = row_list ? list_n : op.a_rows;
    if (n == 0) return;
    LearnArgs la;
    la.gather = keep;
    rowinfo<false>(op, nullptr, 0, rule, bb, bound_out, nnz_out, err, sms, s, row_list, n, la);
}

void launch_num_rowinfo(const RawOperands &op, const int64_t *c_rp, int64_t c_nnz, const BinRule &rule,
                        BinBuffers bb, int *err, int sms, cudaStream_t s, const int *row_list, int64_t list_n,
                        const RowGather *kept) {
    const int64_t n = row_list ? list_n : op.a_rows;
    if (n == 0) return;
    if (kept) {
        k_rowinfo_cached<<<rowinfo_grid(n, sms), 256, 0, s>>>(op, c_rp, c_nnz, rule, bb, kept, err, row_list, n);
        return;
    }
    rowinfo<false>(op, c_rp, c_nnz, rule, bb, nullptr, nullptr, err, sms, s, row_list, n);
}

// Rows whose staged result did not fit (row_nnz < 0): appended to list.
__global__ void __launch_bounds__(256) k_overflow_list(const int *row_nnz, int64_t n, int *list, int *count,
                                                       uint8_t *ovf) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const bool o = row_nnz[i] < 0;
        ovf[i] = o ? 1 : 0;
        const unsigned m = __ballot_sync(__activemask(), o);
        if (o) {
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane_id() == leader) base = atomicAdd(count, __popc(m));
            base = __shfl_sync(m, base, leader);
            list[base + __popc(m & lanemask_lt())] = (int)i;
        }
    }
}

void launch_overflow_list(const int *row_nnz, int64_t n, int *list, int *count, uint8_t *ovf, cudaStream_t s) {
    if (n == 0) return;
    const int64_t blocks = (n + 255) / 256;
    k_overflow_list<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(row_nnz, n, list, count, ovf);
}

// Copy each staged row that fitted to its place in C, split by output
// position so that every warp moves the same number of entries whatever the
// row lengths. Two kernels:
//  * k_compact_walk, for outputs where long stretches belong to rows written
//    elsewhere (the column-window arena's rows, overflowing rows): a warp
//    owns kWalkChunk consecutive entries of C, finds the first row reaching
//    into them by a 32-way search on C's row pointer (each round the lanes
//    test 32 evenly spaced rows, so four rounds cover a million rows), and
//    walks the rows 32 at a time (their bounds, staging offsets and flags in
//    one coalesced round trip), copying each overlap with all lanes, four
//    loads per lane issued before their stores; a skipped row costs one step.
//  * k_compact_rows, for outputs made almost wholly of staged rows: a block
//    owns kCompactChunk consecutive entries, takes its first and last rows
//    from a table (k_chunk_rows) and lists, for each row in between, its start
//    relative to the chunk and the distance from its place in C to its staged
//    copy (a sentinel for a skipped row) in shared memory. Each warp takes an
//    eighth of the chunk, lanes on consecutive entries (the stores line up
//    with 128-byte lines); a lane finds an entry's row by a galloping search
//    from its previous entry's row, and eight float (four double) loads are
//    issued before their stores. A chunk spanning more rows than the list
//    holds (many rows of a few entries) is walked as in k_compact_walk.
constexpr int64_t kWalkChunk = 2048;
constexpr int64_t kCompactChunk = 8192;
constexpr int kCompactNT = 256;
constexpr int kCompactRows = 1024;
constexpr int kCompactBatch = 8;
constexpr int64_t kCompactSkip = INT64_MIN;

// Last row r in [0, n) with c_rp[r] <= p (c_rp[0] = 0 <= p < c_rp[n]); all
// lanes of the warp take part and return it.
__device__ __forceinline__ int64_t compact_find_row(const int64_t *__restrict__ c_rp, int64_t n, int64_t p) {
    const int lane = lane_id();
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t x = lo + lane * step;
        const bool le = x < hi && __ldg(c_rp + x) <= p;
        const int cnt = __popc(__ballot_sync(kFull, le));   // rows lo, lo+step, ... that start at or before p
        const int64_t nlo = lo + (int64_t)(cnt - 1) * step;
        const int64_t nhi = nlo + step < hi ? nlo + step : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Copies C entries [p0, p1) row by row with one warp, from row r_first (the
// row holding p0) on.
template <typename V>
__device__ void compact_walk(int64_t n, int64_t p0, int64_t p1, int64_t r_first, const int64_t *__restrict__ stage_rp,
                             const uint8_t *__restrict__ ovf, const int32_t *__restrict__ sci,
                             const V *__restrict__ sval, const int64_t *__restrict__ c_rp, int32_t *__restrict__ cci,
                             V *__restrict__ cval) {
    const int lane = lane_id();
    int64_t p = p0;
    for (int64_t r0 = r_first; p < p1 && r0 < n; r0 += 32) {
        // rows r0 .. r0+31: lane l holds row r0+l's bounds, staging offset and flag
        const int64_t rl = r0 + lane;
        int64_t rb = p1, re = p1, sb = 0;
        bool skip = true;
        if (rl < n) {
            rb = __ldg(c_rp + rl);
            re = __ldg(c_rp + rl + 1);
            sb = __ldg(stage_rp + rl);
            skip = ovf[rl] != 0;
        }
        for (int j = 0; j < 32 && p < p1; ++j) {
            const int64_t b0 = __shfl_sync(kFull, rb, j), e0 = __shfl_sync(kFull, re, j);
            const int64_t s0 = __shfl_sync(kFull, sb, j);
            const bool sk = __shfl_sync(kFull, skip ? 1 : 0, j) != 0;
            const int64_t a = p > b0 ? p : b0;
            const int64_t b = p1 < e0 ? p1 : e0;
            if (b > a && !sk) {
                const int64_t src = s0 + (a - b0);
                const int m = (int)(b - a);
                for (int k0 = 0; k0 < m; k0 += 128) {
                    int32_t ci[4];
                    V va[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = k0 + 32 * u + lane;
                        if (k < m) {
                            ci[u] = __ldg(sci + src + k);
                            va[u] = __ldg(sval + src + k);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = k0 + 32 * u + lane;
                        if (k < m) {
                            cci[a + k] = ci[u];
                            cval[a + k] = va[u];
                        }
                    }
                }
            }
            if (e0 > p) p = e0;
        }
    }
}

template <typename V>
__global__ void __launch_bounds__(256) k_compact_walk(int64_t n, int64_t c_nnz, const int64_t *__restrict__ stage_rp,
                                                      const uint8_t *__restrict__ ovf, const int32_t *__restrict__ sci,
                                                      const V *__restrict__ sval, const int64_t *__restrict__ c_rp,
                                                      int32_t *__restrict__ cci, V *__restrict__ cval) {
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (c_nnz + kWalkChunk - 1) / kWalkChunk;
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < nchunks; ch += warps) {
        const int64_t p0 = ch * kWalkChunk;
        const int64_t p1 = p0 + kWalkChunk < c_nnz ? p0 + kWalkChunk : c_nnz;
        compact_walk(n, p0, p1, compact_find_row(c_rp, n, p0), stage_rp, ovf, sci, sval, c_rp, cci, cval);
    }
}

// Row holding the first entry of each chunk of kCompactChunk entries of C (a
// thread per row marks the chunks that start inside it).
__global__ void __launch_bounds__(256) k_chunk_rows(int64_t n, const int64_t *__restrict__ c_rp, int *__restrict__ first) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const int64_t b = __ldg(c_rp + r), e = __ldg(c_rp + r + 1);
        for (int64_t k = (b + kCompactChunk - 1) / kCompactChunk; k * kCompactChunk < e; ++k) first[k] = (int)r;
    }
}

template <typename V>
__global__ void __launch_bounds__(kCompactNT, 4) k_compact_rows(int64_t n, int64_t c_nnz, const int64_t *__restrict__ stage_rp,
                                                             const uint8_t *__restrict__ ovf,
                                                             const int32_t *__restrict__ sci, const V *__restrict__ sval,
                                                             const int64_t *__restrict__ c_rp, const int *__restrict__ first,
                                                             int32_t *__restrict__ cci, V *__restrict__ cval) {
    constexpr int kB = sizeof(V) == 4 ? kCompactBatch : kCompactBatch / 2;
    __shared__ int s_start[kCompactRows];
    __shared__ int64_t s_delta[kCompactRows];
    __shared__ int64_t s_last;
    const int tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const int64_t nchunks = (c_nnz + kCompactChunk - 1) / kCompactChunk;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t p0 = ch * kCompactChunk;
        const int64_t p1 = p0 + kCompactChunk < c_nnz ? p0 + kCompactChunk : c_nnz;
        // rows holding entries p0 and p1 - 1 (rl may also be the row starting at p1)
        const int64_t rf = __ldg(first + ch);
        int64_t rl;
        if (ch + 1 < nchunks) {
            rl = __ldg(first + ch + 1);
        } else {
            if (warp == 0) {
                const int64_t r = compact_find_row(c_rp, n, p1 - 1);
                if (lane == 0) s_last = r;
            }
            __syncthreads();
            rl = s_last;
        }
        const int nr = (int)(rl - rf + 1 < (int64_t)kCompactRows + 1 ? rl - rf + 1 : (int64_t)kCompactRows + 1);
        if (nr <= kCompactRows) {
            for (int k = tid; k < nr; k += kCompactNT) {
                const int64_t r = rf + k;
                const int64_t b = __ldg(c_rp + r);
                s_start[k] = b > p0 ? (int)(b - p0) : 0;
                s_delta[k] = ovf[r] ? kCompactSkip : __ldg(stage_rp + r) - b;
            }
            __syncthreads();
            const int m = (int)(p1 - p0);
            constexpr int kPerWarp = (int)(kCompactChunk / (kCompactNT / 32));
            int k = 0;  // row of the lane's previous entry: entries rise, so rows do
            for (int q0 = warp * kPerWarp; q0 < (warp + 1) * kPerWarp && q0 < m; q0 += 32 * kB) {
                int32_t ci[kB];
                V va[kB];
                bool ok[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int q = q0 + u * 32 + lane;
                    ok[u] = false;
                    if (q < m) {
                        if (k + 1 < nr && s_start[k + 1] <= q) {
                            // gallop from k + 1, then bisect: last row with start <= q
                            int lo = k + 1, step = 1;
                            while (lo + step < nr && s_start[lo + step] <= q) {
                                lo += step;
                                step <<= 1;
                            }
                            int hi = lo + step < nr ? lo + step : nr;
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (s_start[mid] <= q) lo = mid;
                                else hi = mid;
                            }
                            k = lo;
                        }
                        const int64_t d = s_delta[k];
                        if (d != kCompactSkip) {
                            ok[u] = true;
                            ci[u] = __ldcs(sci + p0 + q + d);
                            va[u] = __ldcs(sval + p0 + q + d);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int q = q0 + u * 32 + lane;
                    if (ok[u]) {
                        __stcs(cci + p0 + q, ci[u]);
                        __stcs(cval + p0 + q, va[u]);
                    }
                }
            }
        } else {
            const int64_t per = (p1 - p0 + kCompactNT / 32 - 1) / (kCompactNT / 32);
            const int64_t a = p0 + warp * per;
            const int64_t b = a + per < p1 ? a + per : p1;
            if (a < b) compact_walk(n, a, b, compact_find_row(c_rp, n, a), stage_rp, ovf, sci, sval, c_rp, cci, cval);
        }
        __syncthreads();
    }
}

size_t compact_table_bytes(int64_t c_nnz) {
    return sizeof(int) * (size_t)((c_nnz + kCompactChunk - 1) / kCompactChunk);
}

void launch_compact_rows(int dtype, int64_t n, const int64_t *stage_rp, const uint8_t *ovf, const int32_t *stage_ci,
                         const void *stage_val, const int64_t *c_rp, int32_t *c_ci, void *c_val, int64_t c_nnz,
                         int *table, int sms, cudaStream_t s) {
    if (n == 0 || c_nnz <= 0) return;
    if (!table) {
        const int64_t blocks = ((c_nnz + kWalkChunk - 1) / kWalkChunk + 7) / 8;
        const int64_t cap = (int64_t)sms * 8;
        const int grid = (int)(blocks < cap ? blocks : cap);
        if (dtype)
            k_compact_walk<double><<<grid, 256, 0, s>>>(n, c_nnz, stage_rp, ovf, stage_ci, (const double *)stage_val,
                                                        c_rp, c_ci, (double *)c_val);
        else
            k_compact_walk<float><<<grid, 256, 0, s>>>(n, c_nnz, stage_rp, ovf, stage_ci, (const float *)stage_val,
                                                       c_rp, c_ci, (float *)c_val);
        return;
    }
    k_chunk_rows<<<rowinfo_grid(n, sms), 256, 0, s>>>(n, c_rp, table);
    const int64_t chunks = (c_nnz + kCompactChunk - 1) / kCompactChunk;
    const int64_t cap = (int64_t)sms * 4;
    const int grid = (int)(chunks < cap ? chunks : cap);
    if (dtype)
        k_compact_rows<double><<<grid, kCompactNT, 0, s>>>(n, c_nnz, stage_rp, ovf, stage_ci,
                                                           (const double *)stage_val, c_rp, table, c_ci,
                                                           (double *)c_val);
    else
        k_compact_rows<float><<<grid, kCompactNT, 0, s>>>(n, c_nnz, stage_rp, ovf, stage_ci,
                                                          (const float *)stage_val, c_rp, table, c_ci,
                                                          (float *)c_val);
}

void launch_bin_scatter(int64_t n, BinBuffers bb, cudaStream_t s) {
    if (n == 0) return;
    const int64_t per = (int64_t)kScatNT * kScatItems;
    k_bin_scatter<<<(unsigned)((n + per - 1) / per), kScatNT, 0, s>>>(n, bb);
}

size_t scan_scratch_bytes(int64_t n) {
    const int64_t parts = (n + kScanTile - 1) / kScanTile;
    return (size_t)(parts + 1) * sizeof(long long);
}

void launch_scan_rowptr(const int *nnz, int64_t n, int64_t *c_rp, long long *total, void *scratch,
                        cudaStream_t s) {
    long long *part = (long long *)scratch;
    const int64_t parts = (n + kScanTile - 1) / kScanTile;
    if (n > 0) k_scan_reduce<<<(unsigned)parts, kScanNT, 0, s>>>(nnz, n, part);
    k_scan_top<<<1, 1024, 0, s>>>(part, parts, n, c_rp, total);
    if (n > 0) k_scan_down<<<(unsigned)parts, kScanNT, 0, s>>>(nnz, n, part, c_rp);
}

}  // namespace smash
