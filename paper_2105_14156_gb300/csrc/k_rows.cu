// Row planning kernels: per-row product counts, binning, row-pointer scan.
//
// Window Distribution Phase: the number of FMAs of every row is counted from
// the row pointers alone (Gustavson's first pass: flop_i = sum_{k in A_i} |B_k|),
// and each row is assigned to a dense or a sparse (hashed) path by a threshold
// on that count. Rows are then grouped by the table size they need, so that one
// kernel launch serves rows of similar cost (the GPU counterpart of packing
// rows into windows sized to the scratchpad).
#include "device_common.cuh"
#include "kernels.h"

namespace smash {

__device__ __forceinline__ int bin_for(long long size, const BinRule &r) {
    if (size <= 0) return kBinEmpty;
    if (r.dense_ok && size >= r.dense_min) return kBinDense;
    const int tb = table_bits(size, r.inv_load);
    if (tb <= r.max_tbits) return bin_of_tbits(tb);
    return r.dense_ok ? kBinDense : kBinSpill;
}

// One warp per row of A: flop_i and nnz(A_i). The size that bins the row is
// the bound min(flop_i, cols(B)) in the symbolic phase (c_rp == nullptr) and
// the exact length c_rp[i+1] - c_rp[i] in the numeric phase.
__global__ void __launch_bounds__(256) k_rowinfo(RawOperands op, const int64_t *c_rp, int64_t c_nnz, BinRule rule,
                                                 BinBuffers bb, long long *bound_out, int *nnz_out, int *err,
                                                 const int *row_list, int64_t nrows) {
    __shared__ int s_cnt[kNumBins];
    __shared__ long long s_max[kNumBins];
    __shared__ long long s_sum[3][kNumBins];
    __shared__ long long s_prod, s_maxrow;
    if (threadIdx.x < kNumBins) {
        s_cnt[threadIdx.x] = 0;
        s_max[threadIdx.x] = 0;
        s_sum[0][threadIdx.x] = s_sum[1][threadIdx.x] = s_sum[2][threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
        s_prod = 0;
        s_maxrow = 0;
    }
    __syncthreads();
    const int lane = lane_id();
    long long my_prod = 0, my_max = 0;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += warps) {
        const int64_t i = row_list ? row_list[r] : r;
        int64_t ab = __ldg(op.a_rp + i), ae = __ldg(op.a_rp + i + 1);
        if (ab < 0 || ae < ab || ae > op.a_nnz) {
            if (lane == 0) raise_err(err, kErrBadRowPtr);
            ab = ae = 0;
        }
        long long f = 0;
        for (int64_t e = ab + lane; e < ae; e += 32) {
            const int k = __ldg(op.a_ci + e);
            if ((unsigned)k < (unsigned)op.b_rows) {
                const int64_t s = __ldg(op.b_rp + k), t = __ldg(op.b_rp + k + 1);
                if (s >= 0 && t >= s && t <= op.b_nnz) f += t - s;
                else raise_err(err, kErrBadRowPtr);
            } else {
                raise_err(err, kErrBadIndex);
            }
        }
        f = warp_sum(f);
        if (lane == 0) {
            long long size;
            if (c_rp) {
                const int64_t s = c_rp[i], t = c_rp[i + 1];
                size = 0;
                if (s < 0 || t < s || t > c_nnz) raise_err(err, kErrBadRowPtr);
                else size = t - s;
            } else {
                size = f < (long long)op.ncols ? f : (long long)op.ncols;
                bound_out[i] = size;
            }
            const int b = bin_for(size, rule);
            bb.bin[i] = (uint8_t)b;
            atomicAdd(&s_cnt[b], 1);
            atomicMax(&s_max[b], size);
            atomicAdd((unsigned long long *)&s_sum[0][b], (unsigned long long)(ae - ab));
            atomicAdd((unsigned long long *)&s_sum[1][b], (unsigned long long)f);
            atomicAdd((unsigned long long *)&s_sum[2][b], (unsigned long long)size);
            if (!c_rp && b == kBinEmpty) nnz_out[i] = 0;
            my_prod += f;
            my_max = f > my_max ? f : my_max;
        }
    }
    if (lane == 0) {
        atomicAdd((unsigned long long *)&s_prod, (unsigned long long)my_prod);
        atomicMax(&s_maxrow, my_max);
    }
    __syncthreads();
    if (threadIdx.x < kNumBins && s_cnt[threadIdx.x]) {
        const int b = threadIdx.x;
        atomicAdd(bb.counts + b, s_cnt[b]);
        atomicMax(bb.maxsize + b, s_max[b]);
        for (int q = 0; q < 3; ++q)
            atomicAdd((unsigned long long *)(bb.sums + q * 16 + b), (unsigned long long)s_sum[q][b]);
    }
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long *)bb.stats, (unsigned long long)s_prod);
        atomicMax(bb.stats + 1, s_maxrow);
    }
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
    const int64_t blocks = (rows + 7) / 8;
    const int64_t cap = (int64_t)sms * 8;
    return (int)(blocks < cap ? blocks : cap);
}

void launch_sym_rowinfo(const RawOperands &op, const BinRule &rule, BinBuffers bb, long long *bound_out,
                        int *nnz_out, int *err, int sms, cudaStream_t s, const int *row_list, int64_t list_n) {
    const int64_t n = row_list ? list_n : op.a_rows;
    if (n == 0) return;
    k_rowinfo<<<rowinfo_grid(n, sms), 256, 0, s>>>(op, nullptr, 0, rule, bb, bound_out, nnz_out, err, row_list, n);
}

void launch_num_rowinfo(const RawOperands &op, const int64_t *c_rp, int64_t c_nnz, const BinRule &rule,
                        BinBuffers bb, int *err, int sms, cudaStream_t s, const int *row_list, int64_t list_n) {
    const int64_t n = row_list ? list_n : op.a_rows;
    if (n == 0) return;
    k_rowinfo<<<rowinfo_grid(n, sms), 256, 0, s>>>(op, c_rp, c_nnz, rule, bb, nullptr, nullptr, err, row_list, n);
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

// Copy each staged row that fitted to its place in C. Work is split by output
// position: a warp owns a chunk of kCompactChunk consecutive entries of C,
// finds the first row reaching into it by binary search on C's row pointer
// and walks the rows of the chunk, copying each overlap with all lanes
// (coalesced reads and writes, equal work per warp whatever the row lengths).
constexpr int64_t kCompactChunk = 2048;

template <typename V>
__global__ void __launch_bounds__(256) k_compact_rows(int64_t n, int64_t c_nnz, const int64_t *__restrict__ stage_rp,
                                                      const uint8_t *__restrict__ ovf, const int32_t *__restrict__ sci,
                                                      const V *__restrict__ sval, const int64_t *__restrict__ c_rp,
                                                      int32_t *__restrict__ cci, V *__restrict__ cval) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (c_nnz + kCompactChunk - 1) / kCompactChunk;
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < nchunks; ch += warps) {
        const int64_t p0 = ch * kCompactChunk;
        const int64_t p1 = p0 + kCompactChunk < c_nnz ? p0 + kCompactChunk : c_nnz;
        int64_t lo = 0, hi = n;   // last row r with c_rp[r] <= p0 (c_rp[n] = c_nnz > p0)
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(c_rp + mid) <= p0) lo = mid;
            else hi = mid;
        }
        int64_t p = p0;
        for (int64_t r = lo; p < p1 && r < n; ++r) {
            const int64_t rb = __ldg(c_rp + r), re = __ldg(c_rp + r + 1);
            const int64_t a = p > rb ? p : rb;
            const int64_t b = p1 < re ? p1 : re;
            if (b > a && !ovf[r]) {
                const int64_t src = __ldg(stage_rp + r) + (a - rb);
                const int64_t m = b - a;
#pragma unroll 4
                for (int64_t k = lane; k < m; k += 32) {
                    cci[a + k] = __ldg(sci + src + k);
                    cval[a + k] = __ldg(sval + src + k);
                }
            }
            if (re > p) p = re;
        }
    }
}

void launch_compact_rows(int dtype, int64_t n, const int64_t *stage_rp, const int *row_nnz_final,
                         const uint8_t *ovf, const int32_t *stage_ci, const void *stage_val, const int64_t *c_rp,
                         int32_t *c_ci, void *c_val, int64_t c_nnz, int sms, cudaStream_t s) {
    (void)row_nnz_final;
    if (n == 0 || c_nnz <= 0) return;
    const int64_t chunks = (c_nnz + kCompactChunk - 1) / kCompactChunk;
    const int64_t blocks = (chunks + 7) / 8;
    const int64_t cap = (int64_t)sms * 8;
    const int grid = (int)(blocks < cap ? blocks : cap);
    if (dtype)
        k_compact_rows<double><<<grid, 256, 0, s>>>(n, c_nnz, stage_rp, ovf, stage_ci, (const double *)stage_val,
                                                    c_rp, c_ci, (double *)c_val);
    else
        k_compact_rows<float><<<grid, 256, 0, s>>>(n, c_nnz, stage_rp, ovf, stage_ci, (const float *)stage_val,
                                                   c_rp, c_ci, (float *)c_val);
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
