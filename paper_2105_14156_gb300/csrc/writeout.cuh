// Row write-out of the numeric phase (Write-back Phase): gather a row's
// occupied table slots, order them by column and stream them to C.
// Shared by the per-product kernels (k_numeric.cu) and the batched kernel.
#pragma once

#include <climits>

#include "device_common.cuh"

namespace smash {

// Entries of C are written once and not read again by the kernels, so they
// go out with streaming stores (__stcs: evicted from L2 first), which leaves
// L2 to the rows of B that the products gather.
//
// Output of a numeric launch. Exact mode (row_nnz == nullptr): c_rp is C's
// row pointer and every row must have exactly c_rp[i+1]-c_rp[i] entries.
// Capacity mode (learned sizing): c_rp gives each row a capacity; a row that
// fits is written at the start of its range and row_nnz[i] receives its
// length, a row that does not fit (or whose table filled up) gets -1.
template <typename V>
struct NumOutT {
    const int64_t *c_rp;
    int32_t *c_ci;
    V *c_val;
    int64_t c_nnz;
    int *row_nnz;
};

// The same checks on bounds already loaded: a row [s, t) of C, a row [ab, ae)
// of A (raise the error and return false when malformed).
__device__ __forceinline__ bool row_bounds_ok(int64_t s, int64_t t, int64_t c_nnz, int64_t &c0, int &n, int *err) {
    if (s < 0 || t < s || t > c_nnz || t - s > INT_MAX) {
        raise_err(err, kErrBadRowPtr);
        c0 = 0;
        n = 0;
        return false;
    }
    c0 = s;
    n = (int)(t - s);
    return true;
}

__device__ __forceinline__ bool a_bounds_ok(int64_t ab, int64_t ae, int64_t a_nnz, int *err) {
    if (ab < 0 || ae < ab || ae > a_nnz) {
        raise_err(err, kErrBadRowPtr);
        return false;
    }
    return true;
}

template <typename V>
__device__ __forceinline__ bool out_range(const NumOutT<V> &o, int64_t i, int64_t &c0, int &n, int *err) {
    const int64_t s = o.c_rp[i], t = o.c_rp[i + 1];
    if (s < 0 || t < s || t > o.c_nnz || t - s > INT_MAX) {
        raise_err(err, kErrBadRowPtr);
        c0 = 0;
        n = 0;
        return false;
    }
    c0 = s;
    n = (int)(t - s);
    return true;
}

// ----- write-out: warp rank (GS = 32, at most 32 entries) --------------------
template <typename V>
__device__ __forceinline__ void writeout_warp_rank(int *keys, V *vals, int T, int tot, int n_exp,
                                                   const NumOutT<V> &out, int64_t c0) {
    const int lane = lane_id();
    int filled = 0;
    for (int s0 = 0; s0 < T; s0 += 32) {
        const int k = keys[s0 + lane];
        const V v = vals[s0 + lane];
        const bool occ = k != kEmpty;
        const unsigned b = __ballot_sync(kFull, occ);
        __syncwarp();
        if (occ) {
            const int pos = filled + __popc(b & lanemask_lt());
            keys[pos] = k;
            vals[pos] = v;
        }
        filled += __popc(b);
        __syncwarp();
    }
    const int k = lane < tot ? keys[lane] : INT_MAX;
    const V v = lane < tot ? vals[lane] : V(0);
    int rank = 0;
    for (int m = 0; m < tot; ++m) rank += (__shfl_sync(kFull, k, m) < k) ? 1 : 0;
    if (lane < tot && rank < n_exp) {
        __stcs(out.c_ci + (c0 + rank), k);
        __stcs(out.c_val + (c0 + rank), v);
    }
    __syncwarp();
}

// ----- write-out: compaction + bitonic sort in shared memory ------------------
template <typename V, int GS, int NT>
__device__ __forceinline__ void writeout_bitonic(int *keys, V *vals, int T, int n_exp, const NumOutT<V> &out,
                                                 int64_t c0, int *red) {
    using G = Group<GS, NT>;
    const int t = G::tid();
    int n = 0;
    for (int s0 = 0; s0 < T; s0 += GS) {
        const int s = s0 + t;
        // (a table smaller than the group: the threads past its end hold nothing)
        const int k = s < T ? keys[s] : kEmpty;
        const V v = s < T ? vals[s] : V(0);
        const int occ = k != kEmpty ? 1 : 0;
        int ct;
        const int pos = n + G::template excl_scan<int>(occ, red, &ct);
        if (occ) {
            keys[pos] = k;
            vals[pos] = v;
        }
        n += ct;
    }
    int P = 1;
    while (P < n) P <<= 1;
    G::sync();
    for (int s = n + t; s < P; s += GS) keys[s] = INT_MAX;
    G::sync();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int idx = t; idx < (P >> 1); idx += GS) {
                const int lo = 2 * idx - (idx & (j - 1));
                const int hi = lo + j;
                const int a = keys[lo], b = keys[hi];
                const bool asc = (lo & k) == 0;
                if ((a > b) == asc) {
                    keys[lo] = b;
                    keys[hi] = a;
                    const V x = vals[lo];
                    vals[lo] = vals[hi];
                    vals[hi] = x;
                }
            }
            G::sync();
        }
    }
    const int nw = n < n_exp ? n : n_exp;
    for (int s = t; s < nw; s += GS) {
        __stcs(out.c_ci + (c0 + s), keys[s]);
        __stcs(out.c_val + (c0 + s), vals[s]);
    }
}

// ----- write-out: bucket rank ------------------------------------------------
// Counting sort by the high bits of the column, then a rank inside each
// (small) bucket: NB = T/4 buckets, bucket(j) = j >> sh (monotone in j).
// bc[NB]: per-bucket counts, made while the row was hashed (one increment per
// inserted column); gk[cap], gv[cap]: the row's (column, value) pairs
// grouped by bucket, cap = 3T/4 or T/2 (what shared memory allows). The pass
// that groups them also returns the table's occupied slots to EMPTY / 0, so
// the next row needs no clearing. A pair's position is its bucket's start plus
// the number of smaller columns in its bucket. Needs tot <= cap.
template <typename V, int GS, int NT>
__device__ __forceinline__ void writeout_bucket(int *keys, V *vals, int T, int *bc, int *gk, V *gv, int sh, int tot,
                                                int n_exp, const NumOutT<V> &out, int64_t c0, int *red,
                                                int span = -1) {
    // span: the slots that may be occupied (the whole table unless the
    // entries were staged in its first slots)
    if (span < 0) span = T;
    using G = Group<GS, NT>;
    const int t = G::tid();
    const int NB = T >> 2;
    {
        const int per = (NB + GS - 1) / GS;
        const int b0 = min(t * per, NB), b1 = min(b0 + per, NB);
        int loc = 0;
        for (int b = b0; b < b1; ++b) loc += bc[b];
        int tsum;
        int run = G::template excl_scan<int>(loc, red, &tsum);
        for (int b = b0; b < b1; ++b) {
            const int c = bc[b];
            bc[b] = run;
            run += c;
        }
    }
    G::sync();
    // four slots per thread per round, so that their atomics overlap
    for (int s0 = t; s0 < span; s0 += 4 * GS) {
        int k[4], p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) k[u] = s0 + u * GS < span ? keys[s0 + u * GS] : kEmpty;
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = k[u] != kEmpty ? atomicAdd(bc + (k[u] >> sh), 1) : 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k[u] != kEmpty) {
                const int s = s0 + u * GS;
                gk[p[u]] = k[u];
                gv[p[u]] = vals[s];
                keys[s] = kEmpty;
                vals[s] = V(0);
            }
        }
    }
    G::sync();
    // bc[b] is now the end of bucket b
    for (int q = t; q < tot; q += GS) {
        const int k = gk[q];
        const int b = k >> sh;
        const int e = bc[b];
        const int s0 = b ? bc[b - 1] : 0;
        int r = 0;
        for (int x = s0; x < e; ++x) r += gk[x] < k ? 1 : 0;
        const int pos = s0 + r;
        if (pos < n_exp) {
            __stcs(out.c_ci + (c0 + pos), k);
            __stcs(out.c_val + (c0 + pos), gv[q]);
        }
    }
}

// ----- write-out: bucket sort and merge of expanded products -----------------
// For rows whose products were staged as they came (capacity mode, the
// products fit the row's room): the same grouping by bucket as
// writeout_bucket, then each product's place in the column-sorted sequence
// (equal columns ordered by their grouped position) in keys[0..tot),
// vals[0..tot) (the table is empty by then), then one pass over the sequence
// that sums each run of equal columns into one entry of C. Returns the number
// of entries (runs); keys / vals are EMPTY / 0 again afterwards. Needs
// tot <= cap of the grouped pairs and tot <= T.
template <typename V, int GS, int NT>
__device__ __forceinline__ int writeout_bucket_merge(int *keys, V *vals, int T, int *bc, int *gk, V *gv, int sh,
                                                     int tot, const NumOutT<V> &out, int64_t c0, int *red) {
    using G = Group<GS, NT>;
    const int t = G::tid();
    const int NB = T >> 2;
    int n;   // products counted into the buckets (a product with a bad column was not staged)
    {
        const int per = (NB + GS - 1) / GS;
        const int b0 = min(t * per, NB), b1 = min(b0 + per, NB);
        int loc = 0;
        for (int b = b0; b < b1; ++b) loc += bc[b];
        int run = G::template excl_scan<int>(loc, red, &n);
        for (int b = b0; b < b1; ++b) {
            const int c = bc[b];
            bc[b] = run;
            run += c;
        }
    }
    G::sync();
    // grouped by bucket; the staged slots go back to EMPTY / 0
    for (int s = t; s < tot; s += GS) {
        const int k = keys[s];
        if (k != kEmpty) {
            const int p = atomicAdd(bc + (k >> sh), 1);
            gk[p] = k;
            gv[p] = vals[s];
            keys[s] = kEmpty;
            vals[s] = V(0);
        }
    }
    G::sync();
    // bc[b] is now the end of bucket b; place every product
    for (int q = t; q < n; q += GS) {
        const int k = gk[q];
        const int b = k >> sh;
        const int e = bc[b];
        const int s0 = b ? bc[b - 1] : 0;
        int r = 0;
        for (int x = s0; x < e; ++x) {
            const int kx = gk[x];
            r += (kx < k || (kx == k && x < q)) ? 1 : 0;
        }
        keys[s0 + r] = k;
        vals[s0 + r] = gv[q];
    }
    G::sync();
    // runs of equal columns: each thread takes a contiguous chunk of the
    // sequence, counts the run heads in it, one scan of the counts gives each
    // chunk its first place in the row, and each head sums its run (reading
    // past its chunk when the run goes on) and takes the next place
    int runs;
    {
        const int per = (n + GS - 1) / GS;
        const int q0 = min(t * per, n), q1 = min(q0 + per, n);
        int heads = 0;
        for (int q = q0; q < q1; ++q) heads += (q == 0 || keys[q - 1] != keys[q]) ? 1 : 0;
        int d = G::template excl_scan<int>(heads, red, &runs);
        for (int q = q0; q < q1; ++q) {
            const int k = keys[q];
            if (q == 0 || keys[q - 1] != k) {
                V v = vals[q];
                for (int y = q + 1; y < n && keys[y] == k; ++y) v += vals[y];
                __stcs(out.c_ci + (c0 + d), k);
                __stcs(out.c_val + (c0 + d), v);
                ++d;
            }
        }
    }
    G::sync();
    for (int q = t; q < n; q += GS) {
        keys[q] = kEmpty;
        vals[q] = V(0);
    }
    return runs;
}

// Exclusive prefix of popcounts over words [0, nwords) of bm (contiguous
// chunk per thread); returns the total.
template <int GS, int NT>
__device__ __forceinline__ int bitmap_prefix(const unsigned *bm, int *pre, int nwords, int *red) {
    using G = Group<GS, NT>;
    const int t = G::tid();
    const int wpt = (nwords + GS - 1) / GS;
    const int w0 = t * wpt;
    const int w1 = min(w0 + wpt, nwords);
    int loc = 0;
    for (int w = w0; w < w1; ++w) loc += __popc(bm[w]);
    int tot;
    int run = G::template excl_scan<int>(loc, red, &tot);
    for (int w = w0; w < w1; ++w) {
        pre[w] = run;
        run += __popc(bm[w]);
    }
    return tot;
}

// ----- write-out: bitmap rank over the columns of B ---------------------------
template <typename V, int GS, int NT>
__device__ __forceinline__ void writeout_bitmap(const int *keys, const V *vals, int T, unsigned *bm, int *pre,
                                                int words, int n_exp, const NumOutT<V> &out, int64_t c0,
                                                int *red) {
    using G = Group<GS, NT>;
    const int t = G::tid();
    for (int s = t; s < T; s += GS) {
        const int k = keys[s];
        if (k != kEmpty) atomicOr(bm + (k >> 5), 1u << (k & 31));
    }
    G::sync();
    bitmap_prefix<GS, NT>(bm, pre, words, red);
    G::sync();
    for (int s = t; s < T; s += GS) {
        const int k = keys[s];
        if (k != kEmpty) {
            const int w = k >> 5;
            const int pos = pre[w] + __popc(bm[w] & ((1u << (k & 31)) - 1u));
            if (pos < n_exp) {
                __stcs(out.c_ci + (c0 + pos), k);
                __stcs(out.c_val + (c0 + pos), vals[s]);
            }
        }
    }
}

template <typename V, int GS>
__host__ __device__ constexpr size_t num_scratch_bytes() {
    return (prod_scratch_bytes<V, GS>() + 15) & ~size_t(15);
}

// Shared memory of one group of the shared-memory hash kernel: keys[T],
// vals[T], with buckets (bcap > 0) the counters bc[T/4], then one region
// used first by the product staging (while the row's products are merged)
// and then by the write-out's grouped pairs gv[bcap], gk[bcap].
template <typename V, int GS>
__host__ __device__ constexpr size_t hash_group_bytes(int T, int bcap) {
    const size_t pairs = (size_t)bcap * (sizeof(V) + 4);
    const size_t scr = num_scratch_bytes<V, GS>();
    const size_t uni = ((pairs > scr ? pairs : scr) + 15) & ~size_t(15);
    return (size_t)T * (4 + sizeof(V)) + (bcap > 0 ? (size_t)(T >> 2) * 4 : 0) + uni;
}

}  // namespace smash
