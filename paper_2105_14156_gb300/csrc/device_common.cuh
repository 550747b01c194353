// Device-side building blocks shared by the SpGEMM kernels (sm_103a).
//
//  * warp / group scans and reductions; a "group" is GS consecutive threads of
//    a block that work on one row (GS = 32: a warp; GS = NT: the whole block;
//    otherwise a named barrier per group);
//  * the hash slot functions (Eq. hashing and the low-order-bit variant of
//    SMASH Version 2);
//  * product enumeration: every product a_ik * b_kj of one row of A, handed
//    out to the threads of a group so that consecutive lanes read consecutive
//    entries of B (coalesced), whatever the lengths of the rows of B.
//  * bounds checks on every index read from the inputs, recorded in an error
//    word instead of faulting.
#pragma once

#include <climits>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace smash {

constexpr int kEmpty = -1;             // tag of an unused slot (Algorithm SETUP's EMPTY = -1)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBRow = 1 << 21;      // longest supported row of B

// Error word indices.
enum : int {
    kErrBadIndex = 0,      // column index out of range
    kErrBadRowPtr = 1,     // row pointer not monotone / out of range
    kErrBRowTooLong = 2,   // a row of B with >= 2^21 entries
    kErrTableFull = 3,     // a hash table ran out of slots (internal)
    kErrCountMismatch = 4, // numeric row count differs from C.row_ptr
    kErrTimeout = 5,
    kNumErr = 8
};

// Bins. 0: empty rows; 1..12: shared-memory tables with 2^(bin+4) slots;
// 13: dense accumulator; 14: global-memory hash.
constexpr int kMinTBits = 5;
constexpr int kMaxTBits = 16;
constexpr int kBinEmpty = 0;
constexpr int kBinDense = 13;
constexpr int kBinSpill = 14;
constexpr int kNumBins = 15;
// The smallest bins run one thread per row (k_tiny.cu) and hold rows of at
// most kTinyFlopPerSlot * 2^tbits products: tables up to 2^kTinySymTBits
// slots in the symbolic phase, 2^kTinyNumTBits in the numeric one (the
// sizes where that beat a warp per row, measured).
constexpr int kTinySymTBits = 6;
constexpr int kTinyNumTBits = 5;
constexpr int kTinyFlopPerSlot = 2;
__host__ __device__ constexpr int bin_of_tbits(int tbits) { return 1 + tbits - kMinTBits; }
__host__ __device__ constexpr int tbits_of_bin(int bin) { return bin - 1 + kMinTBits; }

__device__ __forceinline__ void raise_err(int *err, int code) {
    if (err) atomicOr(err + code, 1);
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int warp_incl_scan(int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane_id() >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ long long warp_incl_scan64(long long v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(kFull, v, o);
        if (lane_id() >= o) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T t = __shfl_xor_sync(kFull, v, o);
        v = t > v ? t : v;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T t = __shfl_xor_sync(kFull, v, o);
        v = t < v ? t : v;
    }
    return v;
}

// ---------------------------------------------------------------------------
// Groups of GS threads inside a block of NT threads.
template <int GS, int NT>
struct Group {
    static_assert(GS % 32 == 0 && NT % GS == 0 && GS <= NT && NT <= 1024, "group shape");
    static_assert(NT / GS <= 15 || GS == 32, "named barriers: at most 15 groups");
    static constexpr int kWarps = GS / 32;
    static constexpr int kGroups = NT / GS;

    __device__ __forceinline__ static int gid() { return threadIdx.x / GS; }
    __device__ __forceinline__ static int tid() { return threadIdx.x % GS; }
    __device__ __forceinline__ static int wid() { return (threadIdx.x % GS) >> 5; }

    __device__ __forceinline__ static void sync() {
        if constexpr (GS == 32) {
            __syncwarp();
        } else if constexpr (GS == NT) {
            __syncthreads();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(gid() + 1), "n"(GS) : "memory");
        }
    }

    // Exclusive scan of v over the group; *total receives the sum.
    // scratch: kWarps ints private to the group (unused for GS = 32).
    // kFree = false leaves out the closing barrier that lets the scratch be
    // written again: for callers that pass another group barrier before
    // their next scan.
    template <typename T, bool kFree = true>
    __device__ __forceinline__ static T excl_scan(T v, T *scratch, T *total) {
        T incl;
        if constexpr (sizeof(T) == 8) incl = (T)warp_incl_scan64((long long)v);
        else incl = (T)warp_incl_scan((int)v);
        if constexpr (GS == 32) {
            *total = __shfl_sync(kFull, incl, 31);
            return incl - v;
        } else {
            if (lane_id() == 31) scratch[wid()] = incl;
            sync();
            T off = 0, tot = 0;
            const int w = wid();
#pragma unroll 4
            for (int i = 0; i < kWarps; ++i) {
                T x = scratch[i];
                if (i < w) off += x;
                tot += x;
            }
            *total = tot;
            if constexpr (kFree) sync();
            return off + incl - v;
        }
    }

    template <typename T>
    __device__ __forceinline__ static T sum(T v, T *scratch) {
        T tot;
        excl_scan<T>(v, scratch, &tot);
        return tot;
    }
};

// ---------------------------------------------------------------------------
// Rows of a bin handed out to groups by an atomic counter, one row ahead: the
// claim of a group's next row is issued when its current row starts, so the
// atomic's latency is hidden behind the row's work. A warp keeps the claim in
// lane 0's register; larger groups pass it through s_row[2][kGroups]
// alternately (the row's closing group barrier orders the write of one slot
// after the reads of it). Every iteration of the caller's row loop must end
// with a group barrier when GS > 32.
template <typename G>
struct RowClaim {
    int *token;
    int (*s_row)[G::kGroups];
    int nx = 0;    // GS = 32: the claimed next row (lane 0)
    int par = 0;   // GS > 32: slot holding the claimed next row

    __device__ __forceinline__ RowClaim(int *tok, int (*s)[G::kGroups]) : token(tok), s_row(s) {
        if (G::tid() == 0) nx = atomicAdd(token, 1);
        if constexpr (G::kWarps > 1) {
            if (G::tid() == 0) s_row[0][G::gid()] = nx;
            G::sync();
        }
    }

    // The group's row for this iteration (>= count: no more rows); claims the next.
    __device__ __forceinline__ int next(int count) {
        int r;
        if constexpr (G::kWarps == 1) {
            r = __shfl_sync(kFull, nx, 0);
            if (G::tid() == 0 && r < count) nx = atomicAdd(token, 1);
        } else {
            r = s_row[par][G::gid()];
            par ^= 1;
            if (G::tid() == 0 && r < count) s_row[par][G::gid()] = atomicAdd(token, 1);
        }
        return r;
    }
};

// RowClaim that also fetches the claimed row's entry of the row list early:
// prefetch(), called halfway through a row (when the claim's atomic has long
// returned), loads rows[next] into a register, so that the next row starts
// with its row index at hand instead of a load that waits on the atomic's
// result. Larger groups hand the claim and the row index on through shared
// memory in publish(), which the caller makes before the row's closing group
// barrier (after prefetch()). next() returns the row of the bin list and its
// row of A in *i.
template <typename G>
struct RowClaimPf {
    int *token;
    const int *rows;
    int (*s_row)[G::kGroups];
    int (*s_rowi)[G::kGroups];
    int nx = 0;     // group thread 0: the claimed next row
    int nxi = -1;   // group thread 0: its entry of the row list (-1: not fetched)
    int par = 0;

    __device__ __forceinline__ RowClaimPf(int *tok, const int *rws, int (*s)[G::kGroups], int (*si)[G::kGroups])
        : token(tok), rows(rws), s_row(s), s_rowi(si) {
        if (G::tid() == 0) nx = atomicAdd(token, 1);
        if constexpr (G::kWarps > 1) {
            if (G::tid() == 0) {
                s_row[0][G::gid()] = nx;
                s_rowi[0][G::gid()] = -1;
            }
            G::sync();
        }
    }

    __device__ __forceinline__ int next(int count, int *i) {
        int r, ri;
        if constexpr (G::kWarps == 1) {
            r = __shfl_sync(kFull, nx, 0);
            ri = __shfl_sync(kFull, nxi, 0);
        } else {
            r = s_row[par][G::gid()];
            ri = s_rowi[par][G::gid()];
            par ^= 1;
        }
        *i = ri >= 0 ? ri : (r < count ? __ldg(rows + r) : 0);
        if (G::tid() == 0 && r < count) {
            nx = atomicAdd(token, 1);
            nxi = -1;
        }
        return r;
    }

    __device__ __forceinline__ void prefetch(int count) {
        if (G::tid() == 0 && nx < count) nxi = __ldg(rows + nx);
    }

    __device__ __forceinline__ void publish() {
        if constexpr (G::kWarps > 1) {
            if (G::tid() == 0) {
                s_row[par][G::gid()] = nx;
                s_rowi[par][G::gid()] = nxi;
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Hash slot of column j in a table of 2^tbits slots.
struct HashCfg {
    int kind;     // 0 low bits, 1 multiplicative, 2 high bits
    int colbits;  // ceil(log2(cols of B)), for the order-preserving high-bit hash
};

__device__ __forceinline__ uint32_t hash_slot(int j, int tbits, HashCfg hc) {
    if (hc.kind == 0) return (uint32_t)j & ((1u << tbits) - 1u);
    if (hc.kind == 1) return ((uint32_t)j * 2654435769u) >> (32 - tbits);
    int sh = hc.colbits - tbits;
    return sh > 0 ? ((uint32_t)j >> sh) : (uint32_t)j;
}

// ---------------------------------------------------------------------------
// Inputs of one product C = A*B as the kernels see them.
template <typename V>
struct Operands {
    const int64_t *a_rp;
    const int32_t *a_ci;
    const V *a_val;
    const int64_t *b_rp;
    const int32_t *b_ci;
    const V *b_val;
    int64_t a_nnz;
    int64_t b_nnz;
    int32_t b_rows;
    int32_t ncols;
    // Optional column slicing of B: when b_woff != nullptr, each row k of B is
    // stored grouped by column window, and only window `slice` is enumerated:
    // entries [b_woff[k*(nslices+1) + slice], b_woff[k*(nslices+1) + slice+1])
    // (absolute positions in b_ci / b_val).
    const int32_t *b_woff = nullptr;
    int32_t nslices = 0;
    int32_t slice = 0;
};

// Row range of A, checked.
template <typename V>
__device__ __forceinline__ bool a_row_range(const Operands<V> &op, int64_t i, int64_t &ab,
                                            int64_t &ae, int *err) {
    ab = __ldg(op.a_rp + i);
    ae = __ldg(op.a_rp + i + 1);
    if (ab < 0 || ae < ab || ae > op.a_nnz) {
        raise_err(err, kErrBadRowPtr);
        ab = ae = 0;
        return false;
    }
    return true;
}

// The row of B selected by column k of A: start and length (checked; with a
// sliced B only this block's column window).
template <typename V>
__device__ __forceinline__ void b_row_of(const Operands<V> &op, int k, int &len, int64_t &bs, int *err) {
    len = 0;
    bs = 0;
    if (op.b_woff) {
        // sliced B: absolute bounds of row k's entries in this window
        if ((unsigned)k < (unsigned)op.b_rows) {
            const int32_t *w = op.b_woff + (size_t)k * (op.nslices + 1) + op.slice;
            bs = w[0];
            len = w[1] - w[0];
        } else {
            raise_err(err, kErrBadIndex);
        }
        return;
    }
    if ((unsigned)k < (unsigned)op.b_rows) {
        int64_t s = __ldg(op.b_rp + k), t = __ldg(op.b_rp + k + 1);
        if (s >= 0 && t >= s && t <= op.b_nnz) {
            if (t - s < kMaxBRow) {
                bs = s;
                len = (int)(t - s);
            } else {
                raise_err(err, kErrBRowTooLong);
            }
        } else {
            raise_err(err, kErrBadRowPtr);
        }
    } else {
        raise_err(err, kErrBadIndex);
    }
}

// Loads the A entry e and the range of the row of B it selects (checked).
template <typename V, bool NUM>
__device__ __forceinline__ void load_a_entry(const Operands<V> &op, int64_t e, int &len,
                                             int64_t &bs, V &av, int *err) {
    av = V(0);
    b_row_of(op, __ldg(op.a_ci + e), len, bs, err);
    if constexpr (NUM) av = op.a_val[e];
}

template <typename V>
__device__ __forceinline__ V shfl_v(V v, int src) {
    return __shfl_sync(kFull, v, src);
}

// Steps of 32 products whose loads of B are all issued before the first of
// them reaches the callback: the memory-level parallelism of one warp.
constexpr int kProdUnroll = 4;

// Every product of A entries [ab, ae) with their rows of B, enumerated by one
// warp: lane l takes products l, l+32, ... of each batch of 32 A entries.
// f(j, a, b) is called for each product: j = column, a = a_ik, b = b_kj (both
// 0 when !NUM).
template <typename V, bool NUM, typename F>
__device__ __forceinline__ void warp_products(const Operands<V> &op, int64_t ab, int64_t ae,
                                              int *err, F &&f) {
    const int lane = lane_id();
    for (int64_t base = ab; base < ae; base += 32) {
        int len = 0;
        int64_t bs = 0;
        V av = V(0);
        if (base + lane < ae) load_a_entry<V, NUM>(op, base + lane, len, bs, av, err);
        const int incl = warp_incl_scan(len);
        const int total = __shfl_sync(kFull, incl, 31);
        const int64_t start = bs - (incl - len);   // product p of this entry reads b[start + p]
        for (int p0 = 0; p0 < total; p0 += 32 * kProdUnroll) {
            int jv[kProdUnroll];
            V av_u[kProdUnroll], bv[kProdUnroll];
            bool act[kProdUnroll];
#pragma unroll
            for (int u = 0; u < kProdUnroll; ++u) {
                const int p = p0 + 32 * u + lane;
                act[u] = p < total;
                int o = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    int c = __shfl_sync(kFull, incl, o + s - 1);
                    if (c <= p) o += s;
                }
                const int64_t st = __shfl_sync(kFull, start, o);
                av_u[u] = V(0);
                bv[u] = V(0);
                if constexpr (NUM) av_u[u] = shfl_v(av, o);
                jv[u] = 0;
                if (act[u]) {
                    jv[u] = __ldg(op.b_ci + st + p);
                    if constexpr (NUM) bv[u] = __ldg(op.b_val + st + p);
                }
            }
#pragma unroll
            for (int u = 0; u < kProdUnroll; ++u) {
                if (act[u]) {
                    if ((unsigned)jv[u] < (unsigned)op.ncols) f(jv[u], av_u[u], bv[u]);
                    else raise_err(err, kErrBadIndex);
                }
            }
        }
    }
}

// Shared scratch of a group for group_products (GS entries each).
template <typename V>
struct ProdScratch {
    int *incl;       // [GS]
    int64_t *start;  // [GS]
    V *av;           // [GS]
    int *red;        // [GS/32] scan scratch
    int64_t *red64;  // [GS/32]
};

template <typename V, int GS>
__host__ __device__ constexpr size_t prod_scratch_bytes() {
    return (size_t)GS * (4 + 8 + sizeof(V)) + (GS / 32) * (4 + 8) + 16;
}

// The scratch starts at the first 16-byte boundary at or after p; the size
// from prod_scratch_bytes() includes the 16 bytes this may skip.
template <typename V, int GS>
__device__ __forceinline__ ProdScratch<V> carve_prod_scratch(unsigned char *p) {
    p = (unsigned char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    ProdScratch<V> s;
    s.start = (int64_t *)p;
    p += GS * 8;
    s.red64 = (int64_t *)p;
    p += (GS / 32) * 8;
    s.av = (V *)p;
    p += GS * sizeof(V);
    s.incl = (int *)p;
    p += GS * 4;
    s.red = (int *)p;
    return s;
}

// Entry of product q + lane in one step of 32 products of a run of staged
// entries, every one with at least one product, whose inclusive product ends
// relative to q are e (lane l: entry c0 + l; lane 0's entry holds product q,
// so its e >= 1): the number of entries that end at or before q + lane.
__device__ __forceinline__ int step_entry(int e) {
    const unsigned ends = __reduce_or_sync(kFull, (e >= 1 && e <= 31) ? (1u << e) : 0u);
    return __popc(ends & ((2u << lane_id()) - 1u));
}

// Every product of A entries [ab, ae), enumerated by a group of GS threads
// (a warp or more): batches of GS A entries are staged in shared memory (entries with
// an empty row of B dropped), the batch's products are split into one
// contiguous range per warp, and each warp walks its range 32 products at a
// time, kProdUnroll steps per round. The window of 32 staged entries that
// starts at the entry of the step's first product holds every product of the
// step; a lane finds its entry from the set of entry ends inside the step.
// Only the first step of a range needs a binary search over the whole batch.
// The columns of A of the next batch are fetched before the current batch's
// products are walked.
template <typename V, bool NUM, int GS, int NT, typename F>
__device__ __forceinline__ void group_products(const Operands<V> &op, int64_t ab, int64_t ae,
                                               const ProdScratch<V> &sc, int *err, F &&f) {
    using G = Group<GS, NT>;
    const int t = G::tid();
    const int lane = lane_id();
    const int w = G::wid();
    int k_next = -1;
    V av_next = V(0);
    if (ab + t < ae) {
        k_next = __ldg(op.a_ci + ab + t);
        if constexpr (NUM) av_next = op.a_val[ab + t];
    }
    int pbase = 0;   // products of the earlier batches
    for (int64_t base = ab; base < ae; base += GS) {
        int len = 0;
        int64_t bs = 0;
        const V av = av_next;
        if (base + t < ae) b_row_of(op, k_next, len, bs, err);
        // one scan of (entry has products, product count): count in the high half
        const long long packed = ((long long)(len > 0 ? 1 : 0) << 32) | (long long)len;
        long long tot64;
        // the scan's scratch is written again only in the next batch's scan,
        // after the staging barrier below
        const long long ex = G::template excl_scan<long long, false>(packed, (long long *)sc.red64, &tot64);
        const int cidx = (int)(ex >> 32);
        const int excl = (int)(ex & 0xffffffffll);
        const int nf = (int)(tot64 >> 32);
        const int total = (int)(tot64 & 0xffffffffll);
        if (len > 0) {
            sc.incl[cidx] = excl + len;
            sc.start[cidx] = bs - excl;
            if constexpr (NUM) sc.av[cidx] = av;
        }
        if (base + GS + t < ae) {
            k_next = __ldg(op.a_ci + base + GS + t);
            if constexpr (NUM) av_next = op.a_val[base + GS + t];
        }
        G::sync();
        const int per = (total + G::kWarps - 1) / G::kWarps;
        const int lo = w * per;
        const int hi = min(lo + per, total);
        if (lo < hi) {
            int a = 0, b = nf;
            while (a < b) {
                const int m = (a + b) >> 1;
                if (sc.incl[m] <= lo) a = m + 1;
                else b = m;
            }
            int c0 = a;
            for (int pb = lo; pb < hi; pb += 32 * kProdUnroll) {
                int jv[kProdUnroll];
                V av_u[kProdUnroll], bv[kProdUnroll];
                bool act[kProdUnroll];
#pragma unroll
                for (int u = 0; u < kProdUnroll; ++u) {
                    const int q = pb + 32 * u;
                    act[u] = false;
                    jv[u] = 0;
                    av_u[u] = V(0);
                    bv[u] = V(0);
                    if (q < hi) {
                        act[u] = q + lane < hi;
                        const int e0 = sc.incl[c0] - q;   // same for all lanes
                        if (e0 >= 32) {
                            // the whole step lies in entry c0 (long rows of B)
                            if (act[u]) {
                                const int64_t idx = sc.start[c0] + q + lane;
                                jv[u] = __ldg(op.b_ci + idx);
                                if constexpr (NUM) {
                                    bv[u] = __ldg(op.b_val + idx);
                                    av_u[u] = sc.av[c0];
                                }
                            }
                            if (e0 == 32) ++c0;
                        } else {
                            const int c = c0 + lane;
                            const int e = c < nf ? sc.incl[c] - q : INT_MAX;
                            const int ci = c0 + step_entry(e);
                            if (act[u]) {
                                const int64_t idx = sc.start[ci] + q + lane;
                                jv[u] = __ldg(op.b_ci + idx);
                                if constexpr (NUM) {
                                    bv[u] = __ldg(op.b_val + idx);
                                    av_u[u] = sc.av[ci];
                                }
                            }
                            c0 += __popc(__ballot_sync(kFull, e <= 32));
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kProdUnroll; ++u) {
                    if (act[u]) {
                        if ((unsigned)jv[u] < (unsigned)op.ncols) {
                            // (a callback of four arguments also gets the product's
                            // index among the row's products)
                            if constexpr (std::is_invocable_v<F, int, V, V, int>)
                                f(jv[u], av_u[u], bv[u], pbase + pb + 32 * u + lane);
                            else
                                f(jv[u], av_u[u], bv[u]);
                        } else {
                            raise_err(err, kErrBadIndex);
                        }
                    }
                }
            }
        }
        pbase += total;
        // no barrier here: the next batch stages its entries only after the
        // first barrier of its scan, which every warp reaches after its walk
    }
    G::sync();
}

// ---------------------------------------------------------------------------
// Hash table operations. keys: int tags (kEmpty = free); probing is linear,
// +1 slot per collision with wrap-around (Hashing Phase, collision
// resolution). Returns the slot, or -1 if the table is full.
template <bool GLOBAL>
__device__ __forceinline__ int ld_key(const int *k) {
    if constexpr (GLOBAL) {
        int v;
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(k) : "memory");
        return v;
    } else {
        return *(volatile const int *)k;
    }
}

template <bool GLOBAL>
__device__ __forceinline__ int hash_find_or_insert(int *keys, int tbits, HashCfg hc, int j,
                                                   bool &inserted) {
    const uint32_t mask = (1u << tbits) - 1u;
    uint32_t h = hash_slot(j, tbits, hc) & mask;
    inserted = false;
    for (uint32_t n = 0; n <= mask; ++n) {
        int k = ld_key<GLOBAL>(keys + h);
        if (k == j) return (int)h;
        if (k == kEmpty) {
            int old = atomicCAS(keys + h, kEmpty, j);
            if (old == kEmpty) {
                inserted = true;
                return (int)h;
            }
            if (old == j) return (int)h;
        }
        h = (h + 1u) & mask;
    }
    return -1;
}

// Ceil-power-of-two table size for `bound` entries at load `inv_load`.
__host__ __device__ inline int table_bits(int64_t bound, float inv_load) {
    double want = (double)bound * (double)inv_load;
    int b = kMinTBits;
    while (b < 40 && (double)(1ll << b) < want) ++b;
    return b;
}

}  // namespace smash
