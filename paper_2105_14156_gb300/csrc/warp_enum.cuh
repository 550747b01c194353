// Register-staged product enumeration of one warp and compare-and-swap-first
// insertion, shared by the warp-row kernels (k_warp.cuh) and the batched
// kernel (k_batched.cu).
//
// Lane l of each batch of 32 entries of A_i holds entry l (where the row of B
// it selects starts, its length and a_ik), entries whose row of B is empty
// moved out of the way; a scan of the lengths lays the batch's products on
// one line, and each step hands 32 consecutive products to the 32 lanes. The
// entry of product q + l is the number of entries that end at or before it:
// those ending before the step (one ballot) plus those ending inside it (one
// OR-reduction of one bit per end, then a popcount below the lane). Loads of
// B are coalesced: consecutive lanes read consecutive entries of a row of B.
#pragma once

#include <climits>

#include "device_common.cuh"

namespace smash {

constexpr int kWarpUnroll = 4;     // steps of 32 products whose loads are issued together

// Per-warp scratch of the register enumerator: one batch of entries.
template <typename V>
struct EntryScratch {
    int64_t start[32];
    V av[32];
    int len[32];
};

// The row of B selected by column k of A (start and length, checked), for
// kernels that never see B sliced by column window.
template <typename V>
__device__ __forceinline__ void b_row_whole(const Operands<V> &op, int k, int &len, int64_t &bs, int *err) {
    len = 0;
    bs = 0;
    if ((unsigned)k < (unsigned)op.b_rows) {
        const int64_t s = __ldg(op.b_rp + k), t = __ldg(op.b_rp + k + 1);
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

// Insertion of tag j into a shared-memory table of 2^tbits slots: the slot
// (-1: the table is full), and whether this call claimed it.
__device__ __forceinline__ int cas_insert(int *keys, int tbits, HashCfg hc, int j, bool &ins) {
    const uint32_t mask = (1u << tbits) - 1u;
    uint32_t h = hash_slot(j, tbits, hc) & mask;
    ins = false;
    for (uint32_t n = 0; n <= mask; ++n) {
        const int old = atomicCAS(keys + h, kEmpty, j);
        if (old == kEmpty) {
            ins = true;
            return (int)h;
        }
        if (old == j) return (int)h;
        h = (h + 1u) & mask;
    }
    return -1;
}

// Every product a_ik * b_kj of A entries [ab, ae), enumerated by one warp.
// f(act, j, a, b, p) is called by all 32 lanes together once per step of 32
// products (act: the lane holds a product; p: its index among the row's
// products), so that it may use warp votes.
// IT: type of the positions in B (int32_t when B has fewer than 2^31 entries).
template <typename V, typename IT, bool NUM, typename F>
__device__ __forceinline__ void warp_enum(const Operands<V> &op, int64_t ab, int64_t ae, EntryScratch<V> &es,
                                          int *err, F &&f) {
    const int lane = lane_id();
    int pbase = 0;   // products of the earlier batches
    for (int64_t base = ab; base < ae; base += 32) {
        int len = 0;
        int64_t bs = 0;
        V av = V(0);
        if (base + lane < ae) {
            b_row_whole(op, __ldg(op.a_ci + base + lane), len, bs, err);
            if constexpr (NUM) av = op.a_val[base + lane];
        }
        // entries with an empty row of B would share their end with the entry
        // before them: move the others to the low lanes, in order
        const unsigned nz = __ballot_sync(kFull, len > 0);
        const int nv = __popc(nz);
        if (nv < 32 && nz != (1u << nv) - 1u) {
            if (len > 0) {
                const int d = __popc(nz & lanemask_lt());
                es.start[d] = bs;
                es.len[d] = len;
                if constexpr (NUM) es.av[d] = av;
            }
            __syncwarp();
            len = lane < nv ? es.len[lane] : 0;
            bs = lane < nv ? es.start[lane] : 0;
            if constexpr (NUM) av = lane < nv ? es.av[lane] : V(0);
            __syncwarp();
        }
        const int incl = warp_incl_scan(len);
        const int total = __shfl_sync(kFull, incl, 31);
        const IT start = (IT)(bs - (incl - len));   // product p of this entry reads B at start + p
        for (int q0 = 0; q0 < total; q0 += 32 * kWarpUnroll) {
            int jv[kWarpUnroll];
            V a_u[kWarpUnroll], b_u[kWarpUnroll];
            bool act[kWarpUnroll];
#pragma unroll
            for (int u = 0; u < kWarpUnroll; ++u) {
                const int q = q0 + 32 * u;
                act[u] = q + lane < total;
                jv[u] = 0;
                a_u[u] = V(0);
                b_u[u] = V(0);
                if (q < total) {
                    const int c0 = __popc(__ballot_sync(kFull, incl <= q));
                    const int e = incl - q;
                    const unsigned ends = __reduce_or_sync(kFull, (e >= 1 && e <= 31) ? (1u << e) : 0u);
                    const int ci = c0 + __popc(ends & ((2u << lane) - 1u));
                    const IT st = __shfl_sync(kFull, start, ci);
                    if constexpr (NUM) a_u[u] = __shfl_sync(kFull, av, ci);
                    if (act[u]) {
                        const IT idx = st + (IT)(q + lane);
                        jv[u] = __ldg(op.b_ci + idx);
                        if constexpr (NUM) b_u[u] = __ldg(op.b_val + idx);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kWarpUnroll; ++u) {
                if (q0 + 32 * u < total) {
                    bool ok = act[u];
                    if (ok && (unsigned)jv[u] >= (unsigned)op.ncols) {
                        raise_err(err, kErrBadIndex);
                        ok = false;
                    }
                    f(ok, jv[u], a_u[u], b_u[u], pbase + q0 + 32 * u + lane);
                }
            }
        }
        pbase += total;
    }
}

// Every product of A entries [ab, ae), enumerated by a group of GS threads
// (one block, GS = NT): batches of GS entries are staged in shared memory
// (entries with an empty row of B dropped), the batch's products are split
// into one contiguous range per warp, and each warp walks its range 32
// products a step; a lane finds its entry from the set of entry ends inside
// the step (step_entry). f(act, j, a, b, p) is called by all 32 lanes of a
// warp together once per step of its range (p: the product's index among the
// row's products). sc: the group's product scratch (prod_scratch_bytes).
template <typename V, typename IT, bool NUM, int GS, typename F>
__device__ __forceinline__ void group_enum(const Operands<V> &op, int64_t ab, int64_t ae, const ProdScratch<V> &sc,
                                           int *err, F &&f) {
    using G = Group<GS, GS>;
    const int t = G::tid();
    const int lane = lane_id();
    const int w = G::wid();
    int pbase = 0;
    int k_next = -1;
    V av_next = V(0);
    if (ab + t < ae) {
        k_next = __ldg(op.a_ci + ab + t);
        if constexpr (NUM) av_next = op.a_val[ab + t];
    }
    for (int64_t base = ab; base < ae; base += GS) {
        int len = 0;
        int64_t bs = 0;
        const V av = av_next;
        if (base + t < ae) b_row_whole(op, k_next, len, bs, err);
        const long long packed = ((long long)(len > 0 ? 1 : 0) << 32) | (long long)len;
        long long tot64;
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
        const int per = ((total + G::kWarps - 1) / G::kWarps + 31) & ~31;
        const int lo = min(w * per, total);
        const int hi = min(lo + per, total);
        if (lo < hi) {
            int a = 0, b = nf;
            while (a < b) {
                const int m = (a + b) >> 1;
                if (sc.incl[m] <= lo) a = m + 1;
                else b = m;
            }
            int c0 = a;
            for (int pb = lo; pb < hi; pb += 32 * kWarpUnroll) {
                int jv[kWarpUnroll];
                V av_u[kWarpUnroll], bv[kWarpUnroll];
                bool act[kWarpUnroll];
#pragma unroll
                for (int u = 0; u < kWarpUnroll; ++u) {
                    const int q = pb + 32 * u;
                    act[u] = false;
                    jv[u] = 0;
                    av_u[u] = V(0);
                    bv[u] = V(0);
                    if (q < hi) {
                        act[u] = q + lane < hi;
                        const int e0 = sc.incl[c0] - q;   // same for all lanes
                        int ci;
                        if (e0 >= 32) {
                            ci = c0;                      // the whole step lies in entry c0
                            if (e0 == 32) ++c0;
                        } else {
                            const int c = c0 + lane;
                            const int e = c < nf ? sc.incl[c] - q : INT_MAX;
                            ci = c0 + step_entry(e);
                            c0 += __popc(__ballot_sync(kFull, e <= 32));
                        }
                        if (act[u]) {
                            const IT idx = (IT)sc.start[ci] + (IT)(q + lane);
                            jv[u] = __ldg(op.b_ci + idx);
                            if constexpr (NUM) {
                                bv[u] = __ldg(op.b_val + idx);
                                av_u[u] = sc.av[ci];
                            }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kWarpUnroll; ++u) {
                    const int q = pb + 32 * u;
                    if (q < hi) {
                        bool ok = act[u];
                        if (ok && (unsigned)jv[u] >= (unsigned)op.ncols) {
                            raise_err(err, kErrBadIndex);
                            ok = false;
                        }
                        f(ok, jv[u], av_u[u], bv[u], pbase + q + lane);
                    }
                }
            }
        }
        pbase += total;
        // the next batch stages its entries only after the first barrier of
        // its scan, which every warp reaches after its walk
    }
    G::sync();
}

}  // namespace smash
