// Numeric phase: values of C = A*B, rows sorted by column.
//
// Hashing Phase with values: each product a_ik*b_kj is merged into the row's
// table as it is produced: compare-and-swap claims the tag's slot (EMPTY = -1,
// +1 linear probing), an atomic add accumulates the value (the "atomic fetch
// and add" merge). Write-back Phase: the occupied slots are gathered, ordered
// by column and streamed to C's row (Version 1 sorts the table before
// streaming it out; the sort here is one of four, chosen per row):
//   - warp rank:   rows of <= 32 entries held by one warp; each entry's rank is
//                  the number of smaller tags (register shuffles);
//   - bitmap rank: a bitmap over the columns of B plus a prefix count per
//                  32-bit word gives every tag its position directly;
//   - bucket rank: counting sort of the tags by their high bits, then each
//                  tag's rank inside its (small) bucket (writeout.cuh);
//   - bitonic:     the compacted entries are sorted in shared memory (when
//                  the bucket arrays do not fit next to the tables).
// Table placements as in the symbolic phase: shared memory (k_num_hash),
// dense accumulators for dense rows (k_num_window: one column window of the
// row per work item, values indexed by column, occupancy in a bitmap), and a
// global-memory hash table (k_num_spill; Version 3's table in DRAM).
#include <climits>

#include "device_common.cuh"
#include "kernels.h"
#include "writeout.cuh"

namespace smash {

// ----- shared-memory hash rows -----------------------------------------------
// (the register cap of 64 lets 2048 threads per SM be resident: measured
// faster than the uncapped kernel at 72 registers and 43 % of the warps).
// CAP: capacity mode (out.row_nnz set); each mode leaves out the code the
// other needs.
template <typename V, int GS, int NT, bool CAP>
__global__ void __launch_bounds__(NT, 1024 / NT) k_num_hash(Operands<V> op, const int *rows, int count, int *token,
                                                 int tbits, HashCfg hc, int bsh, int bcap, int bm_words,
                                                 int bitmap_ratio, const RowGather *rec, NumOutT<V> out,
                                                 int *err) {
    // bsh >= 0: bucket-rank write-out (its T/4 counters and room for bcap
    // grouped pairs follow each group's table); bsh < 0: bitonic.
    using G = Group<GS, NT>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][G::kGroups], s_rowi[2][G::kGroups];
    const int T = 1 << tbits;
    if (bsh < 0) bcap = 0;
    // group layout (hash_group_bytes): keys, values, bucket counters, then the
    // product staging, whose room the write-out's grouped pairs reuse
    const size_t grp_bytes = hash_group_bytes<V, GS>(T, bcap);
    unsigned char *gb = smem + (size_t)G::gid() * grp_bytes;
    int *keys = (int *)gb;
    V *vals = (V *)(gb + (size_t)T * 4);
    int *bc = (int *)(gb + (size_t)T * (4 + sizeof(V)));    // T/4 bucket counters
    unsigned char *uni = (unsigned char *)(bc + (bcap > 0 ? (T >> 2) : 0));
    V *gv = (V *)uni;                                       // bcap grouped values
    int *gk = (int *)(uni + (size_t)bcap * sizeof(V));      // bcap grouped columns
    const ProdScratch<V> sc = carve_prod_scratch<V, GS>(uni);
    unsigned *bm = (unsigned *)(smem + (size_t)G::kGroups * grp_bytes);
    int *pre = (int *)(bm + bm_words);
    const int t = G::tid();
    bool clean = false;   // the table is EMPTY / 0 (left so by the bucket write-out)
    RowClaimPf<G> claim(token, rows, s_row, s_rowi);
    for (;;) {
        int i;
        const int r = claim.next(count, &i);
        if (r >= count) break;
        // the row's bounds in C and A and its product count, loaded together
        const int64_t cs = out.c_rp[i], ct = out.c_rp[i + 1];
        int64_t ab = __ldg(op.a_rp + i), ae = __ldg(op.a_rp + i + 1);
        const long long f_rec = rec ? rec[i].f : -1;
        int64_t c0;
        int n_exp;
        const bool ok = row_bounds_ok(cs, ct, out.c_nnz, c0, n_exp, err);
        const bool use_bm = (GS == NT) && bm_words > 0 && (long long)bm_words <= (long long)bitmap_ratio * n_exp;
        if (!clean) {
            for (int s = t; s < T; s += GS) {
                keys[s] = kEmpty;
                vals[s] = V(0);
            }
        }
        if (bsh >= 0)
            for (int s = t; s < (T >> 2); s += GS) bc[s] = 0;
        if (use_bm)
            for (int w = t; w < bm_words; w += GS) bm[w] = 0u;
        G::sync();
        if (!ok || !a_bounds_ok(ab, ae, op.a_nnz, err)) ab = ae = 0;
        // Rows with nothing to merge skip the table (exact mode: the row's
        // length equals its product count), and so do rows whose products fit
        // their room (capacity mode: expanded, sorted and merged by the
        // bucket write-out): each product is staged at its index. Float
        // values only: with double values the larger kernel slowed the hashed
        // rows more than the staged rows gained (R-MAT 16, float64).
        constexpr bool kStage = sizeof(V) == 4;
        const long long f_i = kStage && ok ? f_rec : -1;
        const bool direct =
            kStage && !CAP && bsh >= 0 && f_i >= 0 && f_i == (long long)n_exp && f_i <= bcap;
        const bool merge = kStage && CAP && bsh >= 0 && !use_bm && f_i >= 0 && f_i <= (long long)n_exp &&
                           2 * f_i <= T && f_i <= bcap;
        int tot, o;
        if (direct || merge) {
            group_products<V, true, GS, NT>(op, ab, ae, sc, err, [&](int j, V a, V bkj, int p) {
                if ((unsigned)p < (unsigned)T) {
                    keys[p] = j;
                    vals[p] = a * bkj;
                    atomicAdd(bc + (j >> bsh), 1);   // bucket counts for the write-out
                }
            });
            tot = (int)f_i;
            o = 0;
        } else {
            int cnt = 0, ovf = 0;
            group_products<V, true, GS, NT>(op, ab, ae, sc, err, [&](int j, V a, V bkj) {
                bool ins;
                const int h = hash_find_or_insert<false>(keys, tbits, hc, j, ins);
                if (h >= 0) {
                    atomicAdd(vals + h, a * bkj);
                    if (ins) {
                        ++cnt;
                        if (bsh >= 0) atomicAdd(bc + (j >> bsh), 1);   // bucket counts for the write-out
                    }
                } else if (CAP) {
                    ovf = 1;
                } else {
                    raise_err(err, kErrTableFull);
                }
            });
            // one reduction of (overflow flags, inserts): a row has at most
            // T <= 2^14 distinct columns, so the inserts fit the low 16 bits
            if constexpr (GS == 32) {
                tot = warp_sum(cnt);
                o = __any_sync(kFull, ovf);
                __syncwarp();
            } else {
                const int packed = G::template sum<int>(cnt | (ovf << 16), sc.red);
                tot = packed & 0xffff;
                o = packed >> 16;
            }
        }
        claim.prefetch(count);
        if (merge) {
            // (the runs are the row's entries, at most its room)
            const int runs = writeout_bucket_merge<V, GS, NT>(keys, vals, T, bc, gk, gv, bsh, tot, out, c0, sc.red);
            if (t == 0) out.row_nnz[i] = runs;
            clean = true;
            claim.publish();
            G::sync();
            continue;
        }
        bool over = false;
        if (CAP) {
            over = o != 0 || tot > n_exp;
            if (t == 0) out.row_nnz[i] = over ? -1 : tot;
            n_exp = tot;
        } else if (t == 0 && tot != n_exp) {
            raise_err(err, kErrCountMismatch);
        }
        clean = false;
        if (!over) {
            if (GS == 32 && tot <= 32) {
                writeout_warp_rank<V>(keys, vals, T, tot, n_exp, out, c0);
            } else if (use_bm) {
                writeout_bitmap<V, GS, NT>(keys, vals, T, bm, pre, bm_words, n_exp, out, c0, sc.red);
            } else if (bsh >= 0 && tot <= bcap) {
                writeout_bucket<V, GS, NT>(keys, vals, T, bc, gk, gv, bsh, tot, n_exp, out, c0, sc.red,
                                           direct ? tot : T);
                clean = true;
            } else {
                writeout_bitonic<V, GS, NT>(keys, vals, T, n_exp, out, c0, sc.red);
            }
        }
        claim.publish();
        G::sync();
    }
}

// ----- dense rows: (row, column window) work items ---------------------------
// A dense row's accumulator is cut into windows of cpc columns; every (row,
// window) pair is an independent item. The block owns one window's dense
// accumulator (values indexed by column, occupancy in a bitmap) in shared
// memory, enumerates only the products that land in the window (B sliced by
// window), and writes the window's columns in order at the window's offset in
// the row, known from the per-block column counts of the bitmap pass. No two
// blocks ever wait on each other.

// Position of the n-th (0-based) set bit of x (n < popc(x)), by halving.
__device__ __forceinline__ int nth_set_bit(unsigned x, int n) {
    int pos = 0;
    int c = __popc(x & 0xffffu);
    if (n >= c) { n -= c; x >>= 16; pos += 16; }
    c = __popc(x & 0xffu);
    if (n >= c) { n -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xfu);
    if (n >= c) { n -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (n >= c) { n -= c; x >>= 2; pos += 2; }
    if (n >= (int)(x & 1u)) pos += 1;
    return pos;
}

constexpr int kEnumUnroll = 4;   // steps of 32 products whose loads are issued together

// Every product of A entries [ab, ae) whose column lies in slice op.slice of
// the sliced B, enumerated by one warp: lane l of a batch of 32 entries holds
// entry l's slice (start, length, a_ik), entries with an empty slice are
// moved out of the way by shuffles, a scan lays the batch's products on one
// line and each step hands 32 consecutive products to the 32 lanes (as in
// the warp-row enumerator). f(act, j, a, b) is called by all 32 lanes together
// once per step.
template <typename V, typename F>
__device__ __forceinline__ void slice_enum(const Operands<V> &op, int64_t ab, int64_t ae, int *err, F &&f) {
    const int lane = lane_id();
    for (int64_t base = ab; base < ae; base += 32) {
        int len = 0;
        int32_t bs = 0;
        V av = V(0);
        if (base + lane < ae) {
            const int k = __ldg(op.a_ci + base + lane);
            if ((unsigned)k < (unsigned)op.b_rows) {
                const int32_t *w = op.b_woff + (size_t)k * (op.nslices + 1) + op.slice;
                bs = w[0];
                len = w[1] - bs;
            } else {
                raise_err(err, kErrBadIndex);
            }
            av = op.a_val[base + lane];
        }
        const unsigned nz = __ballot_sync(kFull, len > 0);
        if (nz == 0u) continue;
        const int nv = __popc(nz);
        if (nv < 32 && nz != (1u << nv) - 1u) {
            const int src = lane < nv ? nth_set_bit(nz, lane) : 0;
            len = __shfl_sync(kFull, len, src);
            bs = __shfl_sync(kFull, bs, src);
            av = __shfl_sync(kFull, av, src);
            if (lane >= nv) len = 0;
        }
        const int incl = warp_incl_scan(len);
        const int total = __shfl_sync(kFull, incl, 31);
        const int32_t start = bs - (incl - len);   // product p of this entry reads B at start + p
        for (int q0 = 0; q0 < total; q0 += 32 * kEnumUnroll) {
            int jv[kEnumUnroll];
            V a_u[kEnumUnroll], b_u[kEnumUnroll];
            bool act[kEnumUnroll];
#pragma unroll
            for (int u = 0; u < kEnumUnroll; ++u) {
                const int q = q0 + 32 * u;
                act[u] = q + lane < total;
                jv[u] = -1;
                a_u[u] = V(0);
                b_u[u] = V(0);
                if (q < total) {
                    const int c0 = __popc(__ballot_sync(kFull, incl <= q));
                    const int e = incl - q;
                    const unsigned ends = __reduce_or_sync(kFull, (e >= 1 && e <= 31) ? (1u << e) : 0u);
                    const int ci = c0 + __popc(ends & ((2u << lane) - 1u));
                    const int32_t st = __shfl_sync(kFull, start, ci);
                    a_u[u] = __shfl_sync(kFull, av, ci);
                    if (act[u]) {
                        jv[u] = __ldg(op.b_ci + st + q + lane);
                        b_u[u] = __ldg(op.b_val + st + q + lane);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kEnumUnroll; ++u) {
                if (q0 + 32 * u < total) {
                    bool ok = act[u];
                    if (ok && (unsigned)jv[u] >= (unsigned)op.ncols) {
                        raise_err(err, kErrBadIndex);
                        ok = false;
                    }
                    f(ok, jv[u], a_u[u], b_u[u]);
                }
            }
        }
    }
}

// OWN (owner computes): warp q of the block owns the window's columns of
// every kWarps-th group of 32 columns from group q on (B sliced by warp:
// slices [w * kWarps, (w + 1) * kWarps) make up window w; interleaved, so
// that columns crowded at one end of the window spread over all warps) and
// adds its products with plain shared-memory read-modify-writes:
// no other warp touches its columns, and lanes of one step that hit the same
// column take turns (each writes its lane to the column's owner byte, the
// lane that reads itself back adds; the others try again), so no atomic and
// no compare-and-swap retry, and each product costs one add.
template <typename V, int NT, bool OWN>
__global__ void __launch_bounds__(NT) k_num_window(Operands<V> op, const int *rows, int count, int nw, int cpc,
                                                   int subs_per_win, WinCount wc, WinArena ar, NumOutT<V> out,
                                                   unsigned long long *token, int *err) {
    const bool arena = ar.ci != nullptr;
    constexpr int kWarps = NT / 32;
    constexpr int kMaxChunks = kMaxWinCols / 1024;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item[2], s_aoff;
    __shared__ int s_off, s_cnt;
    __shared__ int s_chunk[kMaxChunks + 1];
    const int words = cpc >> 5;
    V *acc = (V *)smem;
    unsigned *bm = (unsigned *)(smem + (size_t)cpc * sizeof(V));
    const ProdScratch<V> sc = carve_prod_scratch<V, NT>((unsigned char *)(bm + words));
    unsigned char *own = (unsigned char *)(bm + words);   // OWN: owner byte of each column
    const int t = threadIdx.x;
    const int lane = lane_id();
    const int wp = t >> 5;
    for (int j = t; j < cpc; j += NT) acc[j] = V(0);
    for (int w = t; w < words; w += NT) bm[w] = 0u;
    const int64_t items = (int64_t)count * nw;
    // items are claimed one ahead (the claim's latency hides behind the
    // current item); s_item[par] holds the claimed next item, written before
    // the item's closing barrier and read after it
    int par = 0;
    if (t == 0) s_item[0] = (long long)atomicAdd(token, 1ull);
    __syncthreads();
    for (;;) {
        const int64_t item = s_item[par];
        par ^= 1;
        if (item >= items) break;
        if (t == 0) s_item[par] = (long long)atomicAdd(token, 1ull);
        const int r = (int)(item / nw);
        const int w = (int)(item - (int64_t)r * nw);
        const int i = rows[r];
        // capacity mode: skip a row that overflowed. In arena mode other blocks
        // update row_nnz[i] meanwhile: one thread reads it for the whole block.
        bool skip = false;
        if (out.row_nnz) {
            if (t == 0) s_off = out.row_nnz[i] < 0 ? 1 : 0;
            __syncthreads();
            skip = s_off != 0;
            __syncthreads();
        }
        int slot = -1;
        int64_t c0 = 0;
        int n_exp = 0;
        if (!arena) {
            slot = wc.wslot[i];
            if (!skip && slot < 0) {
                if (t == 0) raise_err(err, kErrCountMismatch);
                skip = true;
            }
            if (!skip && !out_range(out, i, c0, n_exp, err)) skip = true;
        }
        if (skip) {
            __syncthreads();
            continue;
        }
        if (!arena && wp == 0) {
            const uint16_t *sub = wc.wcnt + (size_t)slot * wc.nsub;
            const int s_lo = w * subs_per_win;
            const int s_hi = min(s_lo + subs_per_win, wc.nsub);
            int before = 0, mine = 0;
            for (int q = lane; q < s_hi; q += 32) {
                const int c = sub[q];
                if (q < s_lo) before += c;
                else mine += c;
            }
            before = warp_sum(before);
            mine = warp_sum(mine);
            if (lane == 0) {
                s_off = before;
                s_cnt = mine;
            }
        }
        const int lo = w * cpc;
        const int width = min(cpc, op.ncols - lo);
        int64_t ab = 0, ae = 0;
        a_row_range(op, i, ab, ae, err);
        if constexpr (OWN) {
            op.slice = w * kWarps + wp;
            slice_enum<V>(op, ab, ae, err, [&](bool act, int j, V a, V bkj) {
                const unsigned off = (unsigned)(j - lo);
                bool pend = act && off < (unsigned)width && ((off >> 5) & (kWarps - 1)) == (unsigned)wp;
                const V v = a * bkj;
                while (__any_sync(kFull, pend)) {
                    if (pend) own[off] = (unsigned char)lane;
                    __syncwarp();
                    const bool win = pend && own[off] == (unsigned char)lane;
                    if (win) {
                        acc[off] += v;
                        const unsigned bit = 1u << (off & 31);
                        unsigned *bw = bm + (off >> 5);
                        if (!(*(volatile unsigned *)bw & bit)) atomicOr(bw, bit);
                    }
                    __syncwarp();
                    pend = pend && !win;
                }
            });
            __syncthreads();
        } else {
            op.slice = w;
            group_products<V, true, NT, NT>(op, ab, ae, sc, err, [&](int j, V a, V bkj) {
                const unsigned off = (unsigned)(j - lo);
                if (off < (unsigned)width) {
                    atomicAdd(acc + off, a * bkj);
                    const unsigned bit = 1u << (off & 31);
                    unsigned *bw = bm + (off >> 5);
                    if (!(*(volatile unsigned *)bw & bit)) atomicOr(bw, bit);
                }
            });
        }
        // write-out in chunks of 32 bitmap words (1024 columns): chunk totals,
        // their prefix, then every chunk's columns in order.
        const int wwords = (width + 31) >> 5;
        const int nch = (wwords + 31) >> 5;
        for (int c = wp; c < nch; c += kWarps) {
            const int x = 32 * c + lane;
            const int tot = warp_sum(x < wwords ? __popc(bm[x]) : 0);
            if (lane == 0) s_chunk[c] = tot;
        }
        __syncthreads();
        if (wp == 0) {
            int run = 0;
            for (int c0w = 0; c0w < nch; c0w += 32) {
                const int c = c0w + lane;
                const int v = c < nch ? s_chunk[c] : 0;
                const int incl = warp_incl_scan(v);
                if (c < nch) s_chunk[c] = run + incl - v;
                run += __shfl_sync(kFull, incl, 31);
            }
            if (lane == 0) s_chunk[nch] = run;
        }
        __syncthreads();
        const int total = s_chunk[nch];
        int base = 0;
        bool ok;
        if (arena) {
            // reserve the window's room in the arena
            if (t == 0) {
                const long long off = (long long)atomicAdd(ar.top, (unsigned long long)total);
                const bool fits = off + total <= ar.cap;
                s_aoff = fits ? off : -1;
                ar.desc_off[item] = fits ? off : -1;
                ar.desc_cnt[item] = total;
                if (fits) atomicAdd(out.row_nnz + i, total);
                else atomicOr(out.row_nnz + i, INT_MIN);
            }
            __syncthreads();
            ok = s_aoff >= 0;
            c0 = ok ? s_aoff : 0;
        } else {
            base = s_off;
            if (t == 0 && total != s_cnt) raise_err(err, kErrCountMismatch);
            ok = total == s_cnt && (int64_t)base + total <= (int64_t)n_exp;
        }
        int32_t *dst_ci = arena ? ar.ci : out.c_ci;
        V *dst_val = arena ? (V *)ar.val : out.c_val;
        for (int c = wp; c < nch; c += kWarps) {
            const int x = 32 * c + lane;
            const unsigned word = x < wwords ? bm[x] : 0u;
            const int incl = warp_incl_scan(__popc(word));
            const int T = __shfl_sync(kFull, incl, 31);
            const int64_t cb = c0 + base + s_chunk[c];
            if (T >= 256) {
                // dense chunk: word by word, lane = bit
                for (int q = 0; q < 32; ++q) {
                    const unsigned wq = __shfl_sync(kFull, word, q);
                    const int pre = __shfl_sync(kFull, incl, q) - __popc(wq);
                    if ((wq >> lane) & 1u) {
                        const int col = ((32 * c + q) << 5) + lane;
                        const V v = acc[col];
                        acc[col] = V(0);
                        const int64_t pos = cb + pre + __popc(wq & lanemask_lt());
                        if (ok) {
                            __stcs(dst_ci + (pos), lo + col);
                            __stcs(dst_val + (pos), v);
                        }
                    }
                }
            } else {
                // sparse chunk: 32 consecutive outputs per step; the owner word of
                // output o is the first lane whose inclusive count exceeds o
                for (int o0 = 0; o0 < T; o0 += 32) {
                    const int o = o0 + lane;
                    int L = 0;
#pragma unroll
                    for (int st = 16; st >= 1; st >>= 1) {
                        const int v = __shfl_sync(kFull, incl, L + st - 1);
                        if (v <= o) L += st;
                    }
                    const unsigned wl = __shfl_sync(kFull, word, L);
                    const int el = __shfl_sync(kFull, incl, L) - __popc(wl);
                    if (o < T) {
                        const int col = ((32 * c + L) << 5) + nth_set_bit(wl, o - el);
                        const V v = acc[col];
                        acc[col] = V(0);
                        if (ok) {
                            __stcs(dst_ci + (cb + o), lo + col);
                            __stcs(dst_val + (cb + o), v);
                        }
                    }
                }
            }
            if (x < wwords) bm[x] = 0u;
        }
        __syncthreads();
    }
}


// ----- global-memory hash rows ------------------------------------------------
template <int NT>
__device__ __forceinline__ void block_minmax(int &mn, int &mx, int *s_mm) {
    mn = warp_min(mn);
    mx = warp_max(mx);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) {
        s_mm[w] = mn;
        s_mm[32 + w] = mx;
    }
    __syncthreads();
    mn = INT_MAX;
    mx = INT_MIN;
    for (int k = 0; k < NT / 32; ++k) {
        mn = min(mn, s_mm[k]);
        mx = max(mx, s_mm[32 + k]);
    }
    __syncthreads();
}

constexpr int kSpillUnroll = 8;

template <typename V, int NT>
__global__ void __launch_bounds__(NT) k_num_spill(Operands<V> op, const int *rows, int count, int *token,
                                                  HashCfg hc, float inv_load, int spill_tbits, int *keys_all,
                                                  V *vals_all, int win_words, NumOutT<V> out, int *err) {
    using G = Group<NT, NT>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row;
    __shared__ int s_mm[64];
    unsigned *bm = (unsigned *)smem;
    int *pre = (int *)(bm + win_words);
    const ProdScratch<V> sc = carve_prod_scratch<V, NT>(smem + (size_t)win_words * 8);
    int *keys = keys_all + ((size_t)blockIdx.x << spill_tbits);
    V *vals = vals_all + ((size_t)blockIdx.x << spill_tbits);
    const int t = threadIdx.x;
    const long long WIN = (long long)win_words * 32;
    for (;;) {
        if (t == 0) s_row = atomicAdd(token, 1);
        __syncthreads();
        const int r = s_row;
        if (r >= count) break;
        const int i = rows[r];
        int64_t c0;
        int n_exp;
        const bool ok = out_range(out, i, c0, n_exp, err);
        int tb = table_bits(n_exp, inv_load);
        if (tb > spill_tbits) {
            if (t == 0) raise_err(err, kErrTableFull);
            tb = spill_tbits;
        }
        const int T = 1 << tb;
        for (int s = t; s < T; s += NT) {
            __stcg(keys + s, kEmpty);
            __stcg(vals + s, V(0));
        }
        __threadfence();
        __syncthreads();
        int64_t ab = 0, ae = 0;
        if (ok) a_row_range(op, i, ab, ae, err);
        int cnt = 0, ovf = 0;
        group_products<V, true, NT, NT>(op, ab, ae, sc, err, [&](int j, V a, V bkj) {
            const V v = a * bkj;
            bool ins;
            const int h = hash_find_or_insert<true>(keys, tb, hc, j, ins);
            if (h >= 0) {
                atomicAdd(vals + h, v);
                cnt += ins ? 1 : 0;
            } else if (out.row_nnz) {
                ovf = 1;
            } else {
                raise_err(err, kErrTableFull);
            }
        });
        __threadfence();
        int tot = G::template sum<int>(cnt, sc.red);
        if (out.row_nnz) {
            const int o = G::template sum<int>(ovf, sc.red);
            const bool over = o != 0 || tot > n_exp;
            if (t == 0) out.row_nnz[i] = over ? -1 : tot;
            n_exp = tot;
            if (over) tot = 0;   // nothing to write
        } else if (t == 0 && tot != n_exp) {
            raise_err(err, kErrCountMismatch);
        }
        // the table lives in global memory: every scan below keeps kSpillUnroll
        // loads in flight per thread
        int mn = INT_MAX, mx = INT_MIN;
        for (int s0 = t; s0 < T; s0 += kSpillUnroll * NT) {
            int k[kSpillUnroll];
#pragma unroll
            for (int u = 0; u < kSpillUnroll; ++u) k[u] = s0 + u * NT < T ? __ldcg(keys + s0 + u * NT) : kEmpty;
#pragma unroll
            for (int u = 0; u < kSpillUnroll; ++u) {
                if (k[u] != kEmpty) {
                    mn = min(mn, k[u]);
                    mx = max(mx, k[u]);
                }
            }
        }
        block_minmax<NT>(mn, mx, s_mm);
        long long done = 0;
        if (tot > 0) {
            for (long long w0 = ((long long)mn / WIN) * WIN; w0 <= (long long)mx; w0 += WIN) {
                for (int w = t; w < win_words; w += NT) bm[w] = 0u;
                __syncthreads();
                for (int s0 = t; s0 < T; s0 += kSpillUnroll * NT) {
                    int k[kSpillUnroll];
#pragma unroll
                    for (int u = 0; u < kSpillUnroll; ++u)
                        k[u] = s0 + u * NT < T ? __ldcg(keys + s0 + u * NT) : kEmpty;
#pragma unroll
                    for (int u = 0; u < kSpillUnroll; ++u) {
                        if (k[u] != kEmpty && k[u] >= w0 && k[u] < w0 + WIN) {
                            const int d = (int)(k[u] - w0);
                            atomicOr(bm + (d >> 5), 1u << (d & 31));
                        }
                    }
                }
                __syncthreads();
                const int wt = bitmap_prefix<NT, NT>(bm, pre, win_words, sc.red);
                __syncthreads();
                for (int s0 = t; s0 < T; s0 += kSpillUnroll * NT) {
                    int k[kSpillUnroll];
                    V v[kSpillUnroll];
#pragma unroll
                    for (int u = 0; u < kSpillUnroll; ++u) {
                        const int s = s0 + u * NT;
                        k[u] = s < T ? __ldcg(keys + s) : kEmpty;
                        v[u] = s < T ? __ldcg(vals + s) : V(0);
                    }
#pragma unroll
                    for (int u = 0; u < kSpillUnroll; ++u) {
                        if (k[u] != kEmpty && k[u] >= w0 && k[u] < w0 + WIN) {
                            const int d = (int)(k[u] - w0);
                            const long long pos =
                                done + pre[d >> 5] + __popc(bm[d >> 5] & ((1u << (d & 31)) - 1u));
                            if (pos < n_exp) {
                                __stcs(out.c_ci + (c0 + pos), k[u]);
                                __stcs(out.c_val + (c0 + pos), v[u]);
                            }
                        }
                    }
                }
                done += wt;
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
int max_smem_per_block() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        cudaGetDevice(&dev);
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cached = v > 0 ? v : 232448;
    }
    return cached;
}

int max_smem_per_sm() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        cudaGetDevice(&dev);
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cached = v > 0 ? v : 233472;
    }
    return cached;
}

template <typename V>
static Operands<V> num_operands(const RawOperands &r) {
    Operands<V> o;
    o.a_rp = r.a_rp;
    o.a_ci = r.a_ci;
    o.a_val = (const V *)r.a_val;
    o.b_rp = r.b_rp;
    o.b_ci = r.b_ci;
    o.b_val = (const V *)r.b_val;
    o.a_nnz = r.a_nnz;
    o.b_nnz = r.b_nnz;
    o.b_rows = r.b_rows;
    o.ncols = r.ncols;
    return o;
}

template <typename V>
static NumOutT<V> num_out(const NumOut &o) {
    return NumOutT<V>{o.c_rp, o.c_ci, (V *)o.c_val, o.c_nnz, o.row_nnz};
}

static int threads_per_row(int tbits, int shift) {
    int t = 1 << (tbits > shift ? tbits - shift : 0);
    if (t < 32) t = 32;
    if (t > 1024) t = 1024;
    return t;
}

static int block_threads(int gs) { return gs < 64 ? 256 : gs; }

template <typename V>
static size_t num_hash_smem(int tbits, int gs, int bm_words, int bcap = 0) {
    const int nt = block_threads(gs);
    const int groups = nt / gs;
    const int T = 1 << tbits;
    size_t grp = 0;
    switch (gs) {
        case 32: grp = hash_group_bytes<V, 32>(T, bcap); break;
        case 64: grp = hash_group_bytes<V, 64>(T, bcap); break;
        case 128: grp = hash_group_bytes<V, 128>(T, bcap); break;
        case 256: grp = hash_group_bytes<V, 256>(T, bcap); break;
        case 512: grp = hash_group_bytes<V, 512>(T, bcap); break;
        default: grp = hash_group_bytes<V, 1024>(T, bcap); break;
    }
    return (size_t)groups * grp + (size_t)bm_words * 8;
}

bool num_hash_bitmap_fits(int dtype, int tbits, int ncols) {
    const int words = (ncols + 31) / 32;
    const size_t s = dtype ? num_hash_smem<double>(tbits, 1024, words) : num_hash_smem<float>(tbits, 1024, words);
    return s <= (size_t)max_smem_per_block();
}

template <typename K>
static int resident_grid(K kernel, int nt, size_t smem, int sms, long long want_blocks, int cap_per_sm = 64) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > cap_per_sm) per_sm = cap_per_sm;
    long long cap = (long long)per_sm * sms;
    return (int)(want_blocks < cap ? want_blocks : cap);
}

template <typename V, int GS>
static void num_hash_go(const Operands<V> &op, const int *rows, int count, int *token, const HashLaunch &hl,
                        float inv_load, int bitmap_ratio, const RowGather *rec, const NumOutT<V> &out, int *err,
                        cudaStream_t s) {
    // one group per block from 64 threads up (block barriers, no named ones)
    constexpr int NT = GS < 64 ? 256 : GS;
    constexpr int groups = NT / GS;
    const int T = 1 << hl.tbits;
    const size_t lim = (size_t)max_smem_per_block();
    int bm_words = 0;
    if (GS == NT && bitmap_ratio > 0) {
        const int words = (op.ncols + 31) / 32;
        if (num_hash_smem<V>(hl.tbits, GS, words, T / 2) <= lim) bm_words = words;
    }
    // bucket-rank write-out when its arrays fit next to the tables: room for
    // the rows' distinct columns, T/2 at loads up to 0.5, else 3T/4 (loads up
    // to 0.75) when that fits
    int bcap = inv_load >= 2.f ? T / 2 : T - T / 4;
    // every row of the bin has more than (T/2)/inv_load columns (else it would
    // sit in a smaller bin): when that already makes the bitmap write-out
    // their choice, the bucket arrays would only take shared memory (and
    // resident groups) away
    const long long n_min = (long long)((T / 2) / inv_load) + 1;
    if (bm_words > 0 && (long long)bm_words <= (long long)bitmap_ratio * n_min) bcap = 0;
    if (bcap > 0 && num_hash_smem<V>(hl.tbits, GS, bm_words, bcap) > lim) bcap = T / 2;
    if (bcap > 0 && num_hash_smem<V>(hl.tbits, GS, bm_words, bcap) > lim) bcap = 0;
    const bool buckets = bcap > 0;
    const size_t smem = num_hash_smem<V>(hl.tbits, GS, bm_words, bcap);
    auto kern = out.row_nnz ? k_num_hash<V, GS, NT, true> : k_num_hash<V, GS, NT, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = resident_grid(kern, NT, smem, hl.sms, (count + groups - 1) / groups);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    // buckets: T/4 of them over the column range, by the high bits
    const int bsh = !buckets ? -1 : hl.colbits > hl.tbits - 2 ? hl.colbits - (hl.tbits - 2) : 0;
    kern<<<grid, NT, smem, s>>>(op, rows, count, token, hl.tbits, hc, bsh, bcap, bm_words, bitmap_ratio, rec, out,
                                err);
}

template <typename V>
static void num_hash_typed(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                           float inv_load, int bitmap_ratio, const RowGather *rec, const NumOut &o, int *err,
                           cudaStream_t s) {
    const Operands<V> op = num_operands<V>(r);
    const NumOutT<V> out = num_out<V>(o);
    switch (threads_per_row(hl.tbits, hl.group_shift)) {
        case 32: num_hash_go<V, 32>(op, rows, count, token, hl, inv_load, bitmap_ratio, rec, out, err, s); break;
        case 64: num_hash_go<V, 64>(op, rows, count, token, hl, inv_load, bitmap_ratio, rec, out, err, s); break;
        case 128: num_hash_go<V, 128>(op, rows, count, token, hl, inv_load, bitmap_ratio, rec, out, err, s); break;
        case 256: num_hash_go<V, 256>(op, rows, count, token, hl, inv_load, bitmap_ratio, rec, out, err, s); break;
        case 512: num_hash_go<V, 512>(op, rows, count, token, hl, inv_load, bitmap_ratio, rec, out, err, s); break;
        default: num_hash_go<V, 1024>(op, rows, count, token, hl, inv_load, bitmap_ratio, rec, out, err, s); break;
    }
}

void launch_num_hash(int dtype, const RawOperands &r, const int *rows, int count, int *token,
                     const HashLaunch &hl, float inv_load, int bitmap_ratio, const RowGather *rec, const NumOut &out,
                     int *err, cudaStream_t s) {
    if (count <= 0) return;
    if (dtype) num_hash_typed<double>(r, rows, count, token, hl, inv_load, bitmap_ratio, rec, out, err, s);
    else num_hash_typed<float>(r, rows, count, token, hl, inv_load, bitmap_ratio, rec, out, err, s);
}

int dense_bitmap_max_cols() {
    const size_t avail = (size_t)max_smem_per_block() - prod_scratch_bytes<float, 1024>() - 64;
    return (int)((avail / 4) * 32);
}

static int window_threads(int blocks_per_sm) { return blocks_per_sm <= 1 ? 1024 : blocks_per_sm == 2 ? 512 : 256; }

// Accumulator, occupancy bitmap, then the product staging (atomic adds) or
// the columns' owner bytes (owner computes).
template <typename V, int NT>
static size_t window_smem(int cpc, bool own) {
    return (size_t)cpc * sizeof(V) + (size_t)(cpc / 32) * 4 + (own ? (size_t)cpc : num_scratch_bytes<V, NT>());
}

template <typename V>
static size_t window_smem_nt(int cpc, int nt, bool own) {
    return nt == 1024 ? window_smem<V, 1024>(cpc, own)
                      : nt == 512 ? window_smem<V, 512>(cpc, own) : window_smem<V, 256>(cpc, own);
}

int window_warps(int blocks_per_sm) { return window_threads(blocks_per_sm < 1 ? 1 : blocks_per_sm) / 32; }

int num_window_cols(int dtype, int blocks_per_sm, bool own) {
    const int bps = blocks_per_sm < 1 ? 1 : blocks_per_sm;
    const int nt = window_threads(bps);
    // per-block budget: the SM's shared memory shared by bps blocks (1 KB
    // reserved per block, ~1 KB of static shared variables)
    long long budget = (long long)max_smem_per_sm() / bps - 1024 - 1024;
    if (budget > max_smem_per_block() - 1024) budget = max_smem_per_block() - 1024;
    int best = 0;
    for (int cpc = kSubCols; cpc <= kMaxWinCols; cpc += kSubCols) {
        const size_t need = dtype ? window_smem_nt<double>(cpc, nt, own) : window_smem_nt<float>(cpc, nt, own);
        if ((long long)need <= budget) best = cpc;
    }
    return best;
}

template <typename V, int NT>
static void num_window_go(Operands<V> op, const BSlices &sl, const int *rows, int count, unsigned long long *token,
                          const HashLaunch &hl, const WinCount &wc, const WinArena &ar, const NumOutT<V> &out,
                          int *err, cudaStream_t s) {
    const bool own = sl.per_win > 1;   // one slice per warp: owner computes
    int cpc = sl.cpc;
    int subs = cpc / kSubCols;
    if (sl.nslices <= 1) {
        cpc = (op.ncols + 31) & ~31;   // one window holds every column
        subs = wc.nsub;
    } else {
        op.b_ci = sl.ci;
        op.b_val = (const V *)sl.val;
        op.b_woff = sl.woff;
        op.nslices = sl.nslices;
    }
    const int nw = sl.nslices <= 1 ? 1 : sl.nslices / sl.per_win;
    const long long items = (long long)count * nw;
    const size_t smem = window_smem<V, NT>(cpc, own);
    if (own) {
        auto kern = k_num_window<V, NT, true>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int grid = resident_grid(kern, NT, smem, hl.sms, items);
        kern<<<grid, NT, smem, s>>>(op, rows, count, nw, cpc, subs, wc, ar, out, token, err);
    } else {
        auto kern = k_num_window<V, NT, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int grid = resident_grid(kern, NT, smem, hl.sms, items);
        kern<<<grid, NT, smem, s>>>(op, rows, count, nw, cpc, subs, wc, ar, out, token, err);
    }
}

template <typename V>
static void num_window_typed(const RawOperands &r, const int *rows, int count, unsigned long long *token,
                             const HashLaunch &hl, const BSlices &sl, const WinCount &wc, const WinArena &ar,
                             const NumOut &o, int *err, cudaStream_t s) {
    const Operands<V> op = num_operands<V>(r);
    const NumOutT<V> out = num_out<V>(o);
    switch (window_threads(hl.dense_blocks)) {
        case 1024: num_window_go<V, 1024>(op, sl, rows, count, token, hl, wc, ar, out, err, s); break;
        case 512: num_window_go<V, 512>(op, sl, rows, count, token, hl, wc, ar, out, err, s); break;
        default: num_window_go<V, 256>(op, sl, rows, count, token, hl, wc, ar, out, err, s); break;
    }
}

void launch_num_window(int dtype, const RawOperands &r, const int *rows, int count, unsigned long long *token,
                       const HashLaunch &hl, const BSlices &sl, const WinCount &wc, const WinArena &ar,
                       const NumOut &out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    cudaMemsetAsync(token, 0, sizeof(unsigned long long), s);
    if (dtype) num_window_typed<double>(r, rows, count, token, hl, sl, wc, ar, out, err, s);
    else num_window_typed<float>(r, rows, count, token, hl, sl, wc, ar, out, err, s);
}

// One warp per (row, window) item of the arena rows: the window's columns go
// to C after those of the row's earlier windows.
template <typename V>
__global__ void __launch_bounds__(256) k_arena_compact(const int *rows, int count, int nw, WinArena ar,
                                                       const uint8_t *ovf, const int64_t *c_rp, int32_t *c_ci,
                                                       V *c_val) {
    const int lane = lane_id();
    const int64_t items = (int64_t)count * nw;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += warps) {
        const int r = (int)(it / nw);
        const int w = (int)(it - (int64_t)r * nw);
        const int i = rows[r];
        if (ovf[i] != 2) continue;
        int before = 0;
        for (int q = lane; q < w; q += 32) before += ar.desc_cnt[(int64_t)r * nw + q];
        before = warp_sum(before);
        const int n = ar.desc_cnt[it];
        const int64_t src = ar.desc_off[it];
        const int64_t dst = c_rp[i] + before;
        // read-only sources (no aliasing with C): several loads in flight
        const int32_t *__restrict__ sci = ar.ci + src;
        const V *__restrict__ sv = (const V *)ar.val + src;
        int32_t *__restrict__ dci = c_ci + dst;
        V *__restrict__ dv = c_val + dst;
        for (int k0 = 0; k0 < n; k0 += 32 * 8) {
            int32_t ci[8];
            V va[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + 32 * u + lane;
                if (k < n) {
                    ci[u] = __ldg(sci + k);
                    va[u] = __ldg(sv + k);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + 32 * u + lane;
                if (k < n) {
                    dci[k] = ci[u];
                    dv[k] = va[u];
                }
            }
        }
    }
}

void launch_arena_compact(int dtype, const int *rows, int count, int nw, const WinArena &ar, const uint8_t *ovf,
                          const int64_t *c_rp, int32_t *c_ci, void *c_val, int sms, cudaStream_t s) {
    if (count <= 0) return;
    const int64_t items = (int64_t)count * nw;
    const int64_t blocks = (items + 7) / 8;
    const int64_t cap = (int64_t)sms * 8;
    const int grid = (int)(blocks < cap ? blocks : cap);
    if (dtype) k_arena_compact<double><<<grid, 256, 0, s>>>(rows, count, nw, ar, ovf, c_rp, c_ci, (double *)c_val);
    else k_arena_compact<float><<<grid, 256, 0, s>>>(rows, count, nw, ar, ovf, c_rp, c_ci, (float *)c_val);
}

__global__ void k_mark_rows(const int *rows, int count, const int *row_nnz, uint8_t *ovf) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < count) {
        const int i = rows[r];
        if (row_nnz[i] >= 0) ovf[i] = 2;
    }
}

void launch_mark_rows(const int *rows, int count, const int *row_nnz, uint8_t *ovf, cudaStream_t s) {
    if (count > 0) k_mark_rows<<<(count + 255) / 256, 256, 0, s>>>(rows, count, row_nnz, ovf);
}

__global__ void k_zero_rows(const int *rows, int count, int *a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < count) a[rows[r]] = 0;
}

void launch_zero_rows(const int *rows, int count, int *a, cudaStream_t s) {
    if (count > 0) k_zero_rows<<<(count + 255) / 256, 256, 0, s>>>(rows, count, a);
}

int num_spill_grid(int dtype, const HashLaunch &hl) {
    (void)dtype;
    const int per = hl.blocks_per_sm > 0 ? hl.blocks_per_sm : 1;
    return hl.sms * per;
}

template <typename V>
static void num_spill_typed(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                            float inv_load, int spill_tbits, void *tables, const NumOut &o, int *err,
                            cudaStream_t s) {
    const Operands<V> op = num_operands<V>(r);
    const NumOutT<V> out = num_out<V>(o);
    int words = (r.ncols + 31) / 32;
    if (words > 16384) words = 16384;
    const size_t smem = (size_t)words * 8 + num_scratch_bytes<V, 1024>();
    auto kern = k_num_spill<V, 1024>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int gridmax = num_spill_grid(sizeof(V) == 8, hl);
    const int grid = count < gridmax ? count : gridmax;
    int *keys = (int *)tables;
    V *vals = (V *)((char *)tables + ((size_t)gridmax << spill_tbits) * 4);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    kern<<<grid, 1024, smem, s>>>(op, rows, count, token, hc, inv_load, spill_tbits, keys, vals, words, out, err);
}

void launch_num_spill(int dtype, const RawOperands &r, const int *rows, int count, int *token,
                      const HashLaunch &hl, float inv_load, int spill_tbits, void *tables, const NumOut &out,
                      int *err, cudaStream_t s) {
    if (count <= 0) return;
    if (dtype) num_spill_typed<double>(r, rows, count, token, hl, inv_load, spill_tbits, tables, out, err, s);
    else num_spill_typed<float>(r, rows, count, token, hl, inv_load, spill_tbits, tables, out, err, s);
}

}  // namespace smash
