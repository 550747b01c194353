// Warp rows: one warp per row of C, for the bins whose tables hold up to a
// few hundred columns (the bulk of the rows of R-MAT products).
//
// Hashing Phase, with the row's partial products enumerated from registers
// (warp_enum.cuh: lanes hold a batch of A's entries, each step hands 32
// consecutive products to the 32 lanes, loads of B coalesced).
//
// Insertion tries the compare-and-swap EMPTY -> j first; a slot that holds
// another tag sends the lane one slot on (linear probing with wrap-around,
// the Hashing Phase's collision resolution). The numeric kernel adds a_ik*b_kj
// to the slot's value (atomic add) and appends every newly claimed slot to a
// list, so that the Write-back Phase visits the row's entries only, never the
// whole table: the entries move to registers (their slots back to EMPTY), a
// counting sort by the high bits of the column groups them by bucket in the
// table's own memory, each entry's rank inside its bucket gives its place, and
// the row streams to C in column order.
//
// Included by k_warp_f32.cu (the symbolic kernel, float values, the launch
// entries) and k_warp_f64.cu (double values): two translation units
// compiled side by side.
#pragma once
#include <climits>

#include "device_common.cuh"
#include "kernels.h"
#include "warp_enum.cuh"
#include "writeout.cuh"

namespace smash {

constexpr int kWarpRowWarps = 4;   // warps (rows in flight) per block
constexpr int kWarpMaxList = 512;  // most columns a warp row may hold (16 per lane)

// Bulk copy (the TMA engine's non-tensor copy) of `bytes` bytes, a multiple
// of 16, from this block's shared memory to global memory of this GPU, both
// addresses 16-byte aligned; issued by one thread, tracked by bulk groups.
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(__cvta_generic_to_global(gdst)),
                 "r"((unsigned)__cvta_generic_to_shared(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until the committed bulk copies have read their shared-memory source
// (bulk_wait_read) or have completed (bulk_wait_all).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Orders this thread's earlier shared-memory writes before later bulk copies.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ----- symbolic --------------------------------------------------------------
template <typename IT, int NW>
__global__ void __launch_bounds__(NW * 32) k_sym_warp(Operands<float> op, const int *rows, int count, int *token,
                                                      int tbits, HashCfg hc, int *nnz_out, int *err) {
    using G = Group<32, NW * 32>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][NW];
    const int T = 1 << tbits;
    const size_t per = (size_t)T * 4 + sizeof(EntryScratch<float>);
    unsigned char *wb = smem + (size_t)G::gid() * per;
    int *keys = (int *)wb;
    EntryScratch<float> &es = *(EntryScratch<float> *)(wb + (size_t)T * 4);
    const int lane = lane_id();
    for (int s = lane; s < T; s += 32) keys[s] = kEmpty;
    __syncwarp();
    RowClaimPf<G> claim(token, rows, s_row, nullptr);
    for (;;) {
        int i;
        const int r = claim.next(count, &i);
        if (r >= count) break;
        int64_t ab, ae;
        a_row_range(op, i, ab, ae, err);
        int cnt = 0, full = 0;
        warp_enum<float, IT, false>(op, ab, ae, es, err, [&](bool act, int j, float, float, int) {
            bool ins = false;
            if (act && cas_insert(keys, tbits, hc, j, ins) < 0) full = 1;
            cnt += __popc(__ballot_sync(kFull, ins));
        });
        claim.prefetch(count);
        if (__any_sync(kFull, full) && lane == 0) raise_err(err, kErrTableFull);
        if (lane == 0) nnz_out[i] = cnt;
        __syncwarp();
        // back to EMPTY for the next row (16-byte stores)
        int4 *k4 = (int4 *)keys;
        for (int s = lane; s < (T >> 2); s += 32) k4[s] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
        __syncwarp();
    }
}

// ----- numeric ---------------------------------------------------------------
// Shared memory of one warp: keys[T], vals[T], list[L] (slots claimed by the
// row), bc[NB] (bucket counts), then the enumerator's scratch. The write-out
// groups the row's entries by bucket in keys[0..n), vals[0..n).
template <typename V>
__host__ __device__ constexpr size_t warp_row_bytes(int T, int L, int NB) {
    return (size_t)T * (4 + sizeof(V)) + (size_t)L * 4 + (size_t)NB * 4 + sizeof(EntryScratch<V>);
}

// K: entries held per lane in the write-out (the list room L <= 32 K).
// rec (may be null): the rows' product counts (kept by the symbolic phase, or
// gathered by the learned planning). In exact mode a row whose length equals
// its product count has no repeated column: nothing to merge, so its products
// skip the table and go straight to the write-out's staging (keys[p], vals[p]
// for product p). In capacity mode a row whose products fit its capacity is
// staged the same way and its equal columns are summed after the sort
// (expand, sort, merge): cheaper than hashing when few columns repeat, which
// is what such a capacity says.
// MODE: 0 exact mode, 1 capacity mode, 2 either, with the bulk copy-out and
// the Version 1 write-back available (the first two leave out the code the
// mode cannot reach: a smaller kernel, fewer instruction-cache misses).
template <typename V, typename IT, int K, int NW, int MODE>
__global__ void __launch_bounds__(NW * 32) k_num_warp(Operands<V> op, const int *rows, int count, int *token,
                                                      int tbits, HashCfg hc, int lcap, int nb, int bsh,
                                                      const RowGather *rec, int bulk, NumOutT<V> out, int *err) {
    using G = Group<32, NW * 32>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][NW];
    const int T = 1 << tbits;
    const int NB = nb;
    unsigned char *wb = smem + (size_t)G::gid() * warp_row_bytes<V>(T, lcap, NB);
    int *keys = (int *)wb;
    V *vals = (V *)(wb + (size_t)T * 4);
    int *list = (int *)(wb + (size_t)T * (4 + sizeof(V)));
    int *bc = list + lcap;
    EntryScratch<V> &es = *(EntryScratch<V> *)(bc + NB);
    const int lane = lane_id();
    for (int s = lane; s < T; s += 32) {
        keys[s] = kEmpty;
        vals[s] = V(0);
    }
    for (int s = lane; s < NB; s += 32) bc[s] = 0;
    __syncwarp();
    RowClaimPf<G> claim(token, rows, s_row, nullptr);
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
        if (!ok || !a_bounds_ok(ab, ae, op.a_nnz, err)) ab = ae = 0;
        int cnt = 0, full = 0;
        // direct: exact mode, the row's length equals its product count (no
        // repeated column). merge: capacity mode, the row's products fit its
        // capacity (the size model sees few repeated columns); its products
        // are staged as they are and equal columns summed after the sort.
        const long long f_i = ok ? f_rec : -1;
        const bool cap = MODE == 1 || (MODE == 2 && out.row_nnz != nullptr);
        const bool direct = !cap && f_i >= 0 && n_exp <= lcap && f_i == (long long)n_exp;
        const bool merge = cap && f_i >= 0 && f_i <= (long long)n_exp && f_i <= lcap && 2 * f_i <= T;
        if (direct || merge) {
            warp_enum<V, IT, true>(op, ab, ae, es, err, [&](bool act, int j, V a, V b, int p) {
                if (act && p < lcap) {
                    keys[p] = j;
                    vals[p] = a * b;
                }
                cnt += __popc(__ballot_sync(kFull, act));
            });
        } else {
            warp_enum<V, IT, true>(op, ab, ae, es, err, [&](bool act, int j, V a, V b, int) {
                bool ins = false;
                int h = -1;
                if (act) {
                    h = cas_insert(keys, tbits, hc, j, ins);
                    if (h >= 0) atomicAdd(vals + h, a * b);
                    else full = 1;
                }
                const unsigned m = __ballot_sync(kFull, ins);
                if (ins) {
                    const int pos = cnt + __popc(m & lanemask_lt());
                    if (pos < lcap) list[pos] = h;
                }
                cnt += __popc(m);
            });
        }
        claim.prefetch(count);
        full = __any_sync(kFull, full);
        const int tot = cnt;
        bool over;
        if (cap) {
            over = full || tot > n_exp || tot > lcap;
            // (a merged row's length is known after the merge)
            if (lane == 0 && (over || !merge)) out.row_nnz[i] = over ? -1 : tot;
        } else {
            over = full || tot != n_exp || tot > lcap;
            if (lane == 0) {
                if (full || tot > lcap) raise_err(err, kErrTableFull);
                else if (tot != n_exp) raise_err(err, kErrCountMismatch);
            }
        }
        __syncwarp();
        if (over) {
            // nothing is written; the table goes back to EMPTY / 0
            if (full || tot > lcap || direct || merge) {
                for (int s = lane; s < T; s += 32) {
                    keys[s] = kEmpty;
                    vals[s] = V(0);
                }
            } else {
                for (int q = lane; q < tot; q += 32) {
                    const int h = list[q];
                    keys[h] = kEmpty;
                    vals[h] = V(0);
                }
            }
        } else if (merge) {
            // expanded products, sorted by column, equal columns summed
            // 1. the products into registers, their staging back to EMPTY / 0,
            //    counts per bucket
            int kk[K], pp[K];
            V vv[K];
#pragma unroll
            for (int x = 0; x < K; ++x) {
                const int q = lane + 32 * x;
                kk[x] = INT_MAX;
                vv[x] = V(0);
                pp[x] = -1;
                if (q < tot) {
                    kk[x] = keys[q];
                    vv[x] = vals[q];
                    keys[q] = kEmpty;
                    vals[q] = V(0);
                    atomicAdd(bc + (kk[x] >> bsh), 1);
                }
            }
            __syncwarp();
            {
                const int run = (NB + 31) >> 5;
                const int b0 = min(lane * run, NB), b1 = min(b0 + run, NB);
                int loc = 0;
                for (int b = b0; b < b1; ++b) loc += bc[b];
                int acc = warp_incl_scan(loc) - loc;
                for (int b = b0; b < b1; ++b) {
                    const int c = bc[b];
                    bc[b] = acc;
                    acc += c;
                }
            }
            __syncwarp();
            // 2. grouped by bucket into keys[0..tot)
#pragma unroll
            for (int x = 0; x < K; ++x) {
                if (lane + 32 * x < tot) {
                    pp[x] = atomicAdd(bc + (kk[x] >> bsh), 1);
                    keys[pp[x]] = kk[x];
                }
            }
            __syncwarp();
            // 3. place of each product in the sorted sequence: its bucket's
            //    start plus the smaller columns of the bucket, equal columns
            //    ordered by their grouped position
#pragma unroll
            for (int x = 0; x < K; ++x) {
                if (lane + 32 * x < tot) {
                    const int b = kk[x] >> bsh;
                    const int e = bc[b];
                    const int s0 = b ? bc[b - 1] : 0;
                    int rk = 0;
                    for (int y = s0; y < e; ++y) {
                        const int ky = keys[y];
                        rk += (ky < kk[x] || (ky == kk[x] && y < pp[x])) ? 1 : 0;
                    }
                    pp[x] = s0 + rk;
                }
            }
            __syncwarp();
            // 4. the sorted sequence in keys[tot..2 tot), vals[tot..2 tot)
#pragma unroll
            for (int x = 0; x < K; ++x) {
                if (lane + 32 * x < tot) {
                    keys[tot + pp[x]] = kk[x];
                    vals[tot + pp[x]] = vv[x];
                }
            }
            __syncwarp();
            // 5. the first of each run of equal columns sums the run and takes
            //    the next place of the row
            int run_tot = 0;
#pragma unroll
            for (int x = 0; x < K; ++x) {
                const int q = lane + 32 * x;
                bool first = false;
                int sk = 0;
                if (q < tot) {
                    sk = keys[tot + q];
                    first = q == 0 || keys[tot + q - 1] != sk;
                }
                const unsigned m = __ballot_sync(kFull, first);
                if (first) {
                    V v = vals[tot + q];
                    for (int y = q + 1; y < tot && keys[tot + y] == sk; ++y) v += vals[tot + y];
                    const int d = run_tot + __popc(m & lanemask_lt());
                    __stcs(out.c_ci + (c0 + d), sk);
                    __stcs(out.c_val + (c0 + d), v);
                }
                run_tot += __popc(m);
            }
            if (lane == 0) out.row_nnz[i] = run_tot;
            __syncwarp();
            for (int q = lane; q < 2 * tot; q += 32) {
                keys[q] = kEmpty;
                vals[q] = V(0);
            }
        } else if (MODE == 2 && hc.kind == 2 && !direct) {
            // Version 1's write-back: the order-preserving hash (the high bits
            // of the column) leaves the table almost sorted in slot order, so
            // the occupied slots are compacted in order (in place: a chunk is
            // read before anything lands on it), the local disorder that
            // collisions left is sorted out by odd-even transposition passes
            // until one pass of each parity swaps nothing, and the row streams
            // to C; then the whole table goes back to EMPTY / 0.
            int filled = 0;
            for (int s0 = 0; s0 < T; s0 += 32) {
                const int k = keys[s0 + lane];
                const V v = vals[s0 + lane];
                const bool occ = k != kEmpty;
                const unsigned m = __ballot_sync(kFull, occ);
                __syncwarp();
                if (occ) {
                    const int d = filled + __popc(m & lanemask_lt());
                    keys[d] = k;
                    vals[d] = v;
                }
                filled += __popc(m);
                __syncwarp();
            }
            for (int pass = 0, quiet = 0; quiet < 2 && pass < tot + 2; ++pass) {
                bool swapped = false;
                for (int x = 2 * lane + (pass & 1); x + 1 < tot; x += 64) {
                    const int a = keys[x], b = keys[x + 1];
                    if (a > b) {
                        keys[x] = b;
                        keys[x + 1] = a;
                        const V va = vals[x];
                        vals[x] = vals[x + 1];
                        vals[x + 1] = va;
                        swapped = true;
                    }
                }
                __syncwarp();
                quiet = __any_sync(kFull, swapped) ? 0 : quiet + 1;
            }
            for (int q = lane; q < tot; q += 32) {
                __stcs(out.c_ci + (c0 + q), keys[q]);
                __stcs(out.c_val + (c0 + q), vals[q]);
            }
            __syncwarp();
            for (int s0 = lane; s0 < T; s0 += 32) {
                keys[s0] = kEmpty;
                vals[s0] = V(0);
            }
        } else if (tot <= 32) {
            // rank of each entry among the row's (at most 32) columns
            int k = INT_MAX;
            V v = V(0);
            if (lane < tot) {
                const int h = direct ? lane : list[lane];
                k = keys[h];
                v = vals[h];
                keys[h] = kEmpty;
                vals[h] = V(0);
            }
            int rank = 0;
            for (int m = 0; m < tot; ++m) rank += __shfl_sync(kFull, k, m) < k ? 1 : 0;
            if (lane < tot) {
                __stcs(out.c_ci + (c0 + rank), k);
                __stcs(out.c_val + (c0 + rank), v);
            }
        } else {
            // 1. the entries into registers, their slots back to EMPTY / 0,
            //    counts per bucket (bucket = column >> bsh, monotone in the column)
            int kk[K];
            V vv[K];
#pragma unroll
            for (int x = 0; x < K; ++x) {
                const int q = lane + 32 * x;
                kk[x] = INT_MAX;
                vv[x] = V(0);
                if (q < tot) {
                    const int h = direct ? q : list[q];
                    kk[x] = keys[h];
                    vv[x] = vals[h];
                    keys[h] = kEmpty;
                    vals[h] = V(0);
                    atomicAdd(bc + (kk[x] >> bsh), 1);
                }
            }
            __syncwarp();
            // 2. bucket starts: each lane sums a run of consecutive buckets
            {
                const int run = (NB + 31) >> 5;
                const int b0 = min(lane * run, NB), b1 = min(b0 + run, NB);
                int loc = 0;
                for (int b = b0; b < b1; ++b) loc += bc[b];
                int acc = warp_incl_scan(loc) - loc;
                for (int b = b0; b < b1; ++b) {
                    const int c = bc[b];
                    bc[b] = acc;
                    acc += c;
                }
            }
            __syncwarp();
            // 3. grouped by bucket into keys[0..tot), vals[0..tot)
#pragma unroll
            for (int x = 0; x < K; ++x) {
                if (lane + 32 * x < tot) {
                    const int p = atomicAdd(bc + (kk[x] >> bsh), 1);
                    keys[p] = kk[x];
                    vals[p] = vv[x];
                }
            }
            __syncwarp();
            // 4. bc[b] is now the end of bucket b: each entry's place is its
            //    bucket's start plus the smaller columns in its bucket.
            // 5. with bulk != 0 (C's arrays 16-byte aligned) the sorted row is
            //    staged in the table's memory, element e at e + (c0 mod 16 bytes),
            //    and streamed to C: the aligned middle by one bulk copy per
            //    array, the ragged ends by the lanes that hold them (Version 3's
            //    bulk copy-out); otherwise every lane stores its entries
            constexpr int UK = 4, UV = 16 / (int)sizeof(V);
            if (MODE == 2 && bulk && tot + UK <= T) {
                int pos[K];
#pragma unroll
                for (int x = 0; x < K; ++x) {
                    pos[x] = -1;
                    if (lane + 32 * x < tot) {
                        const int b = kk[x] >> bsh;
                        const int e = bc[b];
                        const int s0 = b ? bc[b - 1] : 0;
                        int rk = 0;
                        for (int y = s0; y < e; ++y) rk += keys[y] < kk[x] ? 1 : 0;
                        pos[x] = s0 + rk;
                    }
                }
                __syncwarp();
                const int ok_off = (int)(c0 % UK), ov_off = (int)(c0 % UV);
#pragma unroll
                for (int x = 0; x < K; ++x) {
                    if (pos[x] >= 0) {
                        keys[ok_off + pos[x]] = kk[x];
                        vals[ov_off + pos[x]] = vv[x];
                    }
                }
                fence_async_smem();
                __syncwarp();
                const int64_t gk0 = (c0 + UK - 1) / UK * UK, gk1 = (c0 + tot) / UK * UK;
                const int64_t gv0 = (c0 + UV - 1) / UV * UV, gv1 = (c0 + tot) / UV * UV;
                if (lane == 0) {
                    if (gk1 > gk0)
                        bulk_store(out.c_ci + gk0, keys + ok_off + (gk0 - c0), (unsigned)((gk1 - gk0) * 4));
                    if (gv1 > gv0)
                        bulk_store(out.c_val + gv0, vals + ov_off + (gv0 - c0), (unsigned)((gv1 - gv0) * sizeof(V)));
                    bulk_commit();
                }
#pragma unroll
                for (int x = 0; x < K; ++x) {
                    if (pos[x] >= 0) {
                        const int64_t g = c0 + pos[x];
                        if (g < gk0 || g >= gk1) __stcs(out.c_ci + (g), kk[x]);
                        if (g < gv0 || g >= gv1) __stcs(out.c_val + (g), vv[x]);
                    }
                }
                if (lane == 0) bulk_wait_read();
                __syncwarp();
            } else {
#pragma unroll
                for (int x = 0; x < K; ++x) {
                    if (lane + 32 * x < tot) {
                        const int b = kk[x] >> bsh;
                        const int e = bc[b];
                        const int s0 = b ? bc[b - 1] : 0;
                        int rk = 0;
                        for (int y = s0; y < e; ++y) rk += keys[y] < kk[x] ? 1 : 0;
                        __stcs(out.c_ci + (c0 + s0 + rk), kk[x]);
                        __stcs(out.c_val + (c0 + s0 + rk), vv[x]);
                    }
                }
                __syncwarp();
            }
            const int used = min(T, tot + UK);
            for (int q = lane; q < used; q += 32) {
                keys[q] = kEmpty;
                vals[q] = V(0);
            }
        }
        // bucket counts back to zero (the insertion left them untouched when
        // the row took no bucket write-out)
        if (!over && (tot > 32 || merge))
            for (int s = lane; s < NB; s += 32) bc[s] = 0;
        __syncwarp();
    }
    if (MODE == 2 && bulk && lane == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
template <typename V>
static Operands<V> warp_operands(const RawOperands &r) {
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

template <typename K>
static int warp_grid(K kernel, size_t smem, int sms, int count) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarpRowWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const long long want = ((long long)count + kWarpRowWarps - 1) / kWarpRowWarps;
    const long long cap = (long long)per_sm * sms;
    return (int)(want < cap ? want : cap);
}

// List room L: the most columns a row of the bin may hold (T * max_load,
// rounded up to 32, at most T); NB = T / 2 buckets over the column range.
static int warp_lcap(int tbits, float inv_load) {
    const int T = 1 << tbits;
    int L = (int)((double)T / (double)inv_load + 0.999);
    L = (L + 31) & ~31;
    return L < 32 ? 32 : (L > T ? T : L);
}

[[maybe_unused]] static int warp_buckets(int tbits) { return (1 << tbits) >> 1; }

template <typename V, typename IT, int K>
static void num_warp_go(const Operands<V> &op, const int *rows, int count, int *token, const HashLaunch &hl,
                        int L, const RowGather *rec, int bulk_copy, const NumOutT<V> &out, int *err, cudaStream_t s,
                        size_t smem) {
    const int NB = warp_buckets(hl.tbits);
    int nbbits = 0;
    while ((1 << nbbits) < NB) ++nbbits;
    const int bsh = hl.colbits > nbbits ? hl.colbits - nbbits : 0;
    // bulk copies need 16-byte aligned destinations: C's arrays must start
    // on a 16-byte boundary (the row offsets are handled in the kernel)
    const int bulk = (bulk_copy && (uintptr_t)out.c_ci % 16 == 0 && (uintptr_t)out.c_val % 16 == 0) ? 1 : 0;
    const int mode = (bulk || hl.hash_kind == 2) ? 2 : out.row_nnz ? 1 : 0;
    auto kern = mode == 0 ? k_num_warp<V, IT, K, kWarpRowWarps, 0>
              : mode == 1 ? k_num_warp<V, IT, K, kWarpRowWarps, 1> : k_num_warp<V, IT, K, kWarpRowWarps, 2>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    kern<<<warp_grid(kern, smem, hl.sms, count), kWarpRowWarps * 32, smem, s>>>(op, rows, count, token, hl.tbits, hc,
                                                                              L, NB, bsh, rec, bulk, out, err);
}

template <typename V, typename IT>
static void num_warp_k(const Operands<V> &op, const int *rows, int count, int *token, const HashLaunch &hl, int L,
                       const RowGather *rec, int bulk_copy, const NumOutT<V> &out, int *err, cudaStream_t s,
                       size_t smem) {
    const int k = (L + 31) / 32;
    if (k <= 2) num_warp_go<V, IT, 2>(op, rows, count, token, hl, L, rec, bulk_copy, out, err, s, smem);
    else if (k <= 4) num_warp_go<V, IT, 4>(op, rows, count, token, hl, L, rec, bulk_copy, out, err, s, smem);
    else if (k <= 8) num_warp_go<V, IT, 8>(op, rows, count, token, hl, L, rec, bulk_copy, out, err, s, smem);
    else num_warp_go<V, IT, 16>(op, rows, count, token, hl, L, rec, bulk_copy, out, err, s, smem);
}

template <typename V>
static void num_warp_typed(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                           float inv_load, const RowGather *rec, int bulk_copy, const NumOut &o, int *err,
                           cudaStream_t s) {
    const Operands<V> op = warp_operands<V>(r);
    const NumOutT<V> out{o.c_rp, o.c_ci, (V *)o.c_val, o.c_nnz, o.row_nnz};
    const int L = warp_lcap(hl.tbits, inv_load);
    const size_t smem = num_warp_smem(sizeof(V) == 8, hl.tbits, inv_load);
    if (r.b_nnz < INT_MAX) num_warp_k<V, int32_t>(op, rows, count, token, hl, L, rec, bulk_copy, out, err, s, smem);
    else num_warp_k<V, int64_t>(op, rows, count, token, hl, L, rec, bulk_copy, out, err, s, smem);
}

}  // namespace smash
