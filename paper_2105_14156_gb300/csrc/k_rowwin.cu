// Row windows: one shared-memory table for a window of several short rows,
// each entry tagged with (row of the window, column).
//
// The Window Distribution Phase groups rows into windows and one block's
// scratchpad table serves the whole window, its tag made of the output row
// (X coordinate, from A) and the column (Y coordinate, from B). Here a warp
// takes a window of W consecutive rows of a bin (rows whose tables hold at
// most a few dozen columns) and enumerates the products of all of them as one
// line: the window's entries of A are laid end to end (lane r holds where row
// r's entries start and end), each batch of 32 entries finds its rows by a
// search over those ends, and each step hands 32 consecutive products to the
// 32 lanes, whatever row they belong to. A product's tag is
// (r << cb) | j, cb = bits of a column index, so that the tags of a window
// order by row first and by column second.
//
// Numeric phase. A window whose rows have no repeated column (exact mode:
// each row's length equals its product count) or whose products fit their
// capacities (capacity mode) is staged as it is (expand); otherwise its
// products are hashed by tag (compare-and-swap on the tag, atomic add on the
// value, the claimed slots listed). The write-out sorts the window's entries
// by tag (a counting sort over the high bits of the tag, then a rank inside
// each bucket), sums runs of equal tags (merge), counts each row's entries,
// and streams every row whose count is right (exact mode) or fits its
// capacity (capacity mode; the others get -1 and are redone by the exact
// path) to its place in C. The symbolic phase hashes the tags and counts the
// claims of each row.
//
// Every index read from the inputs is checked (error word, never a fault).
#include <climits>

#include "device_common.cuh"
#include "kernels.h"
#include "warp_enum.cuh"
#include "writeout.cuh"

namespace smash {

constexpr int kRowWinWarps = 4;   // warps (windows in flight) per block

// Per-warp bookkeeping of a window (row r of the window in entry r).
struct WinMeta {
    long long wend[32];    // end of row r's entries on the window's line of A entries
    long long wab[32];     // position in A of the line's entry 0 as seen from row r
    long long rbase[32];   // C position of row r's first entry minus its first run's index
    int rstart[32];        // index of row r's first run among the window's runs
    int rc[32];            // entries (runs, claims) of row r
    int rok[32];           // row r is written out
    int rsc[32];           // rows of the compacted batch entries
};

// Shared memory of one warp. Symbolic: the enumerator's scratch, the
// bookkeeping, keys[2^tbits]. Numeric: the same, then vals[ts], keys[ts],
// list[lcap] (slots claimed by the window), bc[nb] (bucket counts).
__host__ __device__ inline size_t rowwin_sym_bytes(const RowWin &rw) {
    return sizeof(EntryScratch<float>) + sizeof(WinMeta) + ((size_t)4 << rw.tbits);
}

__host__ __device__ inline size_t rowwin_num_bytes(const RowWin &rw, int vsz) {
    const size_t es = vsz == 8 ? sizeof(EntryScratch<double>) : sizeof(EntryScratch<float>);
    return es + sizeof(WinMeta) + (size_t)rw.ts * (4 + vsz) + (size_t)rw.lcap * 4 + (size_t)rw.nb * 4;
}

// Every product of the window's rows, enumerated by one warp (the row-window
// counterpart of warp_enum): f(act, j, a, b, p, r) is called by all 32 lanes
// together once per step of 32 products (p: the product's index on the
// window's line, r: its row in the window).
template <typename V, typename IT, bool NUM, typename F>
__device__ __forceinline__ void window_enum(const Operands<V> &op, int nrows, long long total_a, WinMeta &mt,
                                            EntryScratch<V> &es, int *err, F &&f) {
    const int lane = lane_id();
    int pbase = 0;
    for (long long base = 0; base < total_a; base += 32) {
        const long long x = base + lane;
        int len = 0, r = 0;
        int64_t bs = 0;
        V av = V(0);
        if (x < total_a) {
            // row of entry x: the first whose end lies past x (rows without
            // entries share their end with the row before and are skipped)
            int lo = 0, hi = nrows - 1;
            while (lo < hi) {
                const int m = (lo + hi) >> 1;
                if (mt.wend[m] <= x) lo = m + 1;
                else hi = m;
            }
            r = lo;
            const int64_t apos = mt.wab[r] + x;
            b_row_whole(op, __ldg(op.a_ci + apos), len, bs, err);
            if constexpr (NUM) av = op.a_val[apos];
        }
        // entries with an empty row of B move out of the way (as in warp_enum)
        const unsigned nz = __ballot_sync(kFull, len > 0);
        const int nv = __popc(nz);
        if (nv < 32 && nz != (1u << nv) - 1u) {
            if (len > 0) {
                const int d = __popc(nz & lanemask_lt());
                es.start[d] = bs;
                es.len[d] = len;
                mt.rsc[d] = r;
                if constexpr (NUM) es.av[d] = av;
            }
            __syncwarp();
            len = lane < nv ? es.len[lane] : 0;
            bs = lane < nv ? es.start[lane] : 0;
            r = lane < nv ? mt.rsc[lane] : 0;
            if constexpr (NUM) av = lane < nv ? es.av[lane] : V(0);
            __syncwarp();
        }
        const int incl = warp_incl_scan(len);
        const int total = __shfl_sync(kFull, incl, 31);
        const IT start = (IT)(bs - (incl - len));
        for (int q0 = 0; q0 < total; q0 += 32 * kWarpUnroll) {
            int jv[kWarpUnroll], ru[kWarpUnroll];
            V a_u[kWarpUnroll], b_u[kWarpUnroll];
            bool act[kWarpUnroll];
#pragma unroll
            for (int u = 0; u < kWarpUnroll; ++u) {
                const int q = q0 + 32 * u;
                act[u] = q + lane < total;
                jv[u] = 0;
                ru[u] = 0;
                a_u[u] = V(0);
                b_u[u] = V(0);
                if (q < total) {
                    const int c0 = __popc(__ballot_sync(kFull, incl <= q));
                    const int e = incl - q;
                    const unsigned ends = __reduce_or_sync(kFull, (e >= 1 && e <= 31) ? (1u << e) : 0u);
                    const int ci = c0 + __popc(ends & ((2u << lane) - 1u));
                    const IT st = __shfl_sync(kFull, start, ci);
                    ru[u] = __shfl_sync(kFull, r, ci);
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
                    f(ok, jv[u], a_u[u], b_u[u], pbase + q0 + 32 * u + lane, ru[u]);
                }
            }
        }
        pbase += total;
    }
}

// The window's rows, one per lane (lanes past the window hold nothing), and
// its line of A entries laid out in mt.wend / mt.wab.
struct WinRow {
    int i = -1;           // row of A / C
    int64_t ab = 0, ae = 0;
    __device__ __forceinline__ long long na() const { return ae - ab; }
};

__device__ __forceinline__ long long window_line(WinMeta &mt, const WinRow &wr, int nrows) {
    const int lane = lane_id();
    const long long n = lane < nrows ? wr.na() : 0;
    const long long incl = warp_incl_scan64(n);
    if (lane < nrows) {
        mt.wend[lane] = incl;
        mt.wab[lane] = wr.ab - (incl - n);
    }
    __syncwarp();
    return __shfl_sync(kFull, incl, 31);
}

// ----- symbolic --------------------------------------------------------------
template <typename IT, int NW>
__global__ void __launch_bounds__(NW * 32) k_sym_rowwin(Operands<float> op, const int *rows, int count, int *token,
                                                        RowWin rw, HashCfg hc, int *nnz_out, int *err) {
    using G = Group<32, NW * 32>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][NW];
    const int T = 1 << rw.tbits;
    unsigned char *wb = smem + (size_t)G::gid() * rowwin_sym_bytes(rw);
    EntryScratch<float> &es = *(EntryScratch<float> *)wb;
    WinMeta &mt = *(WinMeta *)(wb + sizeof(EntryScratch<float>));
    int *keys = (int *)(wb + sizeof(EntryScratch<float>) + sizeof(WinMeta));
    const int lane = lane_id();
    for (int s = lane; s < T; s += 32) keys[s] = kEmpty;
    mt.rc[lane] = 0;
    __syncwarp();
    const int nwin = (int)(((long long)count + rw.W - 1) / rw.W);
    RowClaim<G> claim(token, s_row);
    for (;;) {
        const int w = claim.next(nwin);
        if (w >= nwin) break;
        const int r0 = w * rw.W;
        const int nrows = min(rw.W, count - r0);
        WinRow wr;
        if (lane < nrows) {
            wr.i = rows[r0 + lane];
            a_row_range(op, wr.i, wr.ab, wr.ae, err);
        }
        const long long total_a = window_line(mt, wr, nrows);
        int full = 0;
        window_enum<float, IT, false>(op, nrows, total_a, mt, es, err, [&](bool act, int j, float, float, int, int r) {
            bool ins = false;
            if (act) {
                if (cas_insert(keys, rw.tbits, hc, (r << rw.cb) | j, ins) < 0) full = 1;
                if (ins) atomicAdd(mt.rc + r, 1);
            }
        });
        if (__any_sync(kFull, full) && lane == 0) raise_err(err, kErrTableFull);
        __syncwarp();
        if (lane < nrows) nnz_out[wr.i] = mt.rc[lane];
        mt.rc[lane] = 0;
        // back to EMPTY for the next window (16-byte stores)
        int4 *k4 = (int4 *)keys;
        for (int s = lane; s < (T >> 2); s += 32) k4[s] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
        __syncwarp();
    }
}

// ----- numeric ---------------------------------------------------------------
// K: entries held per lane in the write-out (rw.lcap <= 32 K).
template <typename V, typename IT, int K, int NW>
__global__ void __launch_bounds__(NW * 32) k_num_rowwin(Operands<V> op, const int *rows, int count, int *token,
                                                        RowWin rw, HashCfg hc, const RowGather *rec, NumOutT<V> out,
                                                        int *err) {
    using G = Group<32, NW * 32>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][NW];
    unsigned char *wb = smem + (size_t)G::gid() * rowwin_num_bytes(rw, (int)sizeof(V));
    EntryScratch<V> &es = *(EntryScratch<V> *)wb;
    WinMeta &mt = *(WinMeta *)(wb + sizeof(EntryScratch<V>));
    V *vals = (V *)(wb + sizeof(EntryScratch<V>) + sizeof(WinMeta));
    int *keys = (int *)(vals + rw.ts);
    int *list = keys + rw.ts;
    int *bc = list + rw.lcap;
    const int lane = lane_id();
    const int cmask = (1 << rw.cb) - 1;
    for (int s = lane; s < rw.ts; s += 32) {
        keys[s] = kEmpty;
        vals[s] = V(0);
    }
    for (int s = lane; s < rw.nb; s += 32) bc[s] = 0;
    mt.rc[lane] = 0;
    __syncwarp();
    const int nwin = (int)(((long long)count + rw.W - 1) / rw.W);
    RowClaim<G> claim(token, s_row);
    for (;;) {
        const int w = claim.next(nwin);
        if (w >= nwin) break;
        const int r0 = w * rw.W;
        const int nrows = min(rw.W, count - r0);
        WinRow wr;
        int64_t c0 = 0;
        int n_exp = 0;
        bool ok = false;
        long long f = -1;
        if (lane < nrows) {
            // the row's bounds in C and A and its product count, loaded together
            wr.i = rows[r0 + lane];
            const int64_t cs = out.c_rp[wr.i], ct = out.c_rp[wr.i + 1];
            int64_t ab = __ldg(op.a_rp + wr.i), ae = __ldg(op.a_rp + wr.i + 1);
            const long long f_rec = rec ? rec[wr.i].f : -1;
            ok = row_bounds_ok(cs, ct, out.c_nnz, c0, n_exp, err);
            if (ok && a_bounds_ok(ab, ae, op.a_nnz, err)) {
                wr.ab = ab;
                wr.ae = ae;
            }
            f = ok ? f_rec : -1;
        }
        // staged (expand) when every row's products can go as they are: no
        // repeated column in exact mode, within the capacity in capacity mode
        const bool fits = lane >= nrows || (f >= 0 && (out.row_nnz ? f <= (long long)n_exp : f == (long long)n_exp));
        const long long fw = warp_sum<long long>(lane < nrows && f > 0 ? f : 0);
        const bool stage = __all_sync(kFull, fits) && fw <= (long long)rw.lcap;
        const long long total_a = window_line(mt, wr, nrows);
        int cnt = 0, full = 0;
        if (stage) {
            window_enum<V, IT, true>(op, nrows, total_a, mt, es, err, [&](bool act, int j, V a, V b, int p, int r) {
                if (act && (unsigned)p < (unsigned)rw.lcap) {
                    keys[p] = (r << rw.cb) | j;
                    vals[p] = a * b;
                }
            });
            // (a product with a bad column leaves its slot EMPTY; the call fails)
            cnt = (int)fw;
        } else {
            window_enum<V, IT, true>(op, nrows, total_a, mt, es, err, [&](bool act, int j, V a, V b, int, int r) {
                bool ins = false;
                int h = -1;
                if (act) {
                    h = cas_insert(keys, rw.tbits, hc, (r << rw.cb) | j, ins);
                    if (h >= 0) atomicAdd(vals + h, a * b);
                    else full = 1;
                }
                const unsigned m = __ballot_sync(kFull, ins);
                if (ins) {
                    const int pos = cnt + __popc(m & lanemask_lt());
                    if (pos < rw.lcap) list[pos] = h;
                }
                cnt += __popc(m);
            });
        }
        full = __any_sync(kFull, full);
        const int tot = cnt;
        if (full || tot > rw.lcap) {
            // the window's table ran out: in capacity mode its rows are redone
            // by the exact path, in exact mode the call fails
            if (out.row_nnz) {
                if (lane < nrows && ok) out.row_nnz[wr.i] = -1;
            } else if (lane == 0) {
                raise_err(err, kErrTableFull);
            }
            __syncwarp();
            for (int s = lane; s < rw.ts; s += 32) {
                keys[s] = kEmpty;
                vals[s] = V(0);
            }
            __syncwarp();
            continue;
        }
        __syncwarp();
        // 1. the entries into registers, their slots back to EMPTY / 0, counts
        //    per bucket (bucket = tag >> bsh, monotone in the tag)
        int kk[K], pp[K];
        V vv[K];
#pragma unroll
        for (int x = 0; x < K; ++x) {
            const int q = lane + 32 * x;
            kk[x] = INT_MAX;
            vv[x] = V(0);
            pp[x] = -1;
            if (q < tot) {
                const int h = stage ? q : list[q];
                const int k = keys[h];
                kk[x] = k < 0 ? 0 : k;
                vv[x] = vals[h];
                keys[h] = kEmpty;
                vals[h] = V(0);
                atomicAdd(bc + (kk[x] >> rw.bsh), 1);
            }
        }
        __syncwarp();
        // 2. bucket starts: each lane sums a run of consecutive buckets
        {
            const int run = (rw.nb + 31) >> 5;
            const int b0 = min(lane * run, rw.nb), b1 = min(b0 + run, rw.nb);
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
        // 3. grouped by bucket into keys[0..tot)
#pragma unroll
        for (int x = 0; x < K; ++x) {
            if (lane + 32 * x < tot) {
                pp[x] = atomicAdd(bc + (kk[x] >> rw.bsh), 1);
                keys[pp[x]] = kk[x];
            }
        }
        __syncwarp();
        // 4. place in the sorted sequence: the bucket's start plus the smaller
        //    tags of the bucket, equal tags ordered by their grouped position;
        //    the sequence goes to keys[tot..2 tot), vals[tot..2 tot)
#pragma unroll
        for (int x = 0; x < K; ++x) {
            if (lane + 32 * x < tot) {
                const int b = kk[x] >> rw.bsh;
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
#pragma unroll
        for (int x = 0; x < K; ++x) {
            if (lane + 32 * x < tot) {
                keys[tot + pp[x]] = kk[x];
                vals[tot + pp[x]] = vv[x];
            }
        }
        __syncwarp();
        // 5. runs of equal tags: each is one entry of C; the window's runs
        //    are numbered in order, each row counts its runs and notes the
        //    number of its first
        const int *sk = keys + tot;
        int run_tot = 0;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            const int q = lane + 32 * x;
            bool first = false;
            int k = 0, prev = -1;
            if (q < tot) {
                k = sk[q];
                prev = q ? sk[q - 1] : -1;
                first = q == 0 || prev != k;
            }
            const unsigned m = __ballot_sync(kFull, first);
            pp[x] = -1;
            if (first) {
                const int d = run_tot + __popc(m & lanemask_lt());
                const int r = k >> rw.cb;
                atomicAdd(mt.rc + r, 1);
                if (q == 0 || (prev >> rw.cb) != r) mt.rstart[r] = d;
                pp[x] = d;
            }
            run_tot += __popc(m);
        }
        __syncwarp();
        // 6. each row's verdict: exact mode wants its expected length,
        //    capacity mode its capacity (else -1: redone by the exact path)
        if (lane < nrows && ok) {
            const int n = mt.rc[lane];
            bool wr_ok;
            if (out.row_nnz) {
                wr_ok = n <= n_exp;
                out.row_nnz[wr.i] = wr_ok ? n : -1;
            } else {
                wr_ok = n == n_exp;
                if (!wr_ok) raise_err(err, kErrCountMismatch);
            }
            mt.rok[lane] = wr_ok ? 1 : 0;
            mt.rbase[lane] = c0 - mt.rstart[lane];
        } else {
            mt.rok[lane] = 0;
        }
        __syncwarp();
        // 7. the first of each run sums the run and stores it at its row's place
#pragma unroll
        for (int x = 0; x < K; ++x) {
            if (pp[x] >= 0) {
                const int q = lane + 32 * x;
                const int k = sk[q];
                V v = vals[tot + q];
                for (int y = q + 1; y < tot && sk[y] == k; ++y) v += vals[tot + y];
                const int r = k >> rw.cb;
                if (mt.rok[r]) {
                    const int64_t g = mt.rbase[r] + pp[x];
                    __stcs(out.c_ci + (g), k & cmask);
                    __stcs(out.c_val + (g), v);
                }
            }
        }
        __syncwarp();
        for (int q = lane; q < 2 * tot; q += 32) {
            keys[q] = kEmpty;
            vals[q] = V(0);
        }
        for (int s = lane; s < rw.nb; s += 32) bc[s] = 0;
        mt.rc[lane] = 0;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
template <typename V>
static Operands<V> rowwin_operands(const RawOperands &r) {
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

template <typename Kern>
static int rowwin_grid(Kern kernel, size_t smem, int sms, long long windows) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRowWinWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const long long want = (windows + kRowWinWarps - 1) / kRowWinWarps;
    const long long cap = (long long)per_sm * sms;
    return (int)(want < cap ? want : cap);
}

size_t sym_rowwin_smem(const RowWin &rw) { return (size_t)kRowWinWarps * rowwin_sym_bytes(rw); }

size_t num_rowwin_smem(const RowWin &rw, int dtype) {
    return (size_t)kRowWinWarps * rowwin_num_bytes(rw, dtype ? 8 : 4);
}

void launch_sym_rowwin(const RawOperands &r, const int *rows, int count, int *token, const RowWin &rw,
                       const HashLaunch &hl, int *nnz_out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    const Operands<float> op = rowwin_operands<float>(r);
    const size_t smem = sym_rowwin_smem(rw);
    const HashCfg hc{hl.hash_kind, rw.cb + rw.wbits};
    const long long windows = ((long long)count + rw.W - 1) / rw.W;
    if (r.b_nnz < INT_MAX) {
        auto kern = k_sym_rowwin<int32_t, kRowWinWarps>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<rowwin_grid(kern, smem, hl.sms, windows), kRowWinWarps * 32, smem, s>>>(op, rows, count, token, rw,
                                                                                      hc, nnz_out, err);
    } else {
        auto kern = k_sym_rowwin<int64_t, kRowWinWarps>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<rowwin_grid(kern, smem, hl.sms, windows), kRowWinWarps * 32, smem, s>>>(op, rows, count, token, rw,
                                                                                      hc, nnz_out, err);
    }
}

template <typename V, typename IT, int K>
static void num_rowwin_go(const Operands<V> &op, const int *rows, int count, int *token, const RowWin &rw,
                          const HashCfg &hc, const RowGather *rec, const NumOutT<V> &out, int *err, int sms,
                          cudaStream_t s) {
    const size_t smem = num_rowwin_smem(rw, sizeof(V) == 8);
    const long long windows = ((long long)count + rw.W - 1) / rw.W;
    auto kern = k_num_rowwin<V, IT, K, kRowWinWarps>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<rowwin_grid(kern, smem, sms, windows), kRowWinWarps * 32, smem, s>>>(op, rows, count, token, rw, hc, rec,
                                                                               out, err);
}

template <typename V, typename IT>
static void num_rowwin_k(const Operands<V> &op, const int *rows, int count, int *token, const RowWin &rw,
                         const HashCfg &hc, const RowGather *rec, const NumOutT<V> &out, int *err, int sms,
                         cudaStream_t s) {
    const int k = (rw.lcap + 31) / 32;
    if (k <= 2) num_rowwin_go<V, IT, 2>(op, rows, count, token, rw, hc, rec, out, err, sms, s);
    else if (k <= 4) num_rowwin_go<V, IT, 4>(op, rows, count, token, rw, hc, rec, out, err, sms, s);
    else num_rowwin_go<V, IT, 8>(op, rows, count, token, rw, hc, rec, out, err, sms, s);
}

template <typename V>
static void num_rowwin_typed(const RawOperands &r, const int *rows, int count, int *token, const RowWin &rw,
                             const HashLaunch &hl, const RowGather *rec, const NumOut &o, int *err, cudaStream_t s) {
    const Operands<V> op = rowwin_operands<V>(r);
    const NumOutT<V> out{o.c_rp, o.c_ci, (V *)o.c_val, o.c_nnz, o.row_nnz};
    const HashCfg hc{hl.hash_kind, rw.cb + rw.wbits};
    if (r.b_nnz < INT_MAX) num_rowwin_k<V, int32_t>(op, rows, count, token, rw, hc, rec, out, err, hl.sms, s);
    else num_rowwin_k<V, int64_t>(op, rows, count, token, rw, hc, rec, out, err, hl.sms, s);
}

void launch_num_rowwin(int dtype, const RawOperands &r, const int *rows, int count, int *token, const RowWin &rw,
                       const HashLaunch &hl, const RowGather *rec, const NumOut &out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    if (dtype) num_rowwin_typed<double>(r, rows, count, token, rw, hl, rec, out, err, s);
    else num_rowwin_typed<float>(r, rows, count, token, rw, hl, rec, out, err, s);
}

}  // namespace smash
