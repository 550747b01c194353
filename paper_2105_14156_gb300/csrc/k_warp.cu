// Warp rows: one warp per row of C, for the bins whose tables hold up to a
// few hundred columns (the bulk of the rows of R-MAT products).
//
// Hashing Phase, with the row's partial products enumerated from registers:
// lane l of each batch of 32 entries of A_i holds entry l (where the row of B
// it selects starts, its length and a_ik), entries whose row of B is empty
// moved out of the way; a scan of the lengths lays the batch's products on
// one line, and each step hands 32 consecutive products to the 32 lanes. The
// entry of product q + l is the number of entries that end at or before it:
// those ending before the step (one ballot) plus those ending inside it (one
// OR-reduction of one bit per end, then a popcount below the lane). Loads of
// B are coalesced: consecutive lanes read consecutive entries of a row of B.
//
// Insertion tries the compare-and-swap EMPTY -> j first; a slot that holds
// another tag sends the lane one slot on (linear probing with wrap-around,
// the Hashing Phase's collision resolution). The numeric kernel adds a_ik*b_kj
// to the slot's value (atomic add) and appends every newly claimed slot to a
// list, so that the Write-back Phase visits the row's entries only, never the
// whole table: a counting sort of the entries by the high bits of the column
// (bucket counts kept at insertion), then each entry's rank inside its bucket,
// and the row streamed to C in column order. The table is returned to EMPTY
// through the same list.
#include <climits>

#include "device_common.cuh"
#include "kernels.h"
#include "writeout.cuh"

namespace smash {

constexpr int kWarpRowWarps = 4;   // warps (rows in flight) per block
constexpr int kWarpUnroll = 4;     // steps of 32 products whose loads are issued together

// Per-warp scratch of the register enumerator: one batch of entries.
template <typename V>
struct EntryScratch {
    int64_t start[32];
    V av[32];
    int len[32];
};

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
// f(act, j, a, b) is called by all 32 lanes together once per step of 32
// products (act: the lane holds a product), so that it may use warp votes.
template <typename V, bool NUM, typename F>
__device__ __forceinline__ void warp_enum(const Operands<V> &op, int64_t ab, int64_t ae, EntryScratch<V> &es,
                                          int *err, F &&f) {
    const int lane = lane_id();
    for (int64_t base = ab; base < ae; base += 32) {
        int len = 0;
        int64_t bs = 0;
        V av = V(0);
        if (base + lane < ae) load_a_entry<V, NUM>(op, base + lane, len, bs, av, err);
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
        const int64_t start = bs - (incl - len);   // product p of this entry reads B at start + p
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
                    const int64_t st = __shfl_sync(kFull, start, ci);
                    if constexpr (NUM) a_u[u] = __shfl_sync(kFull, av, ci);
                    if (act[u]) {
                        const int64_t idx = st + q + lane;
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
                    f(ok, jv[u], a_u[u], b_u[u]);
                }
            }
        }
    }
}

// ----- symbolic --------------------------------------------------------------
template <int NW>
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
    RowClaim<G> claim(token, s_row);
    for (;;) {
        const int r = claim.next(count);
        if (r >= count) break;
        const int i = rows[r];
        int64_t ab, ae;
        a_row_range(op, i, ab, ae, err);
        int cnt = 0, full = 0;
        warp_enum<float, false>(op, ab, ae, es, err, [&](bool act, int j, float, float) {
            bool ins = false;
            if (act && cas_insert(keys, tbits, hc, j, ins) < 0) full = 1;
            cnt += __popc(__ballot_sync(kFull, ins));
        });
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
// row), bc[NB] (bucket counts), gk[L], gv[L] (entries grouped by bucket),
// then the enumerator's scratch.
template <typename V>
__host__ __device__ constexpr size_t warp_row_bytes(int T, int L, int NB) {
    return (size_t)T * (4 + sizeof(V)) + (size_t)L * (8 + sizeof(V)) + (size_t)NB * 4 + sizeof(EntryScratch<V>);
}

template <typename V, int NW>
__global__ void __launch_bounds__(NW * 32) k_num_warp(Operands<V> op, const int *rows, int count, int *token,
                                                      int tbits, HashCfg hc, int lcap, int nbb, int bsh,
                                                      NumOutT<V> out, int *err) {
    using G = Group<32, NW * 32>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][NW];
    const int T = 1 << tbits;
    const int NB = T >> nbb;
    unsigned char *wb = smem + (size_t)G::gid() * warp_row_bytes<V>(T, lcap, NB);
    int *keys = (int *)wb;
    V *vals = (V *)(wb + (size_t)T * 4);
    int *list = (int *)(wb + (size_t)T * (4 + sizeof(V)));
    int *bc = list + lcap;
    int *gk = bc + NB;
    V *gv = (V *)(gk + lcap);
    EntryScratch<V> &es = *(EntryScratch<V> *)(gv + lcap);
    const int lane = lane_id();
    for (int s = lane; s < T; s += 32) {
        keys[s] = kEmpty;
        vals[s] = V(0);
    }
    for (int s = lane; s < NB; s += 32) bc[s] = 0;
    __syncwarp();
    RowClaim<G> claim(token, s_row);
    for (;;) {
        const int r = claim.next(count);
        if (r >= count) break;
        const int i = rows[r];
        int64_t c0;
        int n_exp;
        const bool ok = out_range(out, i, c0, n_exp, err);
        int64_t ab = 0, ae = 0;
        if (ok) a_row_range(op, i, ab, ae, err);
        int cnt = 0, full = 0;
        warp_enum<V, true>(op, ab, ae, es, err, [&](bool act, int j, V a, V b) {
            bool ins = false;
            int h = -1;
            if (act) {
                h = cas_insert(keys, tbits, hc, j, ins);
                if (h >= 0) {
                    atomicAdd(vals + h, a * b);
                    if (ins) atomicAdd(bc + (j >> bsh), 1);
                } else {
                    full = 1;
                }
            }
            const unsigned m = __ballot_sync(kFull, ins);
            if (ins) {
                const int pos = cnt + __popc(m & lanemask_lt());
                if (pos < lcap) list[pos] = h;
            }
            cnt += __popc(m);
        });
        full = __any_sync(kFull, full);
        const int tot = cnt;
        bool over;
        if (out.row_nnz) {
            over = full || tot > n_exp || tot > lcap;
            if (lane == 0) out.row_nnz[i] = over ? -1 : tot;
        } else {
            over = full || tot != n_exp || tot > lcap;
            if (lane == 0) {
                if (full || tot > lcap) raise_err(err, kErrTableFull);
                else if (tot != n_exp) raise_err(err, kErrCountMismatch);
            }
        }
        __syncwarp();
        if (over) {
            // nothing is written; the table and the counts go back to zero
            if (full || tot > lcap) {
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
            for (int s = lane; s < NB; s += 32) bc[s] = 0;
        } else if (tot <= 32) {
            // rank of each entry among the row's (at most 32) columns
            int k = INT_MAX;
            V v = V(0);
            if (lane < tot) {
                const int h = list[lane];
                k = keys[h];
                v = vals[h];
                keys[h] = kEmpty;
                vals[h] = V(0);
            }
            int rank = 0;
            for (int m = 0; m < tot; ++m) rank += __shfl_sync(kFull, k, m) < k ? 1 : 0;
            if (lane < tot) {
                out.c_ci[c0 + rank] = k;
                out.c_val[c0 + rank] = v;
            }
            for (int s = lane; s < NB; s += 32) bc[s] = 0;
        } else {
            // bucket starts: each lane sums a run of consecutive buckets
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
            // group the entries by bucket; the table goes back to EMPTY / 0
            for (int q = lane; q < tot; q += 32) {
                const int h = list[q];
                const int k = keys[h];
                const V v = vals[h];
                keys[h] = kEmpty;
                vals[h] = V(0);
                const int p = atomicAdd(bc + (k >> bsh), 1);
                gk[p] = k;
                gv[p] = v;
            }
            __syncwarp();
            // bc[b] is now the end of bucket b: rank inside the bucket
            for (int q = lane; q < tot; q += 32) {
                const int k = gk[q];
                const int b = k >> bsh;
                const int e = bc[b];
                const int s0 = b ? bc[b - 1] : 0;
                int rk = 0;
                for (int x = s0; x < e; ++x) rk += gk[x] < k ? 1 : 0;
                out.c_ci[c0 + s0 + rk] = k;
                out.c_val[c0 + s0 + rk] = gv[q];
            }
            __syncwarp();
            for (int s = lane; s < NB; s += 32) bc[s] = 0;
        }
        __syncwarp();
    }
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

size_t sym_warp_smem(int tbits) {
    return (size_t)kWarpRowWarps * (((size_t)4 << tbits) + sizeof(EntryScratch<float>));
}

void launch_sym_warp(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                     int *nnz_out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    const Operands<float> op = warp_operands<float>(r);
    const size_t smem = sym_warp_smem(hl.tbits);
    auto kern = k_sym_warp<kWarpRowWarps>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    kern<<<warp_grid(kern, smem, hl.sms, count), kWarpRowWarps * 32, smem, s>>>(op, rows, count, token, hl.tbits, hc,
                                                                              nnz_out, err);
}

// List room L: the most columns a row of the bin may hold (T * max_load,
// rounded up to 32, at most T); NB = T / 4 buckets over the column range.
static int warp_lcap(int tbits, float inv_load) {
    const int T = 1 << tbits;
    int L = (int)((double)T / (double)inv_load + 0.999);
    L = (L + 31) & ~31;
    return L < 32 ? 32 : (L > T ? T : L);
}

size_t num_warp_smem(int dtype, int tbits, float inv_load) {
    const int T = 1 << tbits;
    const int L = warp_lcap(tbits, inv_load);
    const int NB = T >> 2;
    const size_t per = dtype ? warp_row_bytes<double>(T, L, NB) : warp_row_bytes<float>(T, L, NB);
    return (size_t)kWarpRowWarps * per;
}

template <typename V>
static void num_warp_typed(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                           float inv_load, const NumOut &o, int *err, cudaStream_t s) {
    const Operands<V> op = warp_operands<V>(r);
    const NumOutT<V> out{o.c_rp, o.c_ci, (V *)o.c_val, o.c_nnz, o.row_nnz};
    const int L = warp_lcap(hl.tbits, inv_load);
    const int nbb = 2;
    const int NB = (1 << hl.tbits) >> nbb;
    int nbbits = 0;
    while ((1 << nbbits) < NB) ++nbbits;
    const int bsh = hl.colbits > nbbits ? hl.colbits - nbbits : 0;
    const size_t smem = num_warp_smem(sizeof(V) == 8, hl.tbits, inv_load);
    auto kern = k_num_warp<V, kWarpRowWarps>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    kern<<<warp_grid(kern, smem, hl.sms, count), kWarpRowWarps * 32, smem, s>>>(op, rows, count, token, hl.tbits, hc,
                                                                              L, nbb, bsh, out, err);
}

void launch_num_warp(int dtype, const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                     float inv_load, const NumOut &out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    if (dtype) num_warp_typed<double>(r, rows, count, token, hl, inv_load, out, err, s);
    else num_warp_typed<float>(r, rows, count, token, hl, inv_load, out, err, s);
}

}  // namespace smash
