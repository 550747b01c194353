// Numeric phase: values of C = A*B, rows sorted by column.
//
// Hashing Phase with values: each product a_ik*b_kj is merged into the row's
// table as it is produced: compare-and-swap claims the tag's slot (EMPTY = -1,
// +1 linear probing), an atomic add accumulates the value (the "atomic fetch
// and add" merge). Write-back Phase: the occupied slots are gathered, ordered
// by column and streamed to C's row (Version 1 sorts the table before
// streaming it out; the sort here is one of three, chosen per row):
//   - warp rank:   rows of <= 32 entries held by one warp; each entry's rank is
//                  the number of smaller tags (register shuffles);
//   - bitmap rank: a bitmap over the columns of B plus a prefix count per
//                  32-bit word gives every tag its position directly;
//   - bitonic:     the compacted entries are sorted in shared memory.
// Table placements as in the symbolic phase: shared memory (k_num_hash),
// dense accumulator for dense rows (k_num_dense: values indexed by column,
// in shared memory when cols(B) is small, else a global-memory row buffer,
// occupancy in a shared bitmap), and a global-memory hash table (k_num_spill;
// Version 3's table in DRAM).
#include <climits>

#include <cooperative_groups.h>

#include "device_common.cuh"
#include "kernels.h"
#include "writeout.cuh"

namespace smash {

namespace cg = cooperative_groups;

// ----- shared-memory hash rows -----------------------------------------------
template <typename V, int GS, int NT>
__global__ void __launch_bounds__(NT) k_num_hash(Operands<V> op, const int *rows, int count, int *token,
                                                 int tbits, HashCfg hc, int bm_words, int bitmap_ratio,
                                                 NumOutT<V> out, int *err) {
    using G = Group<GS, NT>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[G::kGroups];
    const int T = 1 << tbits;
    const size_t tab_bytes = (size_t)T * (4 + sizeof(V));
    unsigned char *gb = smem + (size_t)G::gid() * tab_bytes;
    int *keys = (int *)gb;
    V *vals = (V *)(gb + (size_t)T * 4);
    unsigned char *scr = smem + (size_t)G::kGroups * tab_bytes + (size_t)G::gid() * num_scratch_bytes<V, GS>();
    const ProdScratch<V> sc = carve_prod_scratch<V, GS>(scr);
    unsigned *bm = (unsigned *)(smem + (size_t)G::kGroups * (tab_bytes + num_scratch_bytes<V, GS>()));
    int *pre = (int *)(bm + bm_words);
    const int t = G::tid();
    for (;;) {
        int r;
        if constexpr (GS == 32) {
            r = 0;
            if (t == 0) r = atomicAdd(token, 1);
            r = __shfl_sync(kFull, r, 0);
        } else {
            if (t == 0) s_row[G::gid()] = atomicAdd(token, 1);
            G::sync();
            r = s_row[G::gid()];
        }
        if (r >= count) break;
        const int i = rows[r];
        int64_t c0;
        int n_exp;
        const bool ok = out_range(out, i, c0, n_exp, err);
        const bool use_bm = (GS == NT) && bm_words > 0 && (long long)bm_words <= (long long)bitmap_ratio * n_exp;
        for (int s = t; s < T; s += GS) {
            keys[s] = kEmpty;
            vals[s] = V(0);
        }
        if (use_bm)
            for (int w = t; w < bm_words; w += GS) bm[w] = 0u;
        G::sync();
        int64_t ab = 0, ae = 0;
        if (ok) a_row_range(op, i, ab, ae, err);
        int cnt = 0, ovf = 0;
        row_products<V, true, GS, NT>(op, ab, ae, sc, err, [&](int j, V a, int64_t idx) {
            const V v = a * b_value(op, idx);
            bool ins;
            const int h = hash_find_or_insert<false>(keys, tbits, hc, j, ins);
            if (h >= 0) {
                atomicAdd(vals + h, v);
                cnt += ins ? 1 : 0;
            } else if (out.row_nnz) {
                ovf = 1;
            } else {
                raise_err(err, kErrTableFull);
            }
        });
        int tot;
        if constexpr (GS == 32) {
            tot = warp_sum(cnt);
            __syncwarp();
        } else {
            tot = G::template sum<int>(cnt, sc.red);
        }
        bool over = false;
        if (out.row_nnz) {
            int o;
            if constexpr (GS == 32) o = __any_sync(kFull, ovf);
            else o = G::template sum<int>(ovf, sc.red);
            over = o != 0 || tot > n_exp;
            if (t == 0) out.row_nnz[i] = over ? -1 : tot;
            n_exp = tot;
        } else if (t == 0 && tot != n_exp) {
            raise_err(err, kErrCountMismatch);
        }
        if (!over) {
            if (GS == 32 && tot <= 32) writeout_warp_rank<V>(keys, vals, T, tot, n_exp, out, c0);
            else if (use_bm) writeout_bitmap<V, GS, NT>(keys, vals, T, bm, pre, bm_words, n_exp, out, c0, sc.red);
            else writeout_bitonic<V, GS, NT>(keys, vals, T, n_exp, out, c0, sc.red);
        }
        G::sync();
    }
}

// ----- dense rows -------------------------------------------------------------
template <typename V, int NT, bool SACC>
__global__ void __launch_bounds__(NT) k_num_dense(Operands<V> op, const int *rows, int count, int *token,
                                                  int words, V *acc_g, NumOutT<V> out, int *err) {
    using G = Group<NT, NT>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row;
    unsigned *bm = (unsigned *)smem;
    int *pre = (int *)(bm + words);
    V *sacc = (V *)(smem + (size_t)words * 8);
    const size_t acc_bytes = SACC ? (((size_t)op.ncols * sizeof(V) + 15) & ~size_t(15)) : 0;
    const ProdScratch<V> sc = carve_prod_scratch<V, NT>(smem + (size_t)words * 8 + acc_bytes);
    V *acc = SACC ? sacc : acc_g + (size_t)blockIdx.x * (size_t)op.ncols;
    const int t = threadIdx.x;
    for (;;) {
        if (t == 0) s_row = atomicAdd(token, 1);
        __syncthreads();
        const int r = s_row;
        if (r >= count) break;
        const int i = rows[r];
        int64_t c0;
        int n_exp;
        const bool ok = out_range(out, i, c0, n_exp, err);
        for (int w = t; w < words; w += NT) bm[w] = 0u;
        if constexpr (SACC)
            for (int j = t; j < op.ncols; j += NT) sacc[j] = V(0);
        __syncthreads();
        int64_t ab = 0, ae = 0;
        if (ok) a_row_range(op, i, ab, ae, err);
        row_products<V, true, NT, NT>(op, ab, ae, sc, err, [&](int j, V a, int64_t idx) {
            const V v = a * b_value(op, idx);
            atomicAdd(acc + j, v);
            const unsigned bit = 1u << (j & 31);
            unsigned *w = bm + (j >> 5);
            if (!(*(volatile unsigned *)w & bit)) atomicOr(w, bit);
        });
        if constexpr (!SACC) __threadfence();
        __syncthreads();
        const int tot = bitmap_prefix<NT, NT>(bm, pre, words, sc.red);
        __syncthreads();
        if (out.row_nnz) {
            const bool over = tot > n_exp;
            if (t == 0) out.row_nnz[i] = over ? -1 : tot;
            if (over) n_exp = 0;   // still drain the accumulator below, write nothing
        } else if (t == 0 && tot != n_exp) {
            raise_err(err, kErrCountMismatch);
        }
        for (int w = t; w < words; w += NT) {
            unsigned bits = bm[w];
            int pos = pre[w];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int j = (w << 5) + b;
                V v;
                if constexpr (SACC) {
                    v = acc[j];
                } else {
                    v = __ldcg(acc + j);
                    __stcg(acc + j, V(0));
                }
                if (pos < n_exp) {
                    out.c_ci[c0 + pos] = j;
                    out.c_val[c0 + pos] = v;
                }
                ++pos;
            }
        }
        if constexpr (!SACC) __threadfence();
        __syncthreads();
    }
}

// ----- dense rows in a thread-block cluster -----------------------------------
// The row's accumulator (one value per column of B) is split over the shared
// memory of the CS blocks of a cluster: block q owns columns
// [q*cpc, (q+1)*cpc). Every block enumerates all products of the row and keeps
// those in its own window, so all accumulation uses local shared-memory
// atomics (a remote, distributed-shared-memory atomic costs about as much as
// twenty local integer ones). Each block ranks its columns by bitmap prefix
// counts; the blocks' counts, exchanged through distributed shared memory,
// give each window's offset, so the row is written sorted without a sort.
// Accumulator and bitmap are cleared as they are read out.
// Hot columns (see k_split.cu) accumulate in private per-warp slots instead:
// their products then contend only within one warp, and the slots are summed
// into the accumulator once per row.
template <typename V, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(1024)
    k_num_dense_cluster(Operands<V> op, const int *rows, int count, int *token, int cpc, const int *splits,
                        NumOutT<V> out, const unsigned *hot_bm_g, const int *hot_col_g, const int *hot_n_g, int H,
                        int *err) {
    constexpr int NT = 1024;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2];
    __shared__ int s_cnt[2];
    __shared__ int s_base, s_total;
    const int words = cpc >> 5;
    V *acc = (V *)smem;
    V *priv = (V *)(smem + (size_t)cpc * sizeof(V));           // [32 warps][H]
    unsigned *bm = (unsigned *)(priv + (size_t)32 * H);
    int *pre = (int *)(bm + words);
    unsigned *hbm = (unsigned *)(pre + words);                   // H > 0 only
    int *hpre = (int *)(hbm + (H > 0 ? words : 0));
    int *hcol = hpre + (H > 0 ? words : 0);
    const ProdScratch<V> sc = carve_prod_scratch<V, NT>((unsigned char *)(hcol + H));
    const int t = threadIdx.x;
    const int wp = t >> 5;
    const unsigned lo = (unsigned)splits[rank];
    const unsigned width = (unsigned)(splits[rank + 1] - splits[rank]);   // <= cpc
    op.slice = rank;   // with a sliced B, enumerate this block's window only
    for (int j = t; j < cpc; j += NT) acc[j] = V(0);
    for (int w = t; w < words; w += NT) bm[w] = 0u;
    int hn = 0;
    if (H > 0) {
        for (int k = t; k < 32 * H; k += NT) priv[k] = V(0);
        for (int w = t; w < words; w += NT) hbm[w] = hot_bm_g[(size_t)rank * words + w];
        hn = hot_n_g[rank];
        for (int k = t; k < hn; k += NT) hcol[k] = hot_col_g[(size_t)rank * H + k];
        __syncthreads();
        bitmap_prefix<NT, NT>(hbm, hpre, words, sc.red);
    }
    for (int it = 0;; ++it) {
        const int par = it & 1;
        if (rank == 0 && t == 0) s_row[par] = atomicAdd(token, 1);
        cl.sync();
        const int r = *cl.map_shared_rank(&s_row[par], 0);
        if (r >= count) break;
        const int i = rows[r];
        int64_t c0;
        int n_exp;
        const bool ok = out_range(out, i, c0, n_exp, err);
        int64_t ab = 0, ae = 0;
        if (ok) a_row_range(op, i, ab, ae, err);
        group_products<V, true, NT, NT>(op, ab, ae, sc, err, [&](int j, V a, int64_t idx) {
            const unsigned off = (unsigned)j - lo;
            if (off < width) {
                const V v = a * b_value(op, idx);
                const unsigned bit = 1u << (off & 31);
                const int w = (int)(off >> 5);
                if (H > 0 && (hbm[w] & bit)) atomicAdd(priv + wp * H + hpre[w] + __popc(hbm[w] & (bit - 1u)), v);
                else atomicAdd(acc + off, v);
                if (!(*(volatile unsigned *)(bm + w) & bit)) atomicOr(bm + w, bit);
            }
        });
        __syncthreads();
        for (int k = t; k < hn; k += NT) {
            V sum = V(0);
            for (int q = 0; q < 32; ++q) {
                sum += priv[q * H + k];
                priv[q * H + k] = V(0);
            }
            acc[hcol[k]] = sum;
        }
        if (H > 0) __syncthreads();
        const int cnt = bitmap_prefix<NT, NT>(bm, pre, words, sc.red);
        if (t == 0) s_cnt[par] = cnt;
        cl.sync();
        if (t == 0) {
            int base = 0, total = 0;
            for (int q = 0; q < CS; ++q) {
                const int c = *cl.map_shared_rank(&s_cnt[par], q);
                if (q < rank) base += c;
                total += c;
            }
            s_base = base;
            s_total = total;
        }
        __syncthreads();
        const int base = s_base;
        if (out.row_nnz) {
            const bool over = s_total > n_exp;
            if (rank == 0 && t == 0) out.row_nnz[i] = over ? -1 : s_total;
            if (over) n_exp = 0;   // still drain the accumulator below, write nothing
        } else if (rank == 0 && t == 0 && s_total != n_exp) {
            raise_err(err, kErrCountMismatch);
        }
        for (int w = t; w < words; w += NT) {
            unsigned bits = bm[w];
            int pos = base + pre[w];
            bm[w] = 0u;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int jl = (w << 5) + b;
                const V v = acc[jl];
                acc[jl] = V(0);
                if (pos < n_exp) {
                    out.c_ci[c0 + pos] = (int)lo + jl;
                    out.c_val[c0 + pos] = v;
                }
                ++pos;
            }
        }
        __syncthreads();
    }
    cl.sync();
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
        row_products<V, true, NT, NT>(op, ab, ae, sc, err, [&](int j, V a, int64_t idx) {
            const V v = a * b_value(op, idx);
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
        int mn = INT_MAX, mx = INT_MIN;
        for (int s = t; s < T; s += NT) {
            const int k = __ldcg(keys + s);
            if (k != kEmpty) {
                mn = min(mn, k);
                mx = max(mx, k);
            }
        }
        block_minmax<NT>(mn, mx, s_mm);
        long long done = 0;
        if (tot > 0) {
            for (long long w0 = ((long long)mn / WIN) * WIN; w0 <= (long long)mx; w0 += WIN) {
                for (int w = t; w < win_words; w += NT) bm[w] = 0u;
                __syncthreads();
                for (int s = t; s < T; s += NT) {
                    const long long k = __ldcg(keys + s);
                    if (k != kEmpty && k >= w0 && k < w0 + WIN) {
                        const int d = (int)(k - w0);
                        atomicOr(bm + (d >> 5), 1u << (d & 31));
                    }
                }
                __syncthreads();
                const int wt = bitmap_prefix<NT, NT>(bm, pre, win_words, sc.red);
                __syncthreads();
                for (int s = t; s < T; s += NT) {
                    const long long k = __ldcg(keys + s);
                    if (k != kEmpty && k >= w0 && k < w0 + WIN) {
                        const int d = (int)(k - w0);
                        const long long pos =
                            done + pre[d >> 5] + __popc(bm[d >> 5] & ((1u << (d & 31)) - 1u));
                        if (pos < n_exp) {
                            out.c_ci[c0 + pos] = (int)k;
                            out.c_val[c0 + pos] = __ldcg(vals + s);
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

static int block_threads(int gs) { return gs < 256 ? 256 : gs; }

template <typename V>
static size_t num_hash_smem(int tbits, int gs, int bm_words) {
    const int nt = block_threads(gs);
    const int groups = nt / gs;
    size_t scr = 0;
    switch (gs) {
        case 32: scr = num_scratch_bytes<V, 32>(); break;
        case 64: scr = num_scratch_bytes<V, 64>(); break;
        case 128: scr = num_scratch_bytes<V, 128>(); break;
        case 256: scr = num_scratch_bytes<V, 256>(); break;
        case 512: scr = num_scratch_bytes<V, 512>(); break;
        default: scr = num_scratch_bytes<V, 1024>(); break;
    }
    return (size_t)groups * (((size_t)(4 + sizeof(V))) << tbits) + (size_t)groups * scr + (size_t)bm_words * 8;
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
                        int bitmap_ratio, const NumOutT<V> &out, int *err, cudaStream_t s) {
    constexpr int NT = GS < 256 ? 256 : GS;
    constexpr int groups = NT / GS;
    int bm_words = 0;
    if (GS == NT && bitmap_ratio > 0) {
        const int words = (op.ncols + 31) / 32;
        if (num_hash_smem<V>(hl.tbits, GS, words) <= (size_t)max_smem_per_block()) bm_words = words;
    }
    const size_t smem = num_hash_smem<V>(hl.tbits, GS, bm_words);
    auto kern = k_num_hash<V, GS, NT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = resident_grid(kern, NT, smem, hl.sms, (count + groups - 1) / groups);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    kern<<<grid, NT, smem, s>>>(op, rows, count, token, hl.tbits, hc, bm_words, bitmap_ratio, out, err);
}

template <typename V>
static void num_hash_typed(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                           int bitmap_ratio, const NumOut &o, int *err, cudaStream_t s) {
    const Operands<V> op = num_operands<V>(r);
    const NumOutT<V> out = num_out<V>(o);
    switch (threads_per_row(hl.tbits, hl.group_shift)) {
        case 32: num_hash_go<V, 32>(op, rows, count, token, hl, bitmap_ratio, out, err, s); break;
        case 64: num_hash_go<V, 64>(op, rows, count, token, hl, bitmap_ratio, out, err, s); break;
        case 128: num_hash_go<V, 128>(op, rows, count, token, hl, bitmap_ratio, out, err, s); break;
        case 256: num_hash_go<V, 256>(op, rows, count, token, hl, bitmap_ratio, out, err, s); break;
        case 512: num_hash_go<V, 512>(op, rows, count, token, hl, bitmap_ratio, out, err, s); break;
        default: num_hash_go<V, 1024>(op, rows, count, token, hl, bitmap_ratio, out, err, s); break;
    }
}

void launch_num_hash(int dtype, const RawOperands &r, const int *rows, int count, int *token,
                     const HashLaunch &hl, float inv_load, int bitmap_ratio, const NumOut &out, int *err,
                     cudaStream_t s) {
    (void)inv_load;
    if (count <= 0) return;
    if (dtype) num_hash_typed<double>(r, rows, count, token, hl, bitmap_ratio, out, err, s);
    else num_hash_typed<float>(r, rows, count, token, hl, bitmap_ratio, out, err, s);
}

template <typename V>
static size_t dense_smem(int ncols, bool sacc) {
    const int words = (ncols + 31) / 32;
    size_t b = (size_t)words * 8 + num_scratch_bytes<V, 1024>();
    if (sacc) b += ((size_t)ncols * sizeof(V) + 15) & ~size_t(15);
    return b;
}

bool num_dense_uses_smem_acc(int dtype, int ncols) {
    const size_t s = dtype ? dense_smem<double>(ncols, true) : dense_smem<float>(ncols, true);
    return s <= (size_t)max_smem_per_block() / 2;   // leave room for two blocks per SM
}

int dense_bitmap_max_cols() {
    const size_t avail = (size_t)max_smem_per_block() - num_scratch_bytes<double, 1024>() - 64;
    return (int)((avail / 8) * 32);
}

int num_dense_grid(int dtype, const HashLaunch &hl, int ncols) {
    (void)ncols;
    (void)dtype;
    const int per = hl.blocks_per_sm > 0 ? hl.blocks_per_sm : 1;
    return hl.sms * per;
}

template <typename V>
static size_t dense_cluster_smem(int cpc, int H) {
    size_t b = (size_t)cpc * sizeof(V) + (size_t)32 * H * sizeof(V) + (size_t)(cpc / 32) * 8 +
               num_scratch_bytes<V, 1024>();
    if (H > 0) b += (size_t)(cpc / 32) * 8 + (size_t)H * 4;
    return b;
}

// Widest window (multiple of 32 columns) one 1024-thread block can accumulate.
int num_dense_cap(int dtype, int H) {
    int lo = 0, hi = 1 << 22;
    while (hi - lo > 32) {
        const int mid = ((lo + hi) / 2) & ~31;
        const size_t need = dtype ? dense_cluster_smem<double>(mid, H) : dense_cluster_smem<float>(mid, H);
        if (need <= (size_t)max_smem_per_block()) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Smallest cluster whose blocks together cover all columns (0: none up to 8).
int num_dense_cluster_size(int dtype, int ncols, int cluster_max, int H) {
    const long long cap = num_dense_cap(dtype, H);
    for (int cs = 1; cs <= 8 && cs <= cluster_max; cs <<= 1)
        if (cap * cs >= ncols) return cs;
    return 0;
}

template <typename V, int CS>
static void dense_cluster_go(Operands<V> op, const BSlices &sl, int cpc, const int *rows, int count, int *token,
                             const NumOutT<V> &out, int *err, cudaStream_t s) {
    const int H = sl.hot_n ? sl.hot_h : 0;
    const size_t smem = dense_cluster_smem<V>(cpc, H);
    if (CS > 1 && sl.woff) {
        op.b_ci = sl.ci;
        op.b_val = (const V *)sl.val;
        op.b_woff = sl.woff;
        op.nslices = CS;
    }
    auto kern = k_num_dense_cluster<V, CS>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        nclusters = 1;
    }
    if (nclusters > count) nclusters = count;
    kern<<<nclusters * CS, 1024, smem, s>>>(op, rows, count, token, cpc, sl.splits, out, sl.hot_bm, sl.hot_col,
                                            sl.hot_n, H, err);
}

template <typename V>
static void num_dense_typed(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                            void *acc, const BSlices &sl, const NumOut &o, int *err, cudaStream_t s) {
    const Operands<V> op = num_operands<V>(r);
    const NumOutT<V> out = num_out<V>(o);
    const int words = (r.ncols + 31) / 32;
    const int cs = sl.splits ? sl.nslices : 0;
    if (cs > 0) {
        switch (cs) {
            case 1: dense_cluster_go<V, 1>(op, sl, sl.cpc, rows, count, token, out, err, s); break;
            case 2: dense_cluster_go<V, 2>(op, sl, sl.cpc, rows, count, token, out, err, s); break;
            case 4: dense_cluster_go<V, 4>(op, sl, sl.cpc, rows, count, token, out, err, s); break;
            default: dense_cluster_go<V, 8>(op, sl, sl.cpc, rows, count, token, out, err, s); break;
        }
    } else {
        const size_t smem = dense_smem<V>(r.ncols, false);
        auto kern = k_num_dense<V, 1024, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int grid = num_dense_grid(sizeof(V) == 8, hl, r.ncols);
        if (grid > count) grid = count;
        kern<<<grid, 1024, smem, s>>>(op, rows, count, token, words, (V *)acc, out, err);
    }
}

void launch_num_dense(int dtype, const RawOperands &r, const int *rows, int count, int *token,
                      const HashLaunch &hl, void *acc, const BSlices &sl, const NumOut &out, int *err,
                      cudaStream_t s) {
    if (count <= 0) return;
    if (dtype) num_dense_typed<double>(r, rows, count, token, hl, acc, sl, out, err, s);
    else num_dense_typed<float>(r, rows, count, token, hl, acc, sl, out, err, s);
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
