// Group rows: one block of GS threads (64 to 1024) per row of C, for the bins
// whose tables hold a thousand columns or more.
//
// The numeric phase of the warp rows (k_warp.cuh), with the row's products
// spread over the block's warps (group_enum in warp_enum.cuh: a batch of A's
// entries staged in shared memory, one contiguous range of the batch's
// products per warp). Each product is inserted with compare-and-swap first
// (EMPTY -> j, +1 linear probing), its value added to the slot, and every
// newly claimed slot appended to the row's list (one shared counter, one
// atomic per warp and step). The Write-back Phase visits the listed entries
// only: a counting sort by the high bits of the column in the table's own
// memory, each entry's rank inside its bucket, the row streamed to C.
// Rows known to repeat no column (exact mode) or whose products fit their
// capacity (capacity mode) skip the table: their products are staged as
// they come, sorted the same way, and equal columns summed after the sort.
//
// Included by k_group_f32.cu and k_group_f64.cu, one value type each (two
// translation units compiled side by side).
#pragma once
#include <climits>

#include "device_common.cuh"
#include "kernels.h"
#include "warp_enum.cuh"
#include "writeout.cuh"

namespace smash {

// Shared memory of a group: keys[T], vals[T], list[L], bc[NB], the product
// scratch of group_enum.
template <typename V, int GS>
__host__ __device__ constexpr size_t group_row_bytes(int T, int L, int NB) {
    return (size_t)T * (4 + sizeof(V)) + (size_t)L * 4 + (size_t)NB * 4 + num_scratch_bytes<V, GS>();
}

// Block-wide exclusive scan of one value per thread (total in *tot).
template <int GS>
__device__ __forceinline__ int group_scan(int v, int *red, int *tot) {
    return Group<GS, GS>::template excl_scan<int>(v, red, tot);
}

template <typename V, typename IT, int K, int GS>
__global__ void __launch_bounds__(GS) k_num_group(Operands<V> op, const int *rows, int count, int *token, int tbits,
                                                  HashCfg hc, int lcap, int nb, int bsh, const RowGather *rec,
                                                  NumOutT<V> out, int *err) {
    using G = Group<GS, GS>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][1];
    __shared__ int s_cnt, s_full;
    const int T = 1 << tbits;
    const int NB = nb;
    int *keys = (int *)smem;
    V *vals = (V *)(smem + (size_t)T * 4);
    int *list = (int *)(smem + (size_t)T * (4 + sizeof(V)));
    int *bc = list + lcap;
    const ProdScratch<V> sc = carve_prod_scratch<V, GS>((unsigned char *)(bc + NB));
    const int t = threadIdx.x;
    const int lane = lane_id();
    for (int s = t; s < T; s += GS) {
        keys[s] = kEmpty;
        vals[s] = V(0);
    }
    for (int s = t; s < NB; s += GS) bc[s] = 0;
    if (t == 0) {
        s_cnt = 0;
        s_full = 0;
    }
    __syncthreads();
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
        const long long f_i = rec && ok ? rec[i].f : -1;
        const bool direct = !out.row_nnz && f_i >= 0 && n_exp <= lcap && f_i == (long long)n_exp;
        const bool merge = out.row_nnz && f_i >= 0 && f_i <= (long long)n_exp && f_i <= lcap && 2 * f_i <= T;
        if (direct || merge) {
            group_enum<V, IT, true, GS>(op, ab, ae, sc, err, [&](bool act, int j, V a, V b, int p) {
                if (act && p < lcap) {
                    keys[p] = j;
                    vals[p] = a * b;
                }
                const unsigned m = __ballot_sync(kFull, act);
                if (lane == 0 && m) atomicAdd(&s_cnt, __popc(m));
            });
        } else {
            group_enum<V, IT, true, GS>(op, ab, ae, sc, err, [&](bool act, int j, V a, V b, int) {
                bool ins = false;
                int h = -1;
                if (act) {
                    h = cas_insert(keys, tbits, hc, j, ins);
                    if (h >= 0) atomicAdd(vals + h, a * b);
                    else s_full = 1;
                }
                const unsigned m = __ballot_sync(kFull, ins);
                int base = 0;
                if (lane == 0 && m) base = atomicAdd(&s_cnt, __popc(m));
                base = __shfl_sync(kFull, base, 0);
                if (ins) {
                    const int pos = base + __popc(m & lanemask_lt());
                    if (pos < lcap) list[pos] = h;
                }
            });
        }
        // group_enum ends with a barrier: the counts are complete (and read by
        // every thread before the barrier below lets them be reset)
        const int tot = s_cnt;
        const bool full = s_full != 0;
        __syncthreads();
        bool over;
        if (out.row_nnz) {
            over = full || tot > n_exp || tot > lcap;
            if (t == 0 && (over || !merge)) out.row_nnz[i] = over ? -1 : tot;
        } else {
            over = full || tot != n_exp || tot > lcap;
            if (t == 0) {
                if (full || tot > lcap) raise_err(err, kErrTableFull);
                else if (tot != n_exp) raise_err(err, kErrCountMismatch);
            }
        }
        if (over) {
            // nothing is written; the table goes back to EMPTY / 0
            if (full || tot > lcap || direct || merge) {
                for (int s = t; s < T; s += GS) {
                    keys[s] = kEmpty;
                    vals[s] = V(0);
                }
            } else {
                for (int q = t; q < tot; q += GS) {
                    const int h = list[q];
                    keys[h] = kEmpty;
                    vals[h] = V(0);
                }
            }
        } else {
            const bool staged = direct || merge;
            // 1. the entries into registers, their slots back to EMPTY / 0,
            //    counts per bucket (bucket = column >> bsh, monotone in the column)
            int kk[K], pp[K];
            V vv[K];
#pragma unroll
            for (int x = 0; x < K; ++x) {
                const int q = t + GS * x;
                kk[x] = INT_MAX;
                vv[x] = V(0);
                pp[x] = -1;
                if (q < tot) {
                    const int h = staged ? q : list[q];
                    kk[x] = keys[h];
                    vv[x] = vals[h];
                    keys[h] = kEmpty;
                    vals[h] = V(0);
                    atomicAdd(bc + (kk[x] >> bsh), 1);
                }
            }
            __syncthreads();
            // 2. bucket starts: each thread sums a run of consecutive buckets
            {
                const int run = (NB + GS - 1) / GS;
                const int b0 = min(t * run, NB), b1 = min(b0 + run, NB);
                int loc = 0;
                for (int b = b0; b < b1; ++b) loc += bc[b];
                int tsum;
                int acc = group_scan<GS>(loc, sc.red, &tsum);
                for (int b = b0; b < b1; ++b) {
                    const int c = bc[b];
                    bc[b] = acc;
                    acc += c;
                }
            }
            __syncthreads();
            // 3. grouped by bucket into keys[0..tot)
#pragma unroll
            for (int x = 0; x < K; ++x) {
                if (t + GS * x < tot) {
                    pp[x] = atomicAdd(bc + (kk[x] >> bsh), 1);
                    keys[pp[x]] = kk[x];
                }
            }
            __syncthreads();
            // 4. bc[b] is now the end of bucket b: each entry's place is its
            //    bucket's start plus the smaller columns of its bucket (equal
            //    columns, in a merged row, ordered by their grouped position)
#pragma unroll
            for (int x = 0; x < K; ++x) {
                if (t + GS * x < tot) {
                    const int b = kk[x] >> bsh;
                    const int e = bc[b];
                    const int s0 = b ? bc[b - 1] : 0;
                    int rk = 0;
                    for (int y = s0; y < e; ++y) {
                        const int ky = keys[y];
                        rk += (ky < kk[x] || (merge && ky == kk[x] && y < pp[x])) ? 1 : 0;
                    }
                    pp[x] = s0 + rk;
                }
            }
            if (!merge) {
#pragma unroll
                for (int x = 0; x < K; ++x) {
                    if (t + GS * x < tot) {
                        __stcs(out.c_ci + (c0 + pp[x]), kk[x]);
                        __stcs(out.c_val + (c0 + pp[x]), vv[x]);
                    }
                }
                __syncthreads();
                for (int q = t; q < tot; q += GS) {
                    keys[q] = kEmpty;
                    vals[q] = V(0);
                }
            } else {
                __syncthreads();
                // 5. the sorted products in keys[tot..2 tot), vals[tot..2 tot);
                //    the first of each run of equal columns sums the run and
                //    takes the next place of the row
#pragma unroll
                for (int x = 0; x < K; ++x) {
                    if (t + GS * x < tot) {
                        keys[tot + pp[x]] = kk[x];
                        vals[tot + pp[x]] = vv[x];
                    }
                }
                __syncthreads();
                int run_tot = 0;
#pragma unroll
                for (int x = 0; x < K; ++x) {
                    if (GS * x < tot) {   // (uniform)
                        const int q = t + GS * x;
                        bool first = false;
                        int sk = 0;
                        if (q < tot) {
                            sk = keys[tot + q];
                            first = q == 0 || keys[tot + q - 1] != sk;
                        }
                        int ct;
                        const int d = run_tot + group_scan<GS>(first ? 1 : 0, sc.red, &ct);
                        if (first) {
                            V v = vals[tot + q];
                            for (int y = q + 1; y < tot && keys[tot + y] == sk; ++y) v += vals[tot + y];
                            __stcs(out.c_ci + (c0 + d), sk);
                            __stcs(out.c_val + (c0 + d), v);
                        }
                        run_tot += ct;
                    }
                }
                if (t == 0) out.row_nnz[i] = run_tot;
                __syncthreads();
                for (int q = t; q < 2 * tot; q += GS) {
                    keys[q] = kEmpty;
                    vals[q] = V(0);
                }
            }
            for (int s = t; s < NB; s += GS) bc[s] = 0;
        }
        if (t == 0) {
            s_cnt = 0;
            s_full = 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
template <typename V>
static Operands<V> group_operands(const RawOperands &r) {
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

// List room L: the most columns a row of the bin may hold (T * max_load,
// rounded up to the group size, at most T); NB = T / 2 buckets.
static int group_lcap(int tbits, float inv_load, int gs) {
    const int T = 1 << tbits;
    int L = (int)((double)T / (double)inv_load + 0.999);
    L = (L + gs - 1) / gs * gs;
    return L > T ? T : L;
}

static int group_threads_of(int tbits, int shift) {
    int t = 1 << (tbits > shift ? tbits - shift : 0);
    return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

template <typename V>
[[maybe_unused]] static size_t group_smem_gs(int tbits, int L, int gs) {
    const int T = 1 << tbits, NB = T >> 1;
    switch (gs) {
        case 64: return group_row_bytes<V, 64>(T, L, NB);
        case 128: return group_row_bytes<V, 128>(T, L, NB);
        case 256: return group_row_bytes<V, 256>(T, L, NB);
        case 512: return group_row_bytes<V, 512>(T, L, NB);
        default: return group_row_bytes<V, 1024>(T, L, NB);
    }
}

template <typename V, typename IT, int K, int GS>
static void num_group_go(const Operands<V> &op, const int *rows, int count, int *token, const HashLaunch &hl, int L,
                         const RowGather *rec, const NumOutT<V> &out, int *err, cudaStream_t s, size_t smem) {
    const int NB = (1 << hl.tbits) >> 1;
    int nbbits = 0;
    while ((1 << nbbits) < NB) ++nbbits;
    const int bsh = hl.colbits > nbbits ? hl.colbits - nbbits : 0;
    auto kern = k_num_group<V, IT, K, GS>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GS, smem);
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)per_sm * hl.sms;
    const int grid = (int)(count < cap ? count : cap);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    kern<<<grid, GS, smem, s>>>(op, rows, count, token, hl.tbits, hc, L, NB, bsh, rec, out, err);
}

template <typename V, typename IT, int GS>
static void num_group_k(const Operands<V> &op, const int *rows, int count, int *token, const HashLaunch &hl, int L,
                        const RowGather *rec, const NumOutT<V> &out, int *err, cudaStream_t s, size_t smem) {
    const int k = (L + GS - 1) / GS;
    if (k <= 4) num_group_go<V, IT, 4, GS>(op, rows, count, token, hl, L, rec, out, err, s, smem);
    else if (k <= 8) num_group_go<V, IT, 8, GS>(op, rows, count, token, hl, L, rec, out, err, s, smem);
    else num_group_go<V, IT, 16, GS>(op, rows, count, token, hl, L, rec, out, err, s, smem);
}

template <typename V, typename IT>
static void num_group_gs(const Operands<V> &op, const int *rows, int count, int *token, const HashLaunch &hl, int L,
                         int gs, const RowGather *rec, const NumOutT<V> &out, int *err, cudaStream_t s, size_t smem) {
    switch (gs) {
        case 64: num_group_k<V, IT, 64>(op, rows, count, token, hl, L, rec, out, err, s, smem); break;
        case 128: num_group_k<V, IT, 128>(op, rows, count, token, hl, L, rec, out, err, s, smem); break;
        case 256: num_group_k<V, IT, 256>(op, rows, count, token, hl, L, rec, out, err, s, smem); break;
        case 512: num_group_k<V, IT, 512>(op, rows, count, token, hl, L, rec, out, err, s, smem); break;
        default: num_group_k<V, IT, 1024>(op, rows, count, token, hl, L, rec, out, err, s, smem); break;
    }
}

template <typename V>
static void num_group_typed(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                            float inv_load, const RowGather *rec, const NumOut &o, int *err, cudaStream_t s) {
    const Operands<V> op = group_operands<V>(r);
    const NumOutT<V> out{o.c_rp, o.c_ci, (V *)o.c_val, o.c_nnz, o.row_nnz};
    const int gs = group_threads_of(hl.tbits, hl.group_shift);
    const int L = group_lcap(hl.tbits, inv_load, gs);
    const size_t smem = num_group_smem(sizeof(V) == 8, hl.tbits, inv_load, hl.group_shift);
    // (B with 2^31 entries or more takes the staged kernel: the planner checks)
    num_group_gs<V, int32_t>(op, rows, count, token, hl, L, gs, rec, out, err, s, smem);
}

}  // namespace smash
