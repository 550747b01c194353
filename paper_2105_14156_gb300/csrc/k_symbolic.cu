// Symbolic phase: the exact number of distinct columns of every row of C.
//
// Hashing Phase without values: every product's column tag is inserted into
// a per-row open-addressing table with compare-and-swap on EMPTY (= -1), +1
// linear probing on collision; the row's count is the number of successful
// inserts. Three table placements, by row size:
//   k_sym_hash   shared-memory table of 2^tbits int32 tags, one thread group
//                per row, rows claimed by atomic tokens (Version 2's
//                tokenization: a work counter instead of a static schedule);
//   k_sym_dense  the paper's "dense row": a bitmap over all columns of B in
//                shared memory (no probing), for rows whose bound is a large
//                fraction of cols(B);
//   k_sym_spill  the table in global memory (Version 3 moved it to DRAM), for
//                rows too large for shared memory when the bitmap does not fit.
#include "device_common.cuh"
#include "kernels.h"

namespace smash {

template <int GS, int NT>
__global__ void __launch_bounds__(NT) k_sym_hash(Operands<float> op, const int *rows, int count, int *token,
                                                 int tbits, HashCfg hc, int *nnz_out, int *err) {
    using G = Group<GS, NT>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][G::kGroups];
    const int T = 1 << tbits;
    int *keys = (int *)smem + (size_t)G::gid() * T;
    // group scratch (GS > 32 only: warp rows enumerate from registers)
    unsigned char *scr = smem + (size_t)G::kGroups * T * 4 + (size_t)G::gid() * prod_scratch_bytes<float, GS>();
    const ProdScratch<float> sc = carve_prod_scratch<float, GS>(scr);
    const int t = G::tid();
    RowClaim<G> claim(token, s_row);
    for (;;) {
        const int r = claim.next(count);
        if (r >= count) break;
        const int i = rows[r];
        for (int s = t; s < T; s += GS) keys[s] = kEmpty;
        G::sync();
        int64_t ab, ae;
        a_row_range(op, i, ab, ae, err);
        int cnt = 0;
        // warp rows: the register-staged enumerator (measured faster here than
        // the shared-memory one, which the numeric warp rows use)
        auto ins_key = [&](int j, float, float) {
            bool ins;
            if (hash_find_or_insert<false>(keys, tbits, hc, j, ins) < 0) raise_err(err, kErrTableFull);
            cnt += ins ? 1 : 0;
        };
        if constexpr (GS == 32) warp_products<float, false>(op, ab, ae, err, ins_key);
        else group_products<float, false, GS, NT>(op, ab, ae, sc, err, ins_key);
        int tot;
        if constexpr (GS == 32) tot = warp_sum(cnt);
        else tot = G::template sum<int>(cnt, sc.red);
        if (t == 0) nnz_out[i] = tot;
        G::sync();
    }
}

// Size check of the numeric count pass (see NumCheck).
__device__ __forceinline__ void count_check(const NumCheck &nc, int i, int tot, int *err) {
    const int64_t s = nc.c_rp[i], t = nc.c_rp[i + 1];
    if (s < 0 || t < s || t > nc.c_nnz) {
        raise_err(err, kErrBadRowPtr);
        if (nc.row_nnz) nc.row_nnz[i] = -1;
        return;
    }
    if (nc.row_nnz) nc.row_nnz[i] = (int64_t)tot <= t - s ? tot : -1;
    else if ((int64_t)tot != t - s) raise_err(err, kErrCountMismatch);
}

// Dense rows: a bitmap over the columns of B; count = popcount. With wc.wcnt
// the row's distinct columns are also counted per block of kSubCols columns
// (slot = wc.slot_base + r), for the numeric dense kernel.
template <int NT>
__global__ void __launch_bounds__(NT) k_sym_dense(Operands<float> op, const int *rows, int count, int *token,
                                                  int words, WinCount wc, int *nnz_out, NumCheck nc, int *err) {
    using G = Group<NT, NT>;
    constexpr int kWarps = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row[2][1];
    unsigned *bm = (unsigned *)smem;
    const ProdScratch<float> sc = carve_prod_scratch<float, NT>(smem + (size_t)words * 4);
    const int t = threadIdx.x;
    const int lane = lane_id();
    const int wp = t >> 5;
    RowClaim<G> claim(token, s_row);
    for (;;) {
        const int r = claim.next(count);
        if (r >= count) break;
        const int i = rows[r];
        int64_t slot = -1;
        if (wc.wcnt && wc.skip_slotted) slot = wc.wslot[i];
        if (slot >= 0) {
            // counted before: only the size check
            int c = 0;
            for (int q = t; q < wc.nsub; q += NT) c += wc.wcnt[slot * wc.nsub + q];
            const int tot = G::template sum<int>(c, sc.red);
            if (t == 0) count_check(nc, i, tot, err);
            __syncthreads();
            continue;
        }
        for (int w = t; w < words; w += NT) bm[w] = 0u;
        __syncthreads();
        int64_t ab, ae;
        a_row_range(op, i, ab, ae, err);
        group_products<float, false, NT, NT>(op, ab, ae, sc, err, [&](int j, float, float) {
            const unsigned bit = 1u << (j & 31);
            unsigned *w = bm + (j >> 5);
            if (!(*(volatile unsigned *)w & bit)) atomicOr(w, bit);
        });
        __syncthreads();
        int cnt = 0;
        for (int w = t; w < words; w += NT) cnt += __popc(bm[w]);
        const int tot = G::template sum<int>(cnt, sc.red);
        if (wc.wcnt) {
            slot = wc.slot_base + r;
            constexpr int kSubWords = kSubCols / 32;
            for (int q = wp; q < wc.nsub; q += kWarps) {
                const int w1 = min((q + 1) * kSubWords, words);
                int c = 0;
                for (int x = q * kSubWords + lane; x < w1; x += 32) c += __popc(bm[x]);
                c = warp_sum(c);
                if (lane == 0) wc.wcnt[slot * wc.nsub + q] = (uint16_t)c;
            }
            if (t == 0) wc.wslot[i] = (int)slot;
        }
        if (t == 0) {
            if (nnz_out) nnz_out[i] = tot;
            else count_check(nc, i, tot, err);
        }
        __syncthreads();
    }
}

// Spill rows: the key table lives in global memory, one slice per block.
template <int NT>
__global__ void __launch_bounds__(NT) k_sym_spill(Operands<float> op, const int *rows, int count, int *token,
                                                  HashCfg hc, float inv_load, const long long *bound,
                                                  int spill_tbits, int *tables, int *nnz_out, int *err) {
    using G = Group<NT, NT>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_row;
    const ProdScratch<float> sc = carve_prod_scratch<float, NT>(smem);
    int *keys = tables + ((size_t)blockIdx.x << spill_tbits);
    const int t = threadIdx.x;
    for (;;) {
        if (t == 0) s_row = atomicAdd(token, 1);
        __syncthreads();
        const int r = s_row;
        if (r >= count) break;
        const int i = rows[r];
        int tb = table_bits(bound[i], inv_load);
        if (tb > spill_tbits) {
            raise_err(err, kErrTableFull);
            tb = spill_tbits;
        }
        const int T = 1 << tb;
        for (int s = t; s < T; s += NT) __stcg(keys + s, kEmpty);
        __syncthreads();
        int64_t ab, ae;
        a_row_range(op, i, ab, ae, err);
        int cnt = 0;
        group_products<float, false, NT, NT>(op, ab, ae, sc, err, [&](int j, float, float) {
            bool ins;
            if (hash_find_or_insert<true>(keys, tb, hc, j, ins) < 0) raise_err(err, kErrTableFull);
            cnt += ins ? 1 : 0;
        });
        const int tot = G::template sum<int>(cnt, sc.red);
        if (t == 0) nnz_out[i] = tot;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
static Operands<float> sym_operands(const RawOperands &r) {
    Operands<float> o;
    o.a_rp = r.a_rp;
    o.a_ci = r.a_ci;
    o.a_val = nullptr;
    o.b_rp = r.b_rp;
    o.b_ci = r.b_ci;
    o.b_val = nullptr;
    o.a_nnz = r.a_nnz;
    o.b_nnz = r.b_nnz;
    o.b_rows = r.b_rows;
    o.ncols = r.ncols;
    return o;
}


template <typename K>
static int resident_grid(K kernel, int nt, size_t smem, int sms, int want_blocks, int cap_per_sm = 64) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > cap_per_sm) per_sm = cap_per_sm;
    long long cap = (long long)per_sm * sms;
    return (int)(want_blocks < cap ? want_blocks : cap);
}

template <int GS, int NT>
static void sym_hash_launch(const Operands<float> &op, const int *rows, int count, int *token, int tbits,
                            HashCfg hc, int sms, int *nnz_out, int *err, cudaStream_t s) {
    constexpr int groups = NT / GS;
    const size_t smem = (size_t)groups * ((size_t)4 << tbits) +
                        (GS > 32 ? (size_t)groups * prod_scratch_bytes<float, GS>() : 0);
    auto kern = k_sym_hash<GS, NT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int want = (count + groups - 1) / groups;
    const int grid = resident_grid(kern, NT, smem, sms, want);
    kern<<<grid, NT, smem, s>>>(op, rows, count, token, tbits, hc, nnz_out, err);
}

static int threads_per_row(int tbits, int shift) {
    int t = 1 << (tbits > shift ? tbits - shift : 0);
    if (t < 32) t = 32;
    if (t > 1024) t = 1024;
    return t;
}

void launch_sym_hash(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                     int *nnz_out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    const Operands<float> op = sym_operands(r);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    switch (threads_per_row(hl.tbits, hl.group_shift)) {
        case 32: sym_hash_launch<32, 256>(op, rows, count, token, hl.tbits, hc, hl.sms, nnz_out, err, s); break;
        case 64: sym_hash_launch<64, 64>(op, rows, count, token, hl.tbits, hc, hl.sms, nnz_out, err, s); break;
        case 128: sym_hash_launch<128, 128>(op, rows, count, token, hl.tbits, hc, hl.sms, nnz_out, err, s); break;
        case 256: sym_hash_launch<256, 256>(op, rows, count, token, hl.tbits, hc, hl.sms, nnz_out, err, s); break;
        case 512: sym_hash_launch<512, 512>(op, rows, count, token, hl.tbits, hc, hl.sms, nnz_out, err, s); break;
        default: sym_hash_launch<1024, 1024>(op, rows, count, token, hl.tbits, hc, hl.sms, nnz_out, err, s); break;
    }
}

// Block size and blocks per SM of the bitmap kernel: as many resident
// threads as the bitmaps allow, then as many rows in flight as possible (or
// the requested blocks per SM).
static void sym_dense_shape(const HashLaunch &hl, int64_t ncols, int &nt, int &per_sm) {
    const size_t words = (size_t)((ncols + 31) / 32);
    const int sm_smem = max_smem_per_sm();
    const int nts[3] = {1024, 512, 256};
    const size_t scr[3] = {prod_scratch_bytes<float, 1024>(), prod_scratch_bytes<float, 512>(),
                           prod_scratch_bytes<float, 256>()};
    int best_nt = 1024, best_b = 1, best_thr = 0;
    for (int q = 0; q < 3; ++q) {
        if (best_thr == (1 << 30)) break;
        const size_t per_block = words * 4 + scr[q] + 1024;
        if (per_block > (size_t)max_smem_per_block() + 1024) continue;
        int b = (int)((size_t)sm_smem / per_block);
        if (b > 2048 / nts[q]) b = 2048 / nts[q];
        if (b < 1) continue;
        if (hl.sym_dense_blocks > 0) {
            if (b >= hl.sym_dense_blocks && nts[q] * hl.sym_dense_blocks <= 2048) {
                best_nt = nts[q];
                best_b = hl.sym_dense_blocks;
                best_thr = 1 << 30;
            }
            continue;
        }
        if (b * nts[q] > best_thr || (b * nts[q] == best_thr && b > best_b)) {
            best_thr = b * nts[q];
            best_nt = nts[q];
            best_b = b;
        }
    }
    nt = best_nt;
    per_sm = best_b;
}

int sym_dense_threads(const HashLaunch &hl, int64_t ncols) {
    int nt, b;
    sym_dense_shape(hl, ncols, nt, b);
    return nt;
}

template <int NT>
static void sym_dense_go(const Operands<float> &op, const int *rows, int count, int *token, int per_sm,
                         const HashLaunch &hl, const WinCount &wc, int *nnz_out, const NumCheck &nc, int *err,
                         cudaStream_t s) {
    const int words = (op.ncols + 31) / 32;
    const size_t smem = (size_t)words * 4 + prod_scratch_bytes<float, NT>();
    auto kern = k_sym_dense<NT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = resident_grid(kern, NT, smem, hl.sms, count, per_sm);
    kern<<<grid, NT, smem, s>>>(op, rows, count, token, words, wc, nnz_out, nc, err);
}

void launch_sym_dense(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                      const WinCount &wc, int *nnz_out, const NumCheck &nc, int *err, cudaStream_t s) {
    if (count <= 0) return;
    const Operands<float> op = sym_operands(r);
    int nt, per_sm;
    sym_dense_shape(hl, r.ncols, nt, per_sm);
    if (nt == 256) sym_dense_go<256>(op, rows, count, token, per_sm, hl, wc, nnz_out, nc, err, s);
    else if (nt == 512) sym_dense_go<512>(op, rows, count, token, per_sm, hl, wc, nnz_out, nc, err, s);
    else sym_dense_go<1024>(op, rows, count, token, per_sm, hl, wc, nnz_out, nc, err, s);
}

int sym_spill_grid(const HashLaunch &hl) {
    const int per = hl.blocks_per_sm > 0 ? hl.blocks_per_sm : 1;
    return hl.sms * per;
}

void launch_sym_spill(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                      float inv_load, const long long *bound, int spill_tbits, int *tables, int *nnz_out,
                      int *err, cudaStream_t s) {
    if (count <= 0) return;
    const Operands<float> op = sym_operands(r);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    const size_t smem = prod_scratch_bytes<float, 1024>();
    auto kern = k_sym_spill<1024>;
    int grid = sym_spill_grid(hl);
    if (grid > count) grid = count;
    kern<<<grid, 1024, smem, s>>>(op, rows, count, token, hc, inv_load, bound, spill_tbits, tables, nnz_out, err);
}

}  // namespace smash
