// Batched SpGEMM: many independent products C_m = A_m * B_m in one persistent,
// work-stealing kernel.
//
// Not in the paper as such; it carries Version 2's tokenization (threads poll
// a shared token counter for the next piece of work instead of a static
// schedule) across products: every block repeatedly claims the next work item
// of a global list with one atomic add, so products of very different sizes
// keep all SMs busy. Items are (a) single large rows, processed by the whole
// block with one block-wide hash table, listed first so they start early, and
// (b) tiles of 8 consecutive rows of one product, one row per warp, each warp
// with its own accumulator: a dense array over the columns of B when B is
// narrow (the paper's "dense row"), else a small hash table.
//
// One cooperative launch runs four phases separated by grid barriers (each
// wait bounded; a barrier that times out sets an error word and the kernel
// returns): symbolic counts, per-product row-pointer scans, product base
// offsets, numeric values with sorted write-out. Rows too large for one
// block's table are done around the kernel by the regular per-product path.
#include "device_common.cuh"
#include "kernels.h"
#include "writeout.cuh"
#include "batch_types.h"

namespace smash {


__device__ __forceinline__ int find_mat(const int64_t *start, int nmat, int64_t g) {
    int lo = 0, hi = nmat;   // last m with start[m] <= g
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename V>
__device__ __forceinline__ Operands<V> mat_ops(const BatchMat &m) {
    Operands<V> o;
    o.a_rp = m.a_rp;
    o.a_ci = m.a_ci;
    o.a_val = (const V *)m.a_val;
    o.b_rp = m.b_rp;
    o.b_ci = m.b_ci;
    o.b_val = (const V *)m.b_val;
    o.a_nnz = m.a_nnz;
    o.b_nnz = m.b_nnz;
    o.b_rows = m.b_rows;
    o.ncols = m.ncols;
    return o;
}

__device__ __forceinline__ int colbits(int n) {
    int b = 0;
    while ((1 << b) < n && b < 31) ++b;
    return b;
}

// Row classification over all products' rows (one warp per row).
__global__ void __launch_bounds__(256) k_batch_rowinfo(BatchArgs p) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_ub = 0, my_f = 0;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < p.nrows; g += warps) {
        const int mi = find_mat(p.row_start, p.nmat, g);
        const BatchMat &M = p.mats[mi];
        const int64_t r = g - p.row_start[mi];
        int64_t ab = __ldg(M.a_rp + r), ae = __ldg(M.a_rp + r + 1);
        if (ab < 0 || ae < ab || ae > M.a_nnz) {
            if (lane == 0) raise_err(p.err, kErrBadRowPtr);
            ab = ae = 0;
        }
        long long f = 0;
        for (int64_t e = ab + lane; e < ae; e += 32) {
            const int k = __ldg(M.a_ci + e);
            if ((unsigned)k < (unsigned)M.b_rows) {
                const int64_t s = __ldg(M.b_rp + k), t = __ldg(M.b_rp + k + 1);
                if (s >= 0 && t >= s && t <= M.b_nnz) f += t - s;
                else raise_err(p.err, kErrBadRowPtr);
            } else {
                raise_err(p.err, kErrBadIndex);
            }
        }
        f = warp_sum(f);
        if (lane == 0) {
            const long long ub = f < (long long)M.ncols ? f : (long long)M.ncols;
            uint8_t c;
            if (ub == 0) c = kRowEmpty;
            else if (M.ncols <= p.dense_max || table_bits(ub, p.inv_load) <= p.warp_bits) c = kRowSmall;
            else if (table_bits(ub, p.inv_load) <= p.block_bits) c = kRowBig;
            else c = kRowHuge;
            p.cls[g] = c;
            p.ub[g] = (int)ub;
            p.nnz[g] = 0;
            if (c == kRowBig) p.big[atomicAdd(p.counters + 0, 1)] = (int)g;
            if (c == kRowHuge) p.huge[atomicAdd(p.counters + 1, 1)] = (int)g;
            my_ub += (unsigned long long)ub;
            my_f += (unsigned long long)f;
        }
    }
    if (lane == 0) {
        atomicAdd(p.sums + 0, my_ub);
        atomicAdd(p.sums + 1, my_f);
    }
}

// Grid barrier for a cooperative launch; returns false after a timeout
// (wait_spins polls). missing > 0 makes the barrier wait for arrivals that
// never come, so that every block's wait runs out (a test of the time-out).
__device__ __forceinline__ bool grid_barrier(int *bar, int *err, long long wait_spins, int missing) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int *gen = bar + 1;
        const int g = *gen;
        __threadfence();
        const int arrived = atomicAdd(bar, 1);
        int ok = 1;
        if (arrived == (int)gridDim.x - 1 + missing) {
            atomicExch(bar, 0);
            __threadfence();
            atomicAdd(bar + 1, 1);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it > wait_spins) {
                    raise_err(err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename V>
struct BatchSmem {
    unsigned char *tab;     // 8 warp tables (or one block table)
    ProdScratch<V> sc;      // block-wide product staging
};

// One small row by one warp: count (NUM = false) or values + write-out.
template <typename V, bool NUM>
__device__ void warp_row(const BatchArgs &p, const BatchMat &M, int64_t g, int64_t r, unsigned char *wtab, int64_t c0,
                         int n_exp, int64_t base) {
    const Operands<V> op = mat_ops<V>(M);
    const int lane = lane_id();
    int64_t ab, ae;
    a_row_range(op, r, ab, ae, p.err);
    const int T = 1 << p.tw_bits;
    if (M.ncols <= p.dense_max && NUM && p.stage_ci) {
        // one-pass row: copy the row staged by the first phase to its place
        const int64_t so = p.stage_off[g];
        for (int q = lane; q < n_exp; q += 32) {
            p.ci_pool[base + c0 + q] = p.stage_ci[so + q];
            ((V *)p.val_pool)[base + c0 + q] = ((const V *)p.stage_val)[so + q];
        }
        return;
    }
    if (M.ncols <= p.dense_max && !NUM && p.stage_ci) {
        // one-pass row: values, count and the sorted row (staged) at once
        const int words = (M.ncols + 31) >> 5;
        V *acc = (V *)wtab;
        unsigned *bm = (unsigned *)(wtab + (((size_t)M.ncols * sizeof(V) + 15) & ~(size_t)15));
        for (int w = lane; w < words; w += 32) bm[w] = 0u;
        for (int j = lane; j < M.ncols; j += 32) acc[j] = V(0);
        __syncwarp();
        warp_products<V, true>(op, ab, ae, p.err, [&](int j, V a, V bkj) {
            atomicAdd(acc + j, a * bkj);
            const unsigned bit = 1u << (j & 31);
            if (!(*(volatile unsigned *)(bm + (j >> 5)) & bit)) atomicOr(bm + (j >> 5), bit);
        });
        __syncwarp();
        const int64_t so = p.stage_off[g];
        const int room = p.ub[g];
        int run = 0;
        for (int w = 0; w < words; ++w) {
            const unsigned bits = bm[w];
            const int j = (w << 5) + lane;
            if ((bits >> lane) & 1u) {
                const int pos = run + __popc(bits & lanemask_lt());
                if (pos < room) {
                    p.stage_ci[so + pos] = j;
                    ((V *)p.stage_val)[so + pos] = acc[j];
                }
            }
            run += __popc(bits);
        }
        if (lane == 0) {
            p.nnz[g] = run;
            if (run > room) raise_err(p.err, kErrTableFull);
        }
        __syncwarp();
        return;
    }
    if (M.ncols <= p.dense_max) {
        // dense accumulator over the columns of B (values, then the bitmap)
        const int words = (M.ncols + 31) >> 5;
        V *acc = (V *)wtab;
        unsigned *bm = (unsigned *)(wtab + (((size_t)M.ncols * sizeof(V) + 15) & ~(size_t)15));
        for (int w = lane; w < words; w += 32) bm[w] = 0u;
        if (NUM)
            for (int j = lane; j < M.ncols; j += 32) acc[j] = V(0);
        __syncwarp();
        warp_products<V, NUM>(op, ab, ae, p.err, [&](int j, V a, V bkj) {
            if (NUM) atomicAdd(acc + j, a * bkj);
            const unsigned bit = 1u << (j & 31);
            if (!(*(volatile unsigned *)(bm + (j >> 5)) & bit)) atomicOr(bm + (j >> 5), bit);
        });
        __syncwarp();
        if (!NUM) {
            int c = 0;
            for (int w = lane; w < words; w += 32) c += __popc(bm[w]);
            c = warp_sum(c);
            if (lane == 0) p.nnz[g] = c;
        } else {
            int run = 0;
            for (int w = 0; w < words; ++w) {
                const unsigned bits = bm[w];
                const int j = (w << 5) + lane;
                if ((bits >> lane) & 1u) {
                    const int pos = run + __popc(bits & lanemask_lt());
                    if (pos < n_exp) {
                        p.ci_pool[base + c0 + pos] = j;
                        ((V *)p.val_pool)[base + c0 + pos] = acc[j];
                    }
                }
                run += __popc(bits);
            }
            if (lane == 0 && run != n_exp) raise_err(p.err, kErrCountMismatch);
        }
        __syncwarp();
        return;
    }
    // hash table of the warp
    const int tb = table_bits(p.ub[g], p.inv_load);
    const int Tr = 1 << tb;
    int *keys = (int *)wtab;
    V *vals = (V *)(wtab + (size_t)T * 4);
    for (int s = lane; s < Tr; s += 32) {
        keys[s] = kEmpty;
        if (NUM) vals[s] = V(0);
    }
    __syncwarp();
    HashCfg hc = p.hc;
    hc.colbits = colbits(M.ncols);
    int cnt = 0;
    warp_products<V, NUM>(op, ab, ae, p.err, [&](int j, V a, V bkj) {
        bool ins;
        const int h = hash_find_or_insert<false>(keys, tb, hc, j, ins);
        if (h < 0) {
            raise_err(p.err, kErrTableFull);
            return;
        }
        if (NUM) atomicAdd(vals + h, a * bkj);
        cnt += ins ? 1 : 0;
    });
    const int tot = warp_sum(cnt);
    __syncwarp();
    if (!NUM) {
        if (lane == 0) p.nnz[g] = tot;
    } else {
        if (lane == 0 && tot != n_exp) raise_err(p.err, kErrCountMismatch);
        NumOutT<V> out{nullptr, p.ci_pool + base, (V *)p.val_pool + base, 0, nullptr};
        if (tot <= 32) writeout_warp_rank<V>(keys, vals, Tr, tot, n_exp, out, c0);
        else writeout_bitonic<V, 32, kBNT>(keys, vals, Tr, n_exp, out, c0, nullptr);
    }
    __syncwarp();
}

// One big row by the whole block.
template <typename V, bool NUM>
__device__ void block_row(const BatchArgs &p, const BatchMat &M, int64_t g, int64_t r, const BatchSmem<V> &sm,
                          int64_t c0, int n_exp, int64_t base) {
    using G = Group<kBNT, kBNT>;
    const Operands<V> op = mat_ops<V>(M);
    int64_t ab, ae;
    a_row_range(op, r, ab, ae, p.err);
    const int Tall = kBW << p.tw_bits;
    const int tb = table_bits(p.ub[g], p.inv_load);
    const int Tr = 1 << tb;
    int *keys = (int *)sm.tab;
    V *vals = (V *)(sm.tab + (size_t)Tall * 4);
    for (int s = threadIdx.x; s < Tr; s += kBNT) {
        keys[s] = kEmpty;
        if (NUM) vals[s] = V(0);
    }
    __syncthreads();
    HashCfg hc = p.hc;
    hc.colbits = colbits(M.ncols);
    int cnt = 0;
    group_products<V, NUM, kBNT, kBNT>(op, ab, ae, sm.sc, p.err, [&](int j, V a, V bkj) {
        bool ins;
        const int h = hash_find_or_insert<false>(keys, tb, hc, j, ins);
        if (h < 0) {
            raise_err(p.err, kErrTableFull);
            return;
        }
        if (NUM) atomicAdd(vals + h, a * bkj);
        cnt += ins ? 1 : 0;
    });
    const int tot = G::template sum<int>(cnt, sm.sc.red);
    if (!NUM) {
        if (threadIdx.x == 0) p.nnz[g] = tot;
    } else {
        if (threadIdx.x == 0 && tot != n_exp) raise_err(p.err, kErrCountMismatch);
        NumOutT<V> out{nullptr, p.ci_pool + base, (V *)p.val_pool + base, 0, nullptr};
        writeout_bitonic<V, kBNT, kBNT>(keys, vals, Tr, n_exp, out, c0, sm.sc.red);
    }
    __syncthreads();
}

// Work of one phase: the big rows first, one per block (claimed with one
// counter); then every warp claims chunks of 32 consecutive rows of the
// flattened row space on its own (a second counter) and serves the small rows
// among them, with no block-wide wait between rows of unequal cost.
constexpr int kRowChunk = 32;

template <typename V, bool NUM>
__device__ bool run_items(const BatchArgs &p, int *token, int *chunks, const BatchSmem<V> &sm, int nbig) {
    __shared__ long long s_item;
    const int w = threadIdx.x >> 5;
    const int lane = lane_id();
    const size_t wbytes = ((size_t)1 << p.tw_bits) * (4 + sizeof(V));
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(token, 1);
        __syncthreads();
        const long long it = s_item;
        __syncthreads();
        if (it >= nbig) break;
        const int64_t g = p.big[it];
        const int mi = find_mat(p.row_start, p.nmat, g);
        const BatchMat &M = p.mats[mi];
        const int64_t r = g - p.row_start[mi];
        int64_t c0 = 0;
        int n_exp = 0;
        int64_t base = 0;
        if (NUM) {
            const int64_t *rp = p.rp_pool + p.row_start[mi] + mi;
            c0 = rp[r];
            n_exp = (int)(rp[r + 1] - rp[r]);
            base = p.base[mi];
        }
        block_row<V, NUM>(p, M, g, r, sm, c0, n_exp, base);
    }
    // small rows: `chunks` counts the chunks of kRowChunk rows handed out
    unsigned char *wtab = sm.tab + (size_t)w * wbytes;
    for (;;) {
        int ch = 0;
        if (lane == 0) ch = atomicAdd(chunks, 1);
        ch = __shfl_sync(kFull, ch, 0);
        const int64_t g0 = (int64_t)ch * kRowChunk;
        if (g0 >= p.nrows) break;
        const int64_t g1 = g0 + kRowChunk < p.nrows ? g0 + kRowChunk : p.nrows;
        // the small rows of the chunk, one at a time
        const bool mine = g0 + lane < g1 && p.cls[g0 + lane] == kRowSmall;
        for (unsigned todo = __ballot_sync(kFull, mine); todo; todo &= todo - 1) {
            const int64_t g = g0 + __ffs(todo) - 1;
            const int mi = find_mat(p.row_start, p.nmat, g);
            const BatchMat &M = p.mats[mi];
            const int64_t r = g - p.row_start[mi];
            int64_t c0 = 0;
            int n_exp = 0;
            int64_t base = 0;
            if (NUM) {
                const int64_t *rp = p.rp_pool + p.row_start[mi] + mi;
                c0 = rp[r];
                n_exp = (int)(rp[r + 1] - rp[r]);
                base = p.base[mi];
            }
            warp_row<V, NUM>(p, M, g, r, wtab, c0, n_exp, base);
        }
    }
    return true;
}

template <typename V>
__global__ void __launch_bounds__(kBNT) k_batched(const BatchArgs *pp) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_w[32];
    // the arguments live in device memory (a recorded launch is replayed with
    // new arguments copied there)
    __shared__ BatchArgs s_p;
    if (threadIdx.x == 0) s_p = *pp;
    __syncthreads();
    const BatchArgs &p = s_p;
    BatchSmem<V> sm;
    sm.tab = smem;
    const size_t tab_bytes = ((size_t)kBW << p.tw_bits) * (4 + sizeof(V));
    sm.sc = carve_prod_scratch<V, kBNT>(smem + tab_bytes);
    const int nbig = p.counters[0];
    int *bar = p.counters + 6;
    // phase 1: symbolic counts
    run_items<V, false>(p, p.counters + 2, p.counters + 8, sm, nbig);
    if (!grid_barrier(bar, p.err, p.wait_spins, p.missing)) return;
    // phase 2: row pointers of each product (one product per block at a time)
    __shared__ int s_m;
    for (;;) {
        if (threadIdx.x == 0) s_m = atomicAdd(p.counters + 5, 1);
        __syncthreads();
        const int mi = s_m;
        __syncthreads();
        if (mi >= p.nmat) break;
        const int64_t r0 = p.row_start[mi], n = p.row_start[mi + 1] - r0;
        int64_t *rp = p.rp_pool + r0 + mi;
        long long carry = 0;
        for (int64_t b0 = 0; b0 < n; b0 += kBNT) {
            const int64_t i = b0 + threadIdx.x;
            const long long v = i < n ? p.nnz[r0 + i] : 0;
            const long long incl = warp_incl_scan64(v);
            if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
            __syncthreads();
            long long off = carry, tot = 0;
            for (int k = 0; k < kBW; ++k) {
                if (k < (int)(threadIdx.x >> 5)) off += s_w[k];
                tot += s_w[k];
            }
            if (i < n) rp[i] = off + incl - v;
            carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            rp[n] = carry;
            p.totals[mi] = carry;
        }
    }
    if (!grid_barrier(bar, p.err, p.wait_spins, p.missing)) return;
    // phase 3: base offsets of the products in the pools
    if (blockIdx.x == 0) {
        long long carry = 0;
        for (int b0 = 0; b0 < p.nmat; b0 += kBNT) {
            const int i = b0 + threadIdx.x;
            const long long v = i < p.nmat ? p.totals[i] : 0;
            const long long incl = warp_incl_scan64(v);
            if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
            __syncthreads();
            long long off = carry, tot = 0;
            for (int k = 0; k < kBW; ++k) {
                if (k < (int)(threadIdx.x >> 5)) off += s_w[k];
                tot += s_w[k];
            }
            if (i < p.nmat) p.base[i] = off + incl - v;
            carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) p.base[p.nmat] = carry;
    }
    if (!grid_barrier(bar, p.err, p.wait_spins, p.missing)) return;
    // phase 4: values
    run_items<V, true>(p, p.counters + 3, p.counters + 9, sm, nbig);
}

// ---------------------------------------------------------------------------
size_t batched_smem(int dtype, int tw_bits) {
    const size_t vs = dtype ? 8 : 4;
    const size_t sc = dtype ? num_scratch_bytes<double, kBNT>() : num_scratch_bytes<float, kBNT>();
    return ((size_t)kBW << tw_bits) * (4 + vs) + sc;
}

int batched_dense_max(int dtype, int tw_bits) {
    const size_t vs = dtype ? 8 : 4;
    const size_t wbytes = ((size_t)1 << tw_bits) * (4 + vs);
    // values (rounded to 16 bytes) + bitmap must fit one warp's table
    long long c = (long long)((wbytes - 16) * 8 / (8 * vs + 1));
    c &= ~31ll;
    return (int)c;
}

void launch_batch_rowinfo(const BatchArgs &p, int sms, cudaStream_t s) {
    if (p.nrows == 0) return;
    const int64_t blocks = (p.nrows + 7) / 8;
    const int64_t cap = (int64_t)sms * 8;
    k_batch_rowinfo<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(p);
}

int batched_grid(int dtype, int tw_bits, int sms) {
    const size_t smem = batched_smem(dtype, tw_bits);
    int per = 0;
    if (dtype) {
        cudaFuncSetAttribute(k_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batched<double>, kBNT, smem);
    } else {
        cudaFuncSetAttribute(k_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batched<float>, kBNT, smem);
    }
    return per * sms;
}

int launch_batched(int dtype, const BatchArgs *p_dev, int tw_bits, int grid, cudaStream_t s) {
    const size_t smem = batched_smem(dtype, tw_bits);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kBNT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (dtype) e = cudaLaunchKernelEx(&cfg, k_batched<double>, p_dev);
    else e = cudaLaunchKernelEx(&cfg, k_batched<float>, p_dev);
    return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace smash
