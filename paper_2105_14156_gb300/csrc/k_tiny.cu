// Rows with few products (the smallest bins): one thread per row.
//
// A bin's rows all hold at most L distinct columns (L = the bin's table size
// times the maximum load) and at most kTinyFlopPerSlot * T products (rows
// with more products are binned one bin up, see bin_for). For such rows a
// hash table per warp costs hundreds of instructions of set-up, clearing and
// write-out per row while the row has a few dozen products. Here each thread
// merges its row's products (the row-wise product of the SMASH HASHING
// algorithm, with a sorted list in place of its table) into a column-sorted
// list in shared memory by insertion: the list is the row's accumulator and,
// being sorted, also its write-back order (SMASH WRITEBACK), so no separate
// sort is needed. Entry e of thread t's
// list sits at e * NT + t: consecutive threads use consecutive banks.
//
// Every index read from the inputs is checked (error word, never a fault); a
// list that would exceed L raises kErrTableFull in exact mode and marks the
// row as overflowed (row_nnz = -1) in capacity mode, as the hash kernels do.
#include <climits>

#include "device_common.cuh"
#include "kernels.h"
#include "writeout.cuh"

namespace smash {

// Loads of B issued together per thread before their products are merged.
constexpr int kTinyLoads = 8;

// Position at which column j belongs in the sorted list keys[0..n) (stride
// NT): the number of entries smaller than j, searched from the end (products
// of one row of B arrive in increasing column order when B is sorted, so the
// search is short). *hit: keys[pos] == j.
template <int NT>
__device__ __forceinline__ int tiny_find(const int *keys, int n, int j, bool *hit) {
    int q = n;
    int k = INT_MIN;
    while (q > 0 && (k = keys[(q - 1) * NT]) > j) --q;
    *hit = q > 0 && k == j;
    return *hit ? q - 1 : q;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_sym_tiny(Operands<float> op, const int *rows, int count, int L,
                                                 int *nnz_out, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    int *keys = (int *)smem + threadIdx.x;
    for (int r = blockIdx.x * NT + threadIdx.x; r < count; r += gridDim.x * NT) {
        const int i = rows[r];
        int64_t ab, ae;
        a_row_range(op, i, ab, ae, err);
        int n = 0;
        // the next A entry's row of B is located while the current one is merged
        int len_nx = 0;
        int64_t bs_nx = 0;
        if (ab < ae) b_row_of(op, __ldg(op.a_ci + ab), len_nx, bs_nx, err);
        for (int64_t e = ab; e < ae; ++e) {
            const int len = len_nx;
            const int64_t bs = bs_nx;
            len_nx = 0;
            if (e + 1 < ae) b_row_of(op, __ldg(op.a_ci + e + 1), len_nx, bs_nx, err);
            for (int p0 = 0; p0 < len; p0 += kTinyLoads) {
                int jj[kTinyLoads];
#pragma unroll
                for (int u = 0; u < kTinyLoads; ++u) jj[u] = p0 + u < len ? __ldg(op.b_ci + bs + p0 + u) : -1;
#pragma unroll
                for (int u = 0; u < kTinyLoads; ++u) {
                    if (p0 + u >= len) break;
                    const int j = jj[u];
                    if ((unsigned)j >= (unsigned)op.ncols) {
                        raise_err(err, kErrBadIndex);
                        continue;
                    }
                    bool hit;
                    const int q = tiny_find<NT>(keys, n, j, &hit);
                    if (hit) continue;
                    if (n == L) {
                        raise_err(err, kErrTableFull);
                        continue;
                    }
                    for (int x = n; x > q; --x) keys[x * NT] = keys[(x - 1) * NT];
                    keys[q * NT] = j;
                    ++n;
                }
            }
        }
        nnz_out[i] = n;
    }
}

template <typename V, int NT>
__global__ void __launch_bounds__(NT) k_num_tiny(Operands<V> op, const int *rows, int count, int L,
                                                 NumOutT<V> out, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    V *vals = (V *)smem + threadIdx.x;
    int *keys = (int *)(smem + (size_t)L * NT * sizeof(V)) + threadIdx.x;
    for (int r = blockIdx.x * NT + threadIdx.x; r < count; r += gridDim.x * NT) {
        const int i = rows[r];
        int64_t c0;
        int n_exp;
        const bool ok = out_range(out, i, c0, n_exp, err);
        int64_t ab = 0, ae = 0;
        if (ok) a_row_range(op, i, ab, ae, err);
        int n = 0;
        bool over = false;
        int len_nx = 0;
        int64_t bs_nx = 0;
        V a_nx = V(0);
        if (ab < ae) {
            b_row_of(op, __ldg(op.a_ci + ab), len_nx, bs_nx, err);
            a_nx = op.a_val[ab];
        }
        for (int64_t e = ab; e < ae; ++e) {
            const int len = len_nx;
            const int64_t bs = bs_nx;
            const V a = a_nx;
            len_nx = 0;
            if (e + 1 < ae) {
                b_row_of(op, __ldg(op.a_ci + e + 1), len_nx, bs_nx, err);
                a_nx = op.a_val[e + 1];
            }
            for (int p0 = 0; p0 < len; p0 += kTinyLoads) {
                int jj[kTinyLoads];
                V bb[kTinyLoads];
#pragma unroll
                for (int u = 0; u < kTinyLoads; ++u) {
                    jj[u] = p0 + u < len ? __ldg(op.b_ci + bs + p0 + u) : -1;
                    bb[u] = p0 + u < len ? __ldg(op.b_val + bs + p0 + u) : V(0);
                }
#pragma unroll
                for (int u = 0; u < kTinyLoads; ++u) {
                    if (p0 + u >= len) break;
                    const int j = jj[u];
                    if ((unsigned)j >= (unsigned)op.ncols) {
                        raise_err(err, kErrBadIndex);
                        continue;
                    }
                    const V v = a * bb[u];
                    bool hit;
                    const int q = tiny_find<NT>(keys, n, j, &hit);
                    if (hit) {
                        vals[q * NT] += v;
                        continue;
                    }
                    if (n == L) {
                        over = true;
                        continue;
                    }
                    for (int x = n; x > q; --x) {
                        keys[x * NT] = keys[(x - 1) * NT];
                        vals[x * NT] = vals[(x - 1) * NT];
                    }
                    keys[q * NT] = j;
                    vals[q * NT] = v;
                    ++n;
                }
            }
        }
        if (out.row_nnz) {
            // capacity mode: the row fits its range or is redone by the exact path
            over = over || n > n_exp;
            out.row_nnz[i] = over ? -1 : n;
            if (over) continue;
        } else if (over || n != n_exp) {
            raise_err(err, over ? kErrTableFull : kErrCountMismatch);
            continue;
        }
        for (int x = 0; x < n; ++x) {
            __stcs(out.c_ci + (c0 + x), keys[x * NT]);
            __stcs(out.c_val + (c0 + x), vals[x * NT]);
        }
    }
}

// ---------------------------------------------------------------------------
constexpr int kTinyNT = 128;

int tiny_list_len(int tbits, float max_load) {
    const int T = 1 << tbits;
    int L = (int)((double)T * (double)max_load + 0.999999);
    L = (L + 3) & ~3;
    return L < 4 ? 4 : (L > T ? T : L);
}

template <typename K>
static int tiny_grid(K kernel, size_t smem, int sms, int count) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kTinyNT, smem);
    if (per_sm < 1) per_sm = 1;
    const long long want = (count + kTinyNT - 1) / kTinyNT;
    const long long cap = (long long)per_sm * sms;
    return (int)(want < cap ? want : cap);
}

void launch_sym_tiny(const RawOperands &r, const int *rows, int count, int tbits, float max_load, int sms,
                     int *nnz_out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    Operands<float> op;
    op.a_rp = r.a_rp;
    op.a_ci = r.a_ci;
    op.a_val = nullptr;
    op.b_rp = r.b_rp;
    op.b_ci = r.b_ci;
    op.b_val = nullptr;
    op.a_nnz = r.a_nnz;
    op.b_nnz = r.b_nnz;
    op.b_rows = r.b_rows;
    op.ncols = r.ncols;
    const int L = tiny_list_len(tbits, max_load);
    const size_t smem = (size_t)L * kTinyNT * 4;
    auto kern = k_sym_tiny<kTinyNT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<tiny_grid(kern, smem, sms, count), kTinyNT, smem, s>>>(op, rows, count, L, nnz_out, err);
}

template <typename V>
static void num_tiny_typed(const RawOperands &r, const int *rows, int count, int tbits, float max_load, int sms,
                           const NumOut &o, int *err, cudaStream_t s) {
    Operands<V> op;
    op.a_rp = r.a_rp;
    op.a_ci = r.a_ci;
    op.a_val = (const V *)r.a_val;
    op.b_rp = r.b_rp;
    op.b_ci = r.b_ci;
    op.b_val = (const V *)r.b_val;
    op.a_nnz = r.a_nnz;
    op.b_nnz = r.b_nnz;
    op.b_rows = r.b_rows;
    op.ncols = r.ncols;
    const NumOutT<V> out{o.c_rp, o.c_ci, (V *)o.c_val, o.c_nnz, o.row_nnz};
    const int L = tiny_list_len(tbits, max_load);
    const size_t smem = (size_t)L * kTinyNT * (4 + sizeof(V));
    auto kern = k_num_tiny<V, kTinyNT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<tiny_grid(kern, smem, sms, count), kTinyNT, smem, s>>>(op, rows, count, L, out, err);
}

void launch_num_tiny(int dtype, const RawOperands &r, const int *rows, int count, int tbits, float max_load,
                     int sms, const NumOut &out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    if (dtype) num_tiny_typed<double>(r, rows, count, tbits, max_load, sms, out, err, s);
    else num_tiny_typed<float>(r, rows, count, tbits, max_load, sms, out, err, s);
}

}  // namespace smash
