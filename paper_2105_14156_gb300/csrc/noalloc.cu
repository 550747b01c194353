// Symbolic phase that allocates no memory.
//
// Some callers cannot allocate device memory at all: code that runs while a
// memory pool is frozen or owned by another runtime, a process with a hard
// device-memory budget already spent, or a host that may only hand over its
// own input and output buffers. For them, spgemm_symbolic_noalloc computes
// C's row pointer with every scratch byte taken from one fixed array compiled
// into this library (a file-scope __device__ array), so the call performs no
// cudaMalloc, no cudaFree and no allocation by any library.
//
// The kernel is a variant of the global-memory hash of the symbolic phase:
// each block owns a slice of the fixed array as its hash table, counts the
// distinct columns of its rows with compare-and-swap inserts, and writes the
// count of row i to c_row_ptr[i+1]; one block then turns those counts into the
// exclusive prefix sum in place.
#include <atomic>

#include "internal.h"

using namespace smash;
using namespace smash::host;

namespace {

constexpr int kNaBlocks = 64;          // blocks, each owning one table slice
constexpr int kNaTableBits = 17;       // 131072 slots per slice
constexpr int kNaThreads = 512;
constexpr int kNaErrWords = 64;        // error words at the start of the array
constexpr long long kNaMaxCols = 1ll << 16;   // every row fits a slice at load 1/2
constexpr size_t kNaWords = (size_t)kNaErrWords + ((size_t)kNaBlocks << kNaTableBits);

// The scratch: 32 MiB + 256 B, held by every device that loads the library.
static __device__ __align__(256) int g_noalloc_scratch[kNaWords];

// Device address of the scratch per device, looked up once (host code may
// not use the array's name as an address). Atomic entries: two host threads
// that make their first call on a device at the same time both look the
// address up and store the same value, without a data race.
std::atomic<int *> g_scratch_addr[256];

__global__ void __launch_bounds__(kNaThreads) k_na_count(Operands<float> op, int64_t n, HashCfg hc,
                                                         int64_t *c_rp, int *scratch) {
    using G = Group<kNaThreads, kNaThreads>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_f[kNaThreads / 32];
    int *err = scratch;
    int *keys = scratch + kNaErrWords + ((size_t)blockIdx.x << kNaTableBits);
    const ProdScratch<float> sc = carve_prod_scratch<float, kNaThreads>(smem);
    const int t = threadIdx.x;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        int64_t ab, ae;
        a_row_range(op, i, ab, ae, err);
        // product count of the row, for the table size
        long long f = 0;
        for (int64_t e = ab + t; e < ae; e += kNaThreads) {
            const int k = __ldg(op.a_ci + e);
            if ((unsigned)k < (unsigned)op.b_rows) {
                const int64_t s = __ldg(op.b_rp + k), u = __ldg(op.b_rp + k + 1);
                if (s >= 0 && u >= s && u <= op.b_nnz) f += u - s;
            }
        }
        f = warp_sum(f);
        if (lane_id() == 0) s_f[t >> 5] = f;
        __syncthreads();
        long long flop = 0;
        for (int w = 0; w < kNaThreads / 32; ++w) flop += s_f[w];
        const long long bound = flop < (long long)op.ncols ? flop : (long long)op.ncols;
        int tb = table_bits(bound, 2.0f);
        if (tb > kNaTableBits) tb = kNaTableBits;   // unreachable while cols <= kNaMaxCols
        const int T = 1 << tb;
        for (int s = t; s < T; s += kNaThreads) __stcg(keys + s, kEmpty);
        __syncthreads();
        int cnt = 0;
        group_products<float, false, kNaThreads, kNaThreads>(op, ab, ae, sc, err, [&](int j, float, float) {
            bool ins;
            if (hash_find_or_insert<true>(keys, tb, hc, j, ins) < 0) raise_err(err, kErrTableFull);
            cnt += ins ? 1 : 0;
        });
        const int tot = G::template sum<int>(cnt, sc.red);
        if (t == 0) c_rp[i + 1] = tot;
        __syncthreads();
    }
}

// In-place exclusive scan of the counts in c_rp[1..n] (one block).
__global__ void __launch_bounds__(1024) k_na_scan(int64_t *c_rp, int64_t n) {
    __shared__ long long s_w[32];
    long long carry = 0;
    for (int64_t b0 = 0; b0 < n; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const long long v = i < n ? c_rp[i + 1] : 0;
        long long incl = warp_incl_scan64(v);
        if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
        __syncthreads();
        long long off = carry;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) off += s_w[w];
        long long tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_w[w];
        __syncthreads();
        if (i < n) c_rp[i + 1] = off + incl;
        carry += tot;
    }
    if (threadIdx.x == 0) c_rp[0] = 0;
}

}  // namespace

extern "C" {

int spgemm_symbolic_noalloc(const smash_csr *A, const smash_csr *B, int64_t *c_row_ptr, int64_t *c_nnz,
                            void *stream) {
    if (!c_row_ptr || !c_nnz) return SMASH_ERR_INVALID_ARG;
    int st = check_csr(A, false);
    if (st) return st;
    if ((st = check_csr(B, false))) return st;
    if (A->cols != B->rows) return SMASH_ERR_SHAPE_MISMATCH;
    if (B->cols > kNaMaxCols) return SMASH_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SMASH_ERR_CUDA;
    int *scratch = g_scratch_addr[dev].load(std::memory_order_relaxed);
    if (!scratch) {
        // one-time set-up on this device (the device is current)
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SMASH_ERR_CUDA;
        }
        scratch = (int *)p;
        g_scratch_addr[dev].store(scratch, std::memory_order_relaxed);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->rows;
    if (cudaMemsetAsync(c_row_ptr, 0, sizeof(int64_t) * (size_t)(n + 1), s) != cudaSuccess ||
        cudaMemsetAsync(scratch, 0, sizeof(int) * kNaErrWords, s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    if (n > 0 && A->nnz > 0 && B->nnz > 0) {
        Operands<float> op;
        op.a_rp = A->row_ptr;
        op.a_ci = A->col_idx;
        op.a_val = nullptr;
        op.b_rp = B->row_ptr;
        op.b_ci = B->col_idx;
        op.b_val = nullptr;
        op.a_nnz = A->nnz;
        op.b_nnz = B->nnz;
        op.b_rows = (int32_t)B->rows;
        op.ncols = (int32_t)B->cols;
        const HashCfg hc{1, colbits_of(B->cols)};
        const int grid = n < kNaBlocks ? (int)n : kNaBlocks;
        k_na_count<<<grid, kNaThreads, prod_scratch_bytes<float, kNaThreads>(), s>>>(op, n, hc, c_row_ptr, scratch);
        k_na_scan<<<1, 1024, 0, s>>>(c_row_ptr, n);
        if (cudaGetLastError() != cudaSuccess) return SMASH_ERR_CUDA;
    }
    int flags[kNumErr];
    int64_t total = 0;
    if (cudaMemcpyAsync(flags, scratch, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&total, c_row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    *c_nnz = total;
    if (flags[kErrBadIndex] || flags[kErrBadRowPtr]) return SMASH_ERR_INVALID_ARG;
    if (flags[kErrBRowTooLong]) return SMASH_ERR_UNSUPPORTED;
    if (flags[kErrTableFull]) return SMASH_ERR_INTERNAL;
    return SMASH_OK;
}

}  // extern "C"
