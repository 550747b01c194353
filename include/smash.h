/*
 * smash.h -- C ABI of a GB300 (sm_103a) row-wise hash SpGEMM library.
 *
 * Operation: C = A * B for sparse A (m x k) and B (k x n) in CSR, computed
 * row by row (Eq. row_wise: C[i,:] = sum_{k in A_i} A[i,k] * B[k,:]) with the
 * partial products of each row merged as they are produced in an
 * open-addressing hash table (atomic compare-and-swap on the column tag,
 * atomic add on the value), as in the "Hashing Phase" of SMASH Version 1 and
 * the low-order-bit hashing of Version 2.
 *
 * Conventions shared by every call:
 *  - All matrix arrays are DEVICE pointers on the handle's device:
 *    row_ptr int64[rows+1], col_idx int32[nnz], val (float or double)[nnz].
 *  - Input rows may hold unsorted and duplicate column indices; duplicates
 *    are separate terms of the sum. Output rows are sorted ascending with
 *    unique columns. A value that cancels to zero is kept as a stored entry:
 *    the structure of C is every (i, j) reached by at least one product.
 *  - rows == 0 and nnz == 0 are legal. A.cols must equal B.rows.
 *  - Limits: rows, cols < 2^31; every row of B holds fewer than 2^21
 *    entries. Out-of-range indices and malformed row pointers are detected by
 *    the kernels' bounds checks and reported as SMASH_ERR_INVALID_ARG, a row
 *    of B over the limit as SMASH_ERR_UNSUPPORTED; no out-of-range access is
 *    made.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - No C++ exception crosses this interface; every call returns a status.
 *  - The library never frees memory it did not allocate. Scratch memory is
 *    owned by the handle (grown on demand through the handle's allocator).
 *  - A handle is not thread-safe: one host thread per handle at a time.
 *  - Calls that return host values (spgemm_symbolic's nnz, spgemm_learned's
 *    sizes) wait on the call's stream only, and read their small counts back
 *    through mapped pinned memory, not through copies: copies the caller runs
 *    on other streams overlap them instead of delaying them.
 */
#ifndef SMASH_H
#define SMASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    SMASH_OK = 0,
    SMASH_ERR_INVALID_ARG = 1,     /* null pointer, negative size, bad index in the data */
    SMASH_ERR_SHAPE_MISMATCH = 2,  /* A.cols != B.rows, or C's shape is not A.rows x B.cols */
    SMASH_ERR_UNSUPPORTED = 3,     /* dtype or size outside the stated limits */
    SMASH_ERR_ALLOC = 4,           /* the allocator returned NULL */
    SMASH_ERR_CUDA = 5,            /* a CUDA runtime call failed */
    SMASH_ERR_TIMEOUT = 6,         /* a bounded in-kernel wait gave up */
    SMASH_ERR_INTERNAL = 7         /* an internal consistency check failed */
};

typedef enum { SMASH_F32 = 0, SMASH_F64 = 1 } smash_dtype;

/* CSR matrix view. The library reads (A, B) or fills (C) the arrays. */
typedef struct {
    int64_t rows;
    int64_t cols;
    int64_t nnz;
    int64_t *row_ptr; /* device, rows+1 entries, row_ptr[0] = 0, row_ptr[rows] = nnz */
    int32_t *col_idx; /* device, nnz entries */
    void *val;        /* device, nnz entries of the call's dtype (may be NULL in symbolic calls) */
} smash_csr;

/* Tuning parameters. None of them changes the result, only the speed.
 * smash_default_params() fills the defaults; the autotuner overwrites them. */
typedef struct {
    int32_t hash_kind;      /* 0: low-order bits j & (T-1) (Version 2);
                               1: multiplicative (Fibonacci) hashing (default: on R-MAT, whose columns
                                  cluster at small indices, the low-order bits make long probe chains);
                               2: high-order bits j >> shift (Version 1, order preserving) */
    float max_load;         /* table sized to next_pow2(bound / max_load) slots; (0.05, 0.95]; default 0.5 */
    int32_t sym_max_tbits;  /* largest shared-memory symbolic table, log2 slots; [5, 15]; default 15 */
    int32_t num_max_tbits;  /* largest shared-memory numeric table, log2 slots; [5, 14]; default 14 */
    int32_t group_shift;    /* threads per row = clamp(T >> group_shift, 32, 1024); [0, 10]; default 4 */
    int32_t dense_ratio;    /* a row whose bound b satisfies b * dense_ratio >= cols(B) uses the dense
                               accumulator (the paper's "dense row"); 0 disables; default 4 */
    int32_t bitmap_ratio;   /* numeric write-out ranks by a column bitmap when cols(B)/32 <=
                               bitmap_ratio * nnz(row); 0 disables; default 4 */
    int32_t spill_blocks_per_sm; /* resident blocks per SM of the spill and dense kernels; default 1 */
    int32_t sym_dense_ratio; /* symbolic phase: a row whose bound b satisfies b * sym_dense_ratio >= cols(B)
                                counts its columns in a shared-memory bitmap; 0 disables; default 64 */
    int32_t dense_blocks;    /* dense rows: resident blocks per SM of the numeric dense kernel (1, 2 or 4);
                                each owns one column window of a row (the widest that fits its share of
                                shared memory); 0 (default): 2 for float64, 4 for float32 */
    int32_t sym_dense_blocks; /* symbolic dense rows: resident blocks per SM of the bitmap kernel (1, 2, 4
                                 or 8; fewer when their bitmaps do not fit); 0 (default): the most resident
                                 threads, then the most blocks */
    int32_t warp_rows;       /* rows served by one warp (tables of at most 32 << group_shift slots):
                                1 (default): products enumerated from registers, compare-and-swap-first
                                probing, write-out driven by the list of claimed slots;
                                0: the shared-memory staged enumeration of the thread-group kernels */
    int32_t bulk_copy;       /* warp rows: 1 stages each sorted row in shared memory and streams it to C
                                with bulk (TMA engine) copies, Version 3's copy-out; 0 (default): each lane
                                stores its entries (measured faster for rows of a few hundred entries) */
    int32_t group_rows;      /* numeric rows served by a block of 64-1024 threads: 1: the products of a row
                                spread over the block's warps, compare-and-swap-first probing, list-driven
                                write-out (and no table for rows without repeated columns; B with fewer
                                than 2^31 entries, else the default kernel runs); 0 (default): the staged
                                enumeration with a write-out that scans the whole table (measured faster on
                                R-MAT products) */
    int32_t row_window;      /* rows of a bin served together by one warp with one shared-memory table
                                whose tags are (row, column) (the paper's windows of rows): 0 disables,
                                else 2..32 rows per window (fewer where the window would hold more
                                than 256 entries or a tag would not fit 31 bits); default 16 */
    int32_t row_window_tbits; /* row windows take the bins whose per-row table has at most
                                 2^row_window_tbits slots, except the 32-slot bins that the
                                 thread-per-row kernel takes (enough rows: measured faster there);
                                 [5, 8]; default 7 */
    int32_t dense_owner;     /* dense rows: 1: each warp of a block owns a slice of the column window (B is
                                sliced per warp) and adds its products with plain shared-memory updates, lanes
                                that hit one column in the same step taking turns (no atomics; the float add
                                has no native shared-memory atomic on this GPU); 0: atomic adds */
} smash_params;

/* Per-call statistics (the last symbolic or numeric call of the handle). */
typedef struct {
    int64_t rows_per_bin[16]; /* 0: empty rows; 1..12: shared-memory tables of 2^(bin+4) slots;
                                 13: dense accumulator; 14: global-memory hash (spill) */
    int64_t products;         /* sum over rows of the product count flop_i */
    int64_t max_row_products;
    int64_t c_nnz;
    int64_t a_nnz_per_bin[16];    /* sum of nnz(A_i) over the rows of each bin */
    int64_t products_per_bin[16]; /* sum of flop_i over the rows of each bin */
    int64_t c_nnz_per_bin[16];    /* sum of nnz(C_i) (numeric calls; the bound min(flop_i, cols) in
                                     symbolic calls) */
} smash_stats;

/* Accumulated device time of one kernel of the library (event timing). */
typedef struct {
    char name[40];    /* kernel family, e.g. "num_hash", "num_dense_cluster", "sym_hash" */
    int32_t bin;      /* bin served by the launch (-1: not a per-bin kernel) */
    int32_t threads;  /* threads per block */
    int64_t launches;
    int64_t rows;     /* rows of C processed, summed over launches */
    int64_t a_nnz;    /* nnz(A_i) of those rows, summed */
    int64_t products; /* products of those rows, summed */
    int64_t c_nnz;    /* nnz(C_i) (or symbolic bound) of those rows, summed */
    double ms;        /* summed CUDA-event time between launch and completion on the call's stream */
    int64_t kernels;  /* CUDA kernels launched by these launches, summed */
} smash_kernel_time;

typedef struct smash_handle smash_handle;

/* Device allocator: alloc(bytes, ctx) returns a device pointer or NULL;
 * free(ptr, ctx) releases it. Default: cudaMalloc / cudaFree. */
typedef void *(*smash_alloc_fn)(size_t bytes, void *ctx);
typedef void (*smash_free_fn)(void *ptr, void *ctx);

/* Fill *p with the default parameters. */
int smash_default_params(smash_params *p);

/* Create a handle bound to CUDA device `device`. params may be NULL (defaults).
 * Writes the handle to *out. */
int smash_create(smash_handle **out, int device, const smash_params *params);

/* Destroy the handle and release its scratch memory (synchronises the device). */
int smash_destroy(smash_handle *h);

/* Replace / read the tuning parameters. Out-of-range values: SMASH_ERR_INVALID_ARG. */
int smash_set_params(smash_handle *h, const smash_params *params);
int smash_get_params(const smash_handle *h, smash_params *params);

/* Route the handle's scratch allocations through (alloc, free, ctx). Frees
 * the current scratch first (synchronising the device). alloc == NULL restores
 * cudaMalloc / cudaFree. If the new allocator cannot provide the handle's
 * error words, the handle goes back to cudaMalloc / cudaFree and the call
 * returns SMASH_ERR_ALLOC. A call whose allocation fails returns
 * SMASH_ERR_ALLOC and leaves nothing allocated for the caller. */
int smash_set_allocator(smash_handle *h, smash_alloc_fn alloc, smash_free_fn free_fn, void *ctx);

/*
 * Symbolic phase: the number of distinct columns of every row of C = A*B,
 * and C's row pointer. This is the "memory required to allocate the output"
 * count of the Window Distribution Phase, computed exactly with key-only
 * hash tables (Hashing Phase without values).
 *   A, B:       inputs (val unused, may be NULL).
 *   c_row_ptr:  device int64[A.rows+1], caller-allocated; receives the
 *               exclusive prefix sum of the row counts (c_row_ptr[0] = 0).
 *   c_nnz:      host int64*, receives nnz(C).
 * Synchronises `stream` before returning.
 */
int spgemm_symbolic(smash_handle *h, const smash_csr *A, const smash_csr *B, int64_t *c_row_ptr,
                    int64_t *c_nnz, void *stream);

/*
 * Numeric phase: fills C.col_idx and C.val of C = A*B (Hashing Phase with
 * values, then the Write-back Phase: each row's table is compacted, sorted by
 * column and streamed to C).
 *   C: C.rows = A.rows, C.cols = B.cols, C.row_ptr = the symbolic phase's
 *      output, C.nnz = its c_nnz, C.col_idx / C.val caller-allocated device
 *      arrays of C.nnz entries.
 *   dtype: element type of A.val, B.val and C.val.
 * Synchronises `stream` once, after binning the rows, to size its launches.
 * Faults detected by the kernels (bad indices, a row count that does not
 * match C.row_ptr) are returned by the next smash_check() call.
 */
int spgemm_numeric(smash_handle *h, const smash_csr *A, const smash_csr *B, smash_dtype dtype,
                   smash_csr *C, void *stream);

/*
 * Symbolic phase that allocates nothing. The paper has no counterpart; this
 * is for callers that cannot allocate device memory at all (a frozen or
 * foreign-owned memory pool, an exhausted device-memory budget, a host that
 * may only pass in its own buffers) and so cannot even create a handle.
 * Same result as spgemm_symbolic: c_row_ptr (device int64[A.rows+1],
 * caller-allocated) receives C's row pointer and *c_nnz (host) nnz(C).
 * All scratch memory comes from one fixed array inside the library
 * (32 MiB + 256 B of device memory, held on every device that loads the
 * library until the process exits); the call performs no cudaMalloc, no
 * cudaFree and no allocation by any library. Limit: cols(B) <= 65536 (every
 * row's hash table must fit one 131072-slot slice); larger inputs return
 * SMASH_ERR_UNSUPPORTED. Uses the current CUDA device; the first call on a
 * device looks up the array's device address (make that first call before any
 * stream capture). Every call shares the array and leaves its contents
 * behind; calls that overlap on the GPU (other streams, other host threads)
 * race and must not be issued. Synchronises `stream`.
 */
int spgemm_symbolic_noalloc(const smash_csr *A, const smash_csr *B, int64_t *c_row_ptr, int64_t *c_nnz,
                            void *stream);

/* Synchronise `stream` and return the status recorded by the kernels of the
 * handle's previous calls (then clear it). */
int smash_check(smash_handle *h, void *stream);

/* Statistics of the handle's last symbolic or numeric call. */
int smash_get_stats(const smash_handle *h, smash_stats *out);

/* ---------------------------------------------------------------------------
 * Learned sizing. The paper has no counterpart: it sizes output with the exact
 * per-row count of its setup phase. Here a small multilayer perceptron
 * predicts y_i = log(1 + nnz(C_i)) of each row from six features of the row
 * (log1p of nnz(A_i), of flop_i, of the longest and the mean selected row of
 * B, of min(flop_i, cols(B)); and min(flop_i, cols(B)) / cols(B)). Network:
 * x = (f - mean) * inv_std, h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2) with
 * 64 units each, y = w3 . h2 + b3. The prediction sizes hash tables, bins and
 * a staging buffer, so the exact symbolic pass is skipped; any row whose
 * prediction proves too small is recomputed by the exact path, so C is always
 * exact. Parameters: SMASH_MLP_PARAMS floats in the order W1 (64x6,
 * row-major), b1, W2 (64x64, row-major), b2, w3, b3. Inference reads bfloat16
 * copies of the weights and accumulates in fp32; training keeps fp32 master
 * weights and Adam moments, all on the device.
 */
#define SMASH_MLP_PARAMS 4673
#define SMASH_MLP_FEATURES 6

typedef struct smash_model smash_model;

typedef struct {
    int32_t epochs;   /* passes over the data; default 8 */
    int32_t batch;    /* minibatch size; default 4096 */
    float lr;         /* Adam step size; default 2e-3 */
    float beta1, beta2, eps;  /* defaults 0.9, 0.999, 1e-8 */
    float weight_decay;       /* L2 term added to the gradient; default 0 */
    uint64_t seed;    /* sample order */
    int32_t reserved[4];
} smash_train_cfg;

typedef struct {
    int64_t rows;           /* rows of C */
    int64_t overflow_rows;  /* rows recomputed by the exact path */
    int64_t staged_nnz;     /* capacity of the staging buffer (sum of predicted capacities) */
    int64_t c_nnz;          /* nnz(C) */
} smash_learned_stats;

int smash_train_cfg_default(smash_train_cfg *cfg);

/* Create a model with He-initialised weights (seeded) and identity
 * normalisation, on the handle's device. */
int smash_model_create(smash_handle *h, smash_model **out, uint64_t seed);
int smash_model_destroy(smash_model *m);

/* Host copies of the fp32 parameters (SMASH_MLP_PARAMS floats) and of the
 * normalisation (mean[6] then inv_std[6]); either pointer may be NULL. */
int smash_model_get(const smash_model *m, float *params, float *norm);
int smash_model_set(smash_model *m, const float *params, const float *norm);

/* Binary file: 8-byte magic "SMASHMLP", int32 version (1), int32 parameter
 * count, then the parameters and the normalisation as little-endian floats. */
int smash_model_save(const smash_model *m, const char *path);
int smash_model_load(smash_model *m, const char *path);

/* Features of every row of C = A*B (device float[A.rows * 6], row-major). */
int smash_row_features(smash_handle *h, const smash_csr *A, const smash_csr *B, float *feats, void *stream);

/* Training samples of the row-size model from C = A*B, made by the method
 * itself: the exact symbolic phase counts nnz(C_i) of every row; every row
 * with at least one product gives one sample, in row order: its six features
 * (feats, device float[A.rows * 6] of room) and the target log1p(nnz(C_i))
 * (targets, device float[A.rows] of room). *count (host) receives the number
 * of samples written. Synchronises the stream. */
int smash_training_rows(smash_handle *h, const smash_csr *A, const smash_csr *B, float *feats, float *targets,
                        int64_t *count, void *stream);

/* Train on n samples: feats device float[n*6] (raw features as produced by
 * smash_row_features), targets device float[n] (log1p of the exact row
 * counts). The normalisation is set from the data's mean and standard
 * deviation. *final_loss (host, may be NULL) receives the last epoch's mean
 * squared error. Synchronises the stream. */
int smash_mlp_train(smash_handle *h, smash_model *m, const float *feats, const float *targets, int64_t n,
                    const smash_train_cfg *cfg, float *final_loss, void *stream);

/* Mean squared error and its gradient over n samples with the current fp32
 * weights: grad device float[SMASH_MLP_PARAMS], *loss host. Synchronises. */
int smash_mlp_gradient(smash_handle *h, smash_model *m, const float *feats, const float *targets, int64_t n,
                       float *grad, float *loss, void *stream);

/* Predictions y (device float[n]) with the bfloat16 inference weights,
 * fp32 activations and accumulation (CUDA cores). */
int smash_mlp_predict(smash_handle *h, const smash_model *m, const float *feats, int64_t n, float *y,
                      void *stream);

/* The same predictions as computed inside spgemm_learned: layer 2 (64x64) on
 * the tensor cores (bf16 operands, the layer-1 activations rounded to bf16,
 * fp32 accumulation), 32 rows per warp. */
int smash_mlp_predict_tc(smash_handle *h, const smash_model *m, const float *feats, int64_t n, float *y,
                         void *stream);

/*
 * C = A*B with learned sizing. Each row gets a capacity
 * min(ceil((1 + margin) * expm1(y_i)), min(flop_i, cols(B))) from the model;
 * rows are binned and hashed with tables sized by it and written to a staging
 * buffer; rows whose result did not fit are recomputed exactly (symbolic then
 * numeric); finally C is assembled. C->row_ptr, C->col_idx and C->val are
 * allocated through the handle's allocator and owned by the caller (release
 * them with the same allocator); C->rows, cols and nnz are set.
 * m == NULL: the same one-pass pipeline without the network, every row sized
 * by its bound min(flop_i, cols(B)) (margin ignored; no row can overflow).
 * margin > -1 (a negative margin forces under-prediction: a test hook).
 * stats may be NULL. Synchronises the stream.
 */
int spgemm_learned(smash_handle *h, const smash_csr *A, const smash_csr *B, smash_dtype dtype,
                   const smash_model *m, float margin, smash_csr *C, smash_learned_stats *stats, void *stream);

/* Release C's three arrays through the handle's allocator (for C filled by
 * spgemm_learned, or C[0] of spgemm_batched). */
int smash_free_csr(smash_handle *h, smash_csr *C);

/* ---------------------------------------------------------------------------
 * Batched products (not in the paper as such: Version 2's token scheduling
 * applied across many independent products). count pairs (A[m], B[m]) give
 * C[m] = A[m] * B[m]. One cooperative, persistent kernel claims work items
 * (single large rows, then tiles of 8 rows of one product) from a global
 * counter and runs the symbolic counts, the row-pointer scans, the products'
 * offsets and the numeric values, separated by grid barriers whose waits are
 * bounded (a timeout returns SMASH_ERR_TIMEOUT). Rows too large for one
 * block's table (flagged "huge") are computed around the launch by the
 * regular per-product path. The launch is recorded in a CUDA graph and
 * replayed.
 * Output: C[m].rows/cols/nnz are set; the arrays of all C[m] are views into
 * three pools allocated through the handle's allocator and owned by the
 * caller: release them with smash_free_csr(h, &C[0]) only (C[0]'s arrays are
 * the pools' starts). Synchronises the stream.
 */
typedef struct {
    int64_t products;
    int64_t rows;       /* rows of all products */
    int64_t big_rows;   /* rows done by a whole block */
    int64_t huge_rows;  /* rows done by the regular path */
    int64_t flop;       /* products a_ik * b_kj */
    int64_t c_nnz;      /* sum of nnz(C[m]) */
} smash_batched_stats;

int spgemm_batched(smash_handle *h, int count, const smash_csr *A, const smash_csr *B, smash_dtype dtype,
                   smash_csr *C, smash_batched_stats *stats, void *stream);

/* Per-warp hash-table size of the batched kernel, 2^bits slots, bits in [6, 12] (default 10). */
int smash_batched_set_table_bits(smash_handle *h, int bits);
int smash_batched_get_table_bits(smash_handle *h, int *bits);

/* Which rows of a batch one warp serves (tables up to 2^(bits - warp_less)
 * slots, 32 threads per row) and which the whole block serves (up to
 * 2^(bits + block_more) slots, 256 threads per row); larger rows take the
 * regular per-product path. warp_less in [0, 3] (default 0), block_more in
 * [0, 3] (default 3). The autotuner sets them with the table size. */
int smash_batched_set_row_cutoffs(smash_handle *h, int warp_less, int block_more);
int smash_batched_get_row_cutoffs(smash_handle *h, int *warp_less, int *block_more);

/* Bounded waits of the batched kernel: each of its grid barriers polls at
 * most wait_spins times (about 256 ns apart; 0 restores the default of about
 * one second), then records a time-out and the kernel returns, so that the
 * call ends with SMASH_ERR_TIMEOUT and the context stays usable.
 * missing_arrivals (0 or 1) is a test hook: 1 makes every barrier wait for
 * one arrival more than the grid has, so that the waits run out. */
int smash_batched_set_wait(smash_handle *h, int64_t wait_spins, int missing_arrivals);

/* Autotuner: times spgemm_batched on the given batch for each table size that
 * fits (2^8 .. 2^11 slots) combined with the row cutoffs (warp_less 0 or 1,
 * block_more 2 or 3), keeps the fastest in the handle and reports its table
 * size (*best_ms: mean of two timed runs after one warm-up). */
int smash_batched_autotune(smash_handle *h, int count, const smash_csr *A, const smash_csr *B, smash_dtype dtype,
                           int *best_bits, float *best_ms, void *stream);

/* Kernel timing (a tracing aid; not needed for results). With enable != 0,
 * every kernel launch of the following calls is bracketed by CUDA events on
 * the call's stream; the totals accumulate per (kernel, bin) until read.
 * Enabling or disabling clears the totals. */
int smash_set_timing(smash_handle *h, int enable);

/* Synchronise the pending events and copy up to `capacity` per-kernel totals
 * into out[]; *count receives the number of distinct (kernel, bin) entries. */
int smash_get_timings(smash_handle *h, smash_kernel_time *out, int capacity, int *count);

/* Human-readable name of a status code (static string). */
const char *smash_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* SMASH_H */
