// Host-side launchers of the SpGEMM kernels (one translation unit each).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace smash {

// Binning rule of one phase: which bin a row of a given size bound goes to.
struct BinRule {
    float inv_load;     // 1 / max_load
    int max_tbits;      // largest shared-memory table (log2 slots)
    int dense_ok;       // dense accumulator allowed (column bitmap fits shared memory)
    int64_t dense_min;  // size >= dense_min goes dense (when dense_ok)
    int tiny_tbits;     // bins of tables up to 2^tiny_tbits slots run one thread per row
};

// Raw device view of a CSR operand pair (values as void*).
struct RawOperands {
    const int64_t *a_rp;
    const int32_t *a_ci;
    const void *a_val;
    const int64_t *b_rp;
    const int32_t *b_ci;
    const void *b_val;
    int64_t a_rows;
    int64_t a_nnz;
    int64_t b_nnz;
    int32_t b_rows;
    int32_t ncols;
};

struct BinBuffers {
    uint8_t *bin;      // [n]
    int *counts;       // [16]  rows per bin
    int *cursor;       // [16]  scatter cursors
    int *tokens;       // [16]  work tokens (row claims) per bin
    long long *maxsize;  // [16] largest size bound per bin
    long long *stats;    // [4]  products, max row products
    int *rows;         // [n]   row ids grouped by bin
    int *offsets;      // [17]  exclusive offsets of the bins in rows[]
    long long *sums;   // [3][16] per bin: sum nnz(A_i), sum flop_i, sum size bound
};

// Per-row counts of the planning passes.
struct RowGather {
    long long f;   // flop_i
    int na;        // nnz(A_i)
    int mx;        // longest selected row of B
};
// k_rows.cu. With row_list != nullptr only the listed rows are planned (the
// caller clears bb.bin first so that the other rows stay in the empty bin).
// keep != nullptr: the symbolic planning also records every planned row's
// counts there; kept != nullptr: the numeric planning reads them instead of
// gathering from B again.
void launch_sym_rowinfo(const RawOperands &op, const BinRule &rule, BinBuffers bb, long long *bound_out,
                        int *nnz_out, int *err, int sms, cudaStream_t s, const int *row_list = nullptr,
                        int64_t list_n = 0, RowGather *keep = nullptr);
void launch_num_rowinfo(const RawOperands &op, const int64_t *c_rp, int64_t c_nnz, const BinRule &rule,
                        BinBuffers bb, int *err, int sms, cudaStream_t s, const int *row_list = nullptr,
                        int64_t list_n = 0, const RowGather *kept = nullptr);
// Learned planning (k_rows.cu): features, the predictor and each row's
// capacity cap_i (mlp.cuh) in the planning passes; rows binned by cap_i.
// Two passes: the rows' flop counts and longest rows of B (gather, one row
// per thread, long rows per warp), then the predictor on the tensor cores
// and the bins.
struct LearnArgs {
    const void *wb = nullptr;     // bf16 weights (device)
    const float *norm = nullptr;  // mean[6], inv_std[6] (device)
    float margin = 0.f;
    int *cap = nullptr;           // out: capacity per row
    RowGather *gather = nullptr;  // scratch: one per row
};
void launch_learned_gather(const RawOperands &op, const BinRule &rule, BinBuffers bb, const LearnArgs &la,
                           int *err, int sms, cudaStream_t s);
void launch_learned_bin(const RawOperands &op, const BinRule &rule, BinBuffers bb, const LearnArgs &la, int sms,
                        cudaStream_t s);
// Learned path helpers (k_rows.cu): rows with row_nnz < 0 -> list; copy the
// staged rows that fitted into C.
void launch_overflow_list(const int *row_nnz, int64_t n, int *list, int *count, uint8_t *ovf, cudaStream_t s);
// Bytes of the chunk table launch_compact_rows takes for a C of c_nnz entries.
size_t compact_table_bytes(int64_t c_nnz);
// table: compact_table_bytes(c_nnz) bytes of scratch for the block copy (most
// rows staged), or null for the row walk (long stretches of C written
// elsewhere: the arena's rows).
void launch_compact_rows(int dtype, int64_t n, const int64_t *stage_rp, const uint8_t *ovf, const int32_t *stage_ci,
                         const void *stage_val, const int64_t *c_rp, int32_t *c_ci, void *c_val, int64_t c_nnz,
                         int *table, int sms, cudaStream_t s);

// k_mlp.cu: row-size predictor (see the file for the network).
constexpr int kMlpParams = 4673;
void launch_features(const RawOperands &op, const int *row_list, int64_t nrows, float *feats, long long *bound,
                     int *err, int sms, cudaStream_t s);
void launch_mlp_infer(const float *feats, const long long *bound, const int *row_list, int64_t nrows,
                      const void *wb, const float *norm, float margin, float *y_out, int *cap_out, int sms,
                      cudaStream_t s);
// Tensor-core forward (mlp_forward_warp) of n rows of raw features.
void launch_mlp_infer_tc(const float *feats, int64_t n, const void *wb, const float *norm, float *y, int sms,
                         cudaStream_t s);
void launch_mlp_grad(const float *feats, const float *targets, int64_t n, int64_t first, int64_t count,
                     unsigned long long mul, const unsigned long long *shift, const float *params, const float *norm,
                     float *grad, float *loss_acc, int sms, cudaStream_t s);
void launch_adam(float *params, float *grad, float *m, float *v, void *wb, float lr, float b1, float b2, float eps,
                 float wd, unsigned long long *stepc, cudaStream_t s);
void launch_epoch_shift(unsigned long long *epoch, unsigned long long *shift, unsigned long long seed,
                        unsigned long long n, cudaStream_t s);
void launch_feat_stats(const float *feats, int64_t n, double *acc, int sms, cudaStream_t s);
// Training samples (k_mlp.cu): the rows with bound > 0, in order: features
// from ftmp and target log1p(nnz[i]); *total receives their number.
void launch_training_rows(int64_t n, const int *nnz, const long long *bound, const float *ftmp, int *keep,
                          int64_t *pos, long long *total, void *scan, float *feats, float *targets, int sms,
                          cudaStream_t s);
void launch_to_bf16(const float *src, void *dst, int n, cudaStream_t s);
void launch_bin_scatter(int64_t n, BinBuffers bb, cudaStream_t s);
size_t scan_scratch_bytes(int64_t n);
void launch_scan_rowptr(const int *nnz, int64_t n, int64_t *c_rp, long long *total,
                        void *scratch, cudaStream_t s);

struct HashLaunch {
    int tbits;          // table size 2^tbits
    int group_shift;    // threads per row = clamp(T >> shift, 32, 1024)
    int hash_kind;
    int colbits;
    int sms;
    int blocks_per_sm;  // for the spill kernels
    int dense_blocks;   // resident blocks per SM of the numeric dense kernel
    int sym_dense_blocks;  // of the bitmap (symbolic dense) kernel; 0: automatic
};

// Distinct columns of the dense rows, counted per block of kSubCols columns
// (the numeric dense kernel places each column window's outputs with them).
// wslot[i]: slot of row i (-1: not counted); wcnt[slot][nsub]: the counts.
constexpr int kSubCols = 4096;
struct WinCount {
    int *wslot = nullptr;
    uint16_t *wcnt = nullptr;
    int nsub = 0;
    int64_t slot_base = 0;   // slot of the r-th listed row = slot_base + r
    int skip_slotted = 0;    // rows that already have a slot are not counted again
};
// Size check of a numeric count pass: exact (row length of c_rp must equal
// the count) or capacity mode (row_nnz[i] = count, or -1 when it exceeds the
// row's capacity).
struct NumCheck {
    const int64_t *c_rp = nullptr;
    int64_t c_nnz = 0;
    int *row_nnz = nullptr;
};

// k_symbolic.cu
void launch_sym_hash(const RawOperands &op, const int *rows, int count, int *token, const HashLaunch &hl,
                     int *nnz_out, int *err, cudaStream_t s);
// Dense rows: bitmap over all columns of B. Symbolic use: nnz_out != nullptr.
// Numeric count pass: nnz_out == nullptr, sizes checked by nc.
void launch_sym_dense(const RawOperands &op, const int *rows, int count, int *token, const HashLaunch &hl,
                      const WinCount &wc, int *nnz_out, const NumCheck &nc, int *err, cudaStream_t s);
int sym_dense_threads(const HashLaunch &hl, int64_t ncols);   // block size launch_sym_dense picks
int sym_spill_grid(const HashLaunch &hl);
void launch_sym_spill(const RawOperands &op, const int *rows, int count, int *token, const HashLaunch &hl,
                      float inv_load, const long long *bound, int spill_tbits, int *tables, int *nnz_out,
                      int *err, cudaStream_t s);

// k_numeric.cu (dtype: 0 float, 1 double)
struct NumOut {
    const int64_t *c_rp;
    int32_t *c_ci;
    void *c_val;
    int64_t c_nnz;
    int *row_nnz = nullptr;  // capacity mode (learned sizing) when set, see k_numeric.cu
};
// Copy of `bytes` (a multiple of 4) of device memory into mapped host memory
// by a kernel (k_rows.cu).
void launch_read_small(const void *src, void *dst_mapped, size_t bytes, cudaStream_t s);
// rec (may be null): per-row product counts; rows with nothing to merge
// (exact mode) or whose products fit their room (capacity mode) skip the table.
void launch_num_hash(int dtype, const RawOperands &op, const int *rows, int count, int *token,
                     const HashLaunch &hl, float inv_load, int bitmap_ratio, const RowGather *rec, const NumOut &out,
                     int *err, cudaStream_t s);
// Warp rows (k_warp.cuh): one warp per row, products enumerated from
// registers, compare-and-swap-first probing, list-driven write-out. The
// *_smem functions give the dynamic shared memory of one block.
size_t sym_warp_smem(int tbits);
size_t num_warp_smem(int dtype, int tbits, float inv_load);
void launch_sym_warp(const RawOperands &op, const int *rows, int count, int *token, const HashLaunch &hl,
                     int *nnz_out, int *err, cudaStream_t s);
// rec (may be null): per-row counts kept by the symbolic phase; rows whose
// exact length equals their product count skip the table.
// bulk_copy: stream sorted rows to C by bulk copies from shared memory.
void launch_num_warp(int dtype, const RawOperands &op, const int *rows, int count, int *token,
                     const HashLaunch &hl, float inv_load, const RowGather *rec, int bulk_copy, const NumOut &out,
                     int *err, cudaStream_t s);
// Group rows (k_group.cuh): a block of 64-1024 threads per row, the numeric
// phase of the warp rows spread over the block's warps.
size_t num_group_smem(int dtype, int tbits, float inv_load, int group_shift);
void launch_num_group(int dtype, const RawOperands &op, const int *rows, int count, int *token,
                      const HashLaunch &hl, float inv_load, const RowGather *rec, const NumOut &out, int *err,
                      cudaStream_t s);
// Row windows (k_rowwin.cu): a warp serves a window of W consecutive rows of
// a bin with one shared-memory table whose tags are (row of the window,
// column). Built by host::row_window_of.
struct RowWin {
    int W;      // rows per window (2..32)
    int wbits;  // bits of a row of the window: W <= 2^wbits
    int cb;     // bits of a column: tag = (row << cb) | column, cb + wbits <= 31
    int tbits;  // the window's hash table holds 2^tbits slots
    int ts;     // slots of the table region (>= 2 lcap: the write-out's sorted sequence)
    int lcap;   // most entries a window holds (W times the bin's row room, multiple of 32, <= 256)
    int nb;     // buckets of the write-out (2^(tbits-1))
    int bsh;    // bucket of a tag: tag >> bsh
};
size_t sym_rowwin_smem(const RowWin &rw);
size_t num_rowwin_smem(const RowWin &rw, int dtype);
void launch_sym_rowwin(const RawOperands &op, const int *rows, int count, int *token, const RowWin &rw,
                       const HashLaunch &hl, int *nnz_out, int *err, cudaStream_t s);
// rec (may be null): per-row product counts; a window whose rows have no
// repeated column (exact mode) or fit their capacities (capacity mode) is
// staged without the table.
void launch_num_rowwin(int dtype, const RawOperands &op, const int *rows, int count, int *token, const RowWin &rw,
                       const HashLaunch &hl, const RowGather *rec, const NumOut &out, int *err, cudaStream_t s);
// Thread-per-row bins (tbits <= BinRule::tiny_tbits, k_tiny.cu): list length of a bin, and
// the symbolic count / numeric merge of its rows.
int tiny_list_len(int tbits, float max_load);
void launch_sym_tiny(const RawOperands &op, const int *rows, int count, int tbits, float max_load, int sms,
                     int *nnz_out, int *err, cudaStream_t s);
void launch_num_tiny(int dtype, const RawOperands &op, const int *rows, int count, int tbits, float max_load,
                     int sms, const NumOut &out, int *err, cudaStream_t s);
// Column windows of the dense rows (k_split.cu): slices of B regrouped by
// window of cpc columns; woff[B.rows][nslices+1] (nslices > 1 only).
struct BSlices {
    int nslices = 0;
    int cpc = 0;        // columns of a window
    int per_win = 1;    // slices per window (> 1: one per warp, owner computes; nslices = windows * per_win)
    const int32_t *woff = nullptr;
    const int32_t *ci = nullptr;
    const void *val = nullptr;
};
size_t window_plan_bytes(const RawOperands &op, int nw, size_t vsz);
// Most slices of B the slicing pass supports.
int window_plan_max_slices();
// host_word: pinned, mapped host int (the sortedness of B is read back),
// host_word_dev: the same int as the kernels see it. Returns the number of
// kernels launched.
// nw windows of cpc columns, per slices per window (1: the window itself).
int launch_window_plan(int dtype, const RawOperands &op, int nw, int per, int cpc, void *ws, BSlices &sl, int sms,
                       cudaStream_t s, int *host_word, int *host_word_dev);
// Widest column window (a multiple of kSubCols, at most kMaxWinCols) of the
// numeric dense kernel at `blocks_per_sm` resident blocks per SM; 0: none.
constexpr int kMaxWinCols = 65536;
int num_window_cols(int dtype, int blocks_per_sm, bool own);
// Warps of a block of the numeric dense kernel at blocks_per_sm blocks per SM.
int window_warps(int blocks_per_sm);
// Arena mode of the dense kernel (learned path, capacity mode): no counts;
// each (row, window) item reserves room for its columns in one arena by an
// atomic add on *top, writes them there in order and records (offset, count)
// in desc_off / desc_cnt[item]; out.row_nnz[i] accumulates the row's total,
// or gets its sign bit set when the arena ran out (the row falls back).
struct WinArena {
    unsigned long long *top = nullptr;
    int64_t cap = 0;            // entries
    int32_t *ci = nullptr;
    void *val = nullptr;
    int64_t *desc_off = nullptr;
    int *desc_cnt = nullptr;
};
// (row, window) work items of the dense rows; counts from wc (or arena mode
// when ar.ci != nullptr); token: a 64-bit item counter (zeroed here).
void launch_num_window(int dtype, const RawOperands &op, const int *rows, int count, unsigned long long *token,
                       const HashLaunch &hl, const BSlices &sl, const WinCount &wc, const WinArena &ar,
                       const NumOut &out, int *err, cudaStream_t s);
// Copies the arena rows (ovf[i] == 2) of the dense bin into C.
void launch_arena_compact(int dtype, const int *rows, int count, int nw, const WinArena &ar, const uint8_t *ovf,
                          const int64_t *c_rp, int32_t *c_ci, void *c_val, int sms, cudaStream_t s);
// ovf[i] = 2 for the listed rows with row_nnz[i] >= 0.
void launch_mark_rows(const int *rows, int count, const int *row_nnz, uint8_t *ovf, cudaStream_t s);
// a[rows[r]] = 0 for r < count.
void launch_zero_rows(const int *rows, int count, int *a, cudaStream_t s);
int num_spill_grid(int dtype, const HashLaunch &hl);
void launch_num_spill(int dtype, const RawOperands &op, const int *rows, int count, int *token,
                      const HashLaunch &hl, float inv_load, int spill_tbits, void *tables,
                      const NumOut &out, int *err, cudaStream_t s);

// Shared-memory limits used by the planner.
int max_smem_per_block();
int max_smem_per_sm();
int dense_bitmap_max_cols();          // widest B whose column bitmap fits one block
bool num_hash_bitmap_fits(int dtype, int tbits, int ncols);

}  // namespace smash
