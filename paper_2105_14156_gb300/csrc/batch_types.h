// Shared definitions of the batched path (device kernel and host driver).
#pragma once

#include <cstdint>

#include "device_common.cuh"

namespace smash {

constexpr int kBW = 8;                 // warps per block = rows per tile
constexpr int kBNT = kBW * 32;

// Classification of a row.
enum : uint8_t { kRowEmpty = 0, kRowSmall = 1, kRowBig = 2, kRowHuge = 3 };

struct BatchMat {
    const int64_t *a_rp;
    const int32_t *a_ci;
    const void *a_val;
    const int64_t *b_rp;
    const int32_t *b_ci;
    const void *b_val;
    int64_t a_nnz;
    int64_t b_nnz;
    int32_t a_rows;
    int32_t b_rows;
    int32_t ncols;
    int32_t pad;
    int64_t row_off;  // first row of this product in the flattened row space
    int64_t tile_off; // first tile of this product
};

struct BatchArgs {
    const BatchMat *mats;
    int nmat;
    int64_t nrows;          // all products' rows
    int64_t ntiles;
    const int64_t *row_start;   // [nmat+1]
    const int64_t *tile_start;  // [nmat+1]
    uint8_t *cls;           // [nrows]
    int *ub;                // [nrows] min(flop, cols)
    int *nnz;               // [nrows]
    int *big;               // [nrows] list of big rows
    int *huge;              // [nrows] list of huge rows
    int *counters;          // [12]: 0 nbig, 1 nhuge, 2..4 item tokens, 5 matrix token, 6..7 barrier,
                            // 8..9 row-chunk tokens of the two row phases
    unsigned long long *sums;   // [4]: sum ub, sum flop
    int64_t *rp_pool;       // row pointers: product m at row_start[m] + m
    int32_t *ci_pool;
    void *val_pool;
    int64_t *base;          // [nmat+1] first entry of product m in the pools
    int64_t *totals;        // [nmat]
    int *err;
    int tw_bits;            // per-warp table: 2^tw_bits slots
    int warp_bits;          // rows whose table needs at most 2^warp_bits slots: one warp (<= tw_bits)
    int block_bits;         // ... at most 2^block_bits slots: the whole block (<= tw_bits + 3); larger:
                            // the regular per-product path
    int dense_max;          // per-warp dense accumulator when cols <= dense_max
    HashCfg hc;             // colbits filled per product
    float inv_load;
    // dense-accumulator rows in one pass: the first phase computes their values
    // and stages each sorted row at stage_off[g] (room: min(flop, cols)); the
    // last phase copies it to its exact place (null: two passes, as the rest)
    const int64_t *stage_off;
    int32_t *stage_ci;
    void *stage_val;
    long long wait_spins;   // a grid barrier gives up after this many polls (~256 ns each)
    int missing;            // test hook: arrivals a barrier waits for beyond the grid (0: none)
};

size_t batched_smem(int dtype, int tw_bits);
int batched_dense_max(int dtype, int tw_bits);
void launch_batch_rowinfo(const BatchArgs &p, int sms, cudaStream_t s);
int batched_grid(int dtype, int tw_bits, int sms);
// p_dev: the arguments in device memory (read by every block at start).
int launch_batched(int dtype, const BatchArgs *p_dev, int tw_bits, int grid, cudaStream_t s);

}  // namespace smash
