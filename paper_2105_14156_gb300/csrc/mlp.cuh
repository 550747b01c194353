// Row-size predictor shared by its kernels (k_mlp.cu) and the planner of the
// learned path (k_rows.cu): parameter layout, the six row features and the
// forward pass of one row.
//
// Not part of the paper: a multilayer perceptron predicts y_i = log(1 +
// nnz(C_i)) of every output row from six features of the row, so that hash
// tables, bins and C's staging allocation can be sized without the exact
// symbolic pass (rows whose prediction proves too small fall back to the exact
// path). Network: x = (f - mean) * inv_std (6 inputs), h1 = relu(W1 x + b1),
// h2 = relu(W2 h1 + b2) (64 units each), y = w3 . h2 + b3. Parameters are one
// flat float vector W1 (64x6, row-major), b1, W2 (64x64, row-major), b2, w3,
// b3. Inference reads a bfloat16 copy of the weights and accumulates in fp32.
//
// The features of row i are computed from the row pointers alone (the same
// information as the flop count of the Window Distribution Phase):
//   f0 = log1p(nnz(A_i))            f1 = log1p(flop_i)
//   f2 = log1p(max_k |B_k|)         f3 = log1p(flop_i / nnz(A_i))
//   f4 = log1p(min(flop_i, cols))   f5 = min(flop_i, cols) / cols
#pragma once

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "kernels.h"

namespace smash {

constexpr int kHid = 64;
constexpr int kFeat = 6;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kFeat;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid;
static_assert(kOffB3 + 1 == kMlpParams, "parameter layout");

// The six features of a row with na = nnz(A_i) entries, flop_i = f and
// longest selected row of B mx (float arithmetic: a few significant digits
// are all the network needs).
__device__ __forceinline__ void row_features(long long na, long long f, long long mx, long long ncols, float *x) {
    const float fa = (float)na;
    const long long ub = f < ncols ? f : ncols;
    x[0] = log1pf(fa);
    x[1] = log1pf((float)f);
    x[2] = log1pf((float)mx);
    x[3] = log1pf(na > 0 ? (float)f / fa : 0.f);
    x[4] = log1pf((float)ub);
    x[5] = ncols > 0 ? (float)ub / (float)ncols : 0.f;
}

// Shared-memory copy of the inference weights (fp32) laid out for the
// forward passes below: W1 rows padded to 8 with b1 in slot 6, b2, w3, b3 and
// the feature normalisation (mean[6], inv_std[6]); then, for mlp_forward
// only, W2 transposed.
constexpr int kSmW1 = 0;                       // [64][8]
constexpr int kSmB2 = kSmW1 + kHid * 8;
constexpr int kSmW3 = kSmB2 + kHid;
constexpr int kSmB3 = kSmW3 + kHid;
constexpr int kSmNorm = kSmB3 + 4;
constexpr int kSmSmall = kSmNorm + 2 * kFeat;  // end of the part both passes read
constexpr int kSmW2T = kSmSmall;               // [64][64], W2T[v][u] = W2[u][v]
constexpr int kSmFloats = kSmW2T + kHid * kHid;
static_assert(kSmSmall % 4 == 0, "16-byte alignment of W2T and of the bf16 fragments");

// Tensor-core pass (mlp_forward_warp): the part both passes read, then W2 as
// bf16 in the order of the mma B fragments, frag[kt][nt][lane] = {b0, b1}
// (4 x 8 x 32 uint2); then one h1 tile per warp of the block, 32 rows x 64
// bf16 with a row stride of 36 words (conflict-free A-fragment reads).
constexpr int kSmW2Frag = kSmSmall;                   // in 4-byte words
constexpr int kH1Stride = 36;                         // words per row of an h1 tile
constexpr int kSmH1 = kSmW2Frag + 4 * 8 * 32 * 2;
constexpr int kH1Words = 32 * kH1Stride;              // per warp
__host__ __device__ constexpr int mlp_tc_words(int warps) { return kSmH1 + warps * kH1Words; }

__device__ __forceinline__ void load_mlp_small(float *sm, const __nv_bfloat16 *wb, const float *norm) {
    for (int k = threadIdx.x; k < kHid * 8; k += blockDim.x) {
        const int v = k >> 3, c = k & 7;
        sm[kSmW1 + k] = c < kFeat ? __bfloat162float(wb[kOffW1 + v * kFeat + c])
                                  : (c == kFeat ? __bfloat162float(wb[kOffB1 + v]) : 0.f);
    }
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        sm[kSmB2 + k] = __bfloat162float(wb[kOffB2 + k]);
        sm[kSmW3 + k] = __bfloat162float(wb[kOffW3 + k]);
    }
    if (threadIdx.x == 0) sm[kSmB3] = __bfloat162float(wb[kOffB3]);
    if (threadIdx.x < 2 * kFeat) sm[kSmNorm + threadIdx.x] = norm[threadIdx.x];
}

__device__ __forceinline__ void load_mlp(float *sm, const __nv_bfloat16 *wb, const float *norm) {
    load_mlp_small(sm, wb, norm);
    for (int k = threadIdx.x; k < kHid * kHid; k += blockDim.x) {
        const int v = k / kHid, u = k % kHid;
        sm[kSmW2T + k] = __bfloat162float(wb[kOffW2 + u * kHid + v]);
    }
}

// The part both passes read plus W2's B fragments for mlp_forward_warp.
// Fragment (kt, nt) of lane l = 4g + q: b0 = W2[n][k0], W2[n][k0+1] and b1 =
// W2[n][k0+8], W2[n][k0+9] with n = 8 nt + g, k0 = 16 kt + 2q (B[k][n] =
// W2[n][k]).
__device__ __forceinline__ void load_mlp_tc(float *sm, const __nv_bfloat16 *wb, const float *norm) {
    load_mlp_small(sm, wb, norm);
    uint32_t *fr = (uint32_t *)(sm + kSmW2Frag);
    for (int k = threadIdx.x; k < 4 * 8 * 32; k += blockDim.x) {
        const int lane = k & 31, nt = (k >> 5) & 7, kt = k >> 8;
        const int n = nt * 8 + (lane >> 2), k0 = kt * 16 + 2 * (lane & 3);
        const __nv_bfloat16 *row = wb + kOffW2 + n * kHid;
        __nv_bfloat162 lo, hi;
        lo.x = row[k0];
        lo.y = row[k0 + 1];
        hi.x = row[k0 + 8];
        hi.y = row[k0 + 9];
        fr[2 * k] = *(const uint32_t *)&lo;
        fr[2 * k + 1] = *(const uint32_t *)&hi;
    }
}

// y for raw features f (sm: the layout above, 16-byte aligned). The 64
// outputs of layer 2 are accumulated 16 at a time, layer 1 recomputed for
// each group: few registers per thread, so that planning kernels that call
// it keep their occupancy.
__device__ __forceinline__ float mlp_forward(const float *sm, const float *f) {
    float x[kFeat];
#pragma unroll
    for (int c = 0; c < kFeat; ++c) x[c] = (f[c] - sm[kSmNorm + c]) * sm[kSmNorm + kFeat + c];
    float y = sm[kSmB3];
#pragma unroll 1
    for (int g = 0; g < kHid; g += 16) {
        float a[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) a[j] = sm[kSmB2 + g + j];
#pragma unroll 4
        for (int v = 0; v < kHid; ++v) {
            const float4 wa = *(const float4 *)(sm + kSmW1 + v * 8);
            const float4 wc = *(const float4 *)(sm + kSmW1 + v * 8 + 4);
            float h = wc.z;
            h = fmaf(wa.x, x[0], h);
            h = fmaf(wa.y, x[1], h);
            h = fmaf(wa.z, x[2], h);
            h = fmaf(wa.w, x[3], h);
            h = fmaf(wc.x, x[4], h);
            h = fmaf(wc.y, x[5], h);
            h = fmaxf(h, 0.f);
            const float4 *w2 = (const float4 *)(sm + kSmW2T + v * kHid + g);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 ww = w2[q];
                a[4 * q] = fmaf(ww.x, h, a[4 * q]);
                a[4 * q + 1] = fmaf(ww.y, h, a[4 * q + 1]);
                a[4 * q + 2] = fmaf(ww.z, h, a[4 * q + 2]);
                a[4 * q + 3] = fmaf(ww.w, h, a[4 * q + 3]);
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) y = fmaf(sm[kSmW3 + g + j], fmaxf(a[j], 0.f), y);
    }
    return y;
}

// y of the 32 rows of a warp, one per lane (raw features f of the lane's row;
// rows of invalid lanes are computed and discarded). Layer 1 in fp32 on the
// CUDA cores, each lane for its own row, into the warp's h1 tile (bf16);
// layer 2, the 64x64 contraction, on the tensor cores: two 16-row tiles,
// each 4 (k) x 8 (n) mma.m16n8k16 with bf16 operands and fp32 accumulators;
// layer 3 in fp32. Fragment layouts of m16n8k16 (g = lane / 4, q = lane %
// 4): A holds rows g and g + 8 at columns 2q, 2q+1, 2q+8, 2q+9; B holds
// columns (k) 2q, 2q+1, 2q+8, 2q+9 of output n = g; C holds rows g, g + 8 at
// outputs 2q, 2q+1. The caller gives each warp its own tile (kH1Words words).
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *(const uint32_t *)&p;
}

__device__ __forceinline__ void mma_bf16_16816(float *c, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float mlp_forward_warp(const float *sm, const float *f, uint32_t *h1t) {
    const int lane = lane_id();
    const int g = lane >> 2, q = lane & 3;
    float x[kFeat];
#pragma unroll
    for (int c = 0; c < kFeat; ++c) x[c] = (f[c] - sm[kSmNorm + c]) * sm[kSmNorm + kFeat + c];
    // layer 1: this lane's row, two units per word
    uint32_t *myrow = h1t + lane * kH1Stride;
#pragma unroll 4
    for (int v = 0; v < kHid; v += 2) {
        float h[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float4 wa = *(const float4 *)(sm + kSmW1 + (v + e) * 8);
            const float4 wc = *(const float4 *)(sm + kSmW1 + (v + e) * 8 + 4);
            float a = wc.z;
            a = fmaf(wa.x, x[0], a);
            a = fmaf(wa.y, x[1], a);
            a = fmaf(wa.z, x[2], a);
            a = fmaf(wa.w, x[3], a);
            a = fmaf(wc.x, x[4], a);
            a = fmaf(wc.y, x[5], a);
            h[e] = fmaxf(a, 0.f);
        }
        myrow[v >> 1] = pack_bf16(h[0], h[1]);
    }
    __syncwarp();
    const uint2 *fr = (const uint2 *)(sm + kSmW2Frag);
    float y_mine = 0.f;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const uint32_t *r0 = h1t + (mt * 16 + g) * kH1Stride;
        const uint32_t *r1 = r0 + 8 * kH1Stride;
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const int w0 = kt * 8 + q;
            uint32_t a[4];
            a[0] = r0[w0];
            a[1] = r1[w0];
            a[2] = r0[w0 + 4];
            a[3] = r1[w0 + 4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint2 b = fr[(kt * 8 + nt) * 32 + lane];
                mma_bf16_16816(acc[nt], a, b.x, b.y);
            }
        }
        // layer 3 on this lane's outputs 2q, 2q+1 of every n-tile, then the
        // sum over the four lanes of the group
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int u = nt * 8 + 2 * q;
            const float bu0 = sm[kSmB2 + u], bu1 = sm[kSmB2 + u + 1];
            const float wu0 = sm[kSmW3 + u], wu1 = sm[kSmW3 + u + 1];
            y0 = fmaf(wu0, fmaxf(acc[nt][0] + bu0, 0.f), y0);
            y0 = fmaf(wu1, fmaxf(acc[nt][1] + bu1, 0.f), y0);
            y1 = fmaf(wu0, fmaxf(acc[nt][2] + bu0, 0.f), y1);
            y1 = fmaf(wu1, fmaxf(acc[nt][3] + bu1, 0.f), y1);
        }
        y0 += __shfl_xor_sync(kFull, y0, 1);
        y0 += __shfl_xor_sync(kFull, y0, 2);
        y1 += __shfl_xor_sync(kFull, y1, 1);
        y1 += __shfl_xor_sync(kFull, y1, 2);
        // row mt*16 + r sits in lane 4r (r < 8: y0) or 4(r - 8) (y1)
        const int r = lane - mt * 16;
        const float from0 = __shfl_sync(kFull, y0, (r & 7) * 4);
        const float from1 = __shfl_sync(kFull, y1, (r & 7) * 4);
        if (r >= 0 && r < 16) y_mine = r < 8 ? from0 : from1;
    }
    __syncwarp();
    return y_mine + sm[kSmB3];
}

// Capacity of a row from its prediction: clamp(ceil((1+margin) expm1(y)), 1,
// bound); rows with bound 0 get 0.
__device__ __forceinline__ long long cap_of(float y, float margin, long long bound) {
    if (bound <= 0) return 0;
    const float pred = expm1f(fminf(y, 40.f));
    float c = ceilf((1.f + margin) * pred);
    if (!(c >= 1.f)) c = 1.f;
    return c >= (float)bound ? bound : (long long)c;
}

}  // namespace smash
