// Row-size predictor: features, inference and training kernels (the network
// and its features are described in mlp.cuh). Training keeps fp32 master
// weights and Adam moments; inference reads the bf16 copy.
#include <cuda_bf16.h>

#include "device_common.cuh"
#include "kernels.h"
#include "mlp.cuh"

namespace smash {

// One warp per row (all rows, or the rows of a list).
__global__ void __launch_bounds__(256) k_features(RawOperands op, const int *row_list, int64_t nrows, float *feats,
                                                  long long *bound, int *err) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += warps) {
        const int64_t i = row_list ? row_list[r] : r;
        int64_t ab = __ldg(op.a_rp + i), ae = __ldg(op.a_rp + i + 1);
        if (ab < 0 || ae < ab || ae > op.a_nnz) {
            if (lane == 0) raise_err(err, kErrBadRowPtr);
            ab = ae = 0;
        }
        long long f = 0, mx = 0;
        for (int64_t e = ab + lane; e < ae; e += 32) {
            const int k = __ldg(op.a_ci + e);
            if ((unsigned)k < (unsigned)op.b_rows) {
                const int64_t s = __ldg(op.b_rp + k), t = __ldg(op.b_rp + k + 1);
                if (s >= 0 && t >= s && t <= op.b_nnz) {
                    f += t - s;
                    mx = (t - s) > mx ? (t - s) : mx;
                }
            }
        }
        f = warp_sum(f);
        mx = warp_max(mx);
        if (lane == 0) {
            row_features(ae - ab, f, mx, op.ncols, feats + (size_t)i * kFeat);
            if (bound) bound[i] = f < (long long)op.ncols ? f : (long long)op.ncols;
        }
    }
}

// Inference: one thread per row. cap_i = cap_of(y_i, margin, bound_i).
// Weights: bf16 in global memory, fp32 in shared.
__global__ void __launch_bounds__(256) k_mlp_infer(const float *feats, const long long *bound, const int *row_list,
                                                   int64_t nrows, const __nv_bfloat16 *wb, const float *norm,
                                                   float margin, float *y_out, int *cap_out) {
    __shared__ __align__(16) float sm[kSmFloats];
    load_mlp(sm, wb, norm);
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride) {
        const int64_t i = row_list ? row_list[r] : r;
        float f[kFeat];
#pragma unroll
        for (int c = 0; c < kFeat; ++c) f[c] = feats[(size_t)i * kFeat + c];
        const float y = mlp_forward(sm, f);
        if (y_out) y_out[r] = y;
        if (cap_out) cap_out[i] = (int)cap_of(y, margin, bound[i]);
    }
}

// Inference with layer 2 on the tensor cores: one warp per 32 rows.
__global__ void __launch_bounds__(256) k_mlp_infer_tc(const float *feats, int64_t nrows, const __nv_bfloat16 *wb,
                                                      const float *norm, float *y_out) {
    extern __shared__ __align__(16) float s_mlp[];
    load_mlp_tc(s_mlp, wb, norm);
    __syncthreads();
    const int lane = lane_id();
    uint32_t *h1t = (uint32_t *)(s_mlp + kSmH1) + (threadIdx.x >> 5) * kH1Words;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < nrows;
         base += warps * 32) {
        const int64_t r = base + lane;
        float f[kFeat];
#pragma unroll
        for (int c = 0; c < kFeat; ++c) f[c] = r < nrows ? feats[(size_t)r * kFeat + c] : 0.f;
        const float y = mlp_forward_warp(s_mlp, f, h1t);
        if (r < nrows) y_out[r] = y;
    }
}

// Training: loss and gradient of a minibatch, TILE samples per block.
// Sample s of minibatch step uses data index perm(base + s) with
// perm(q) = (a*q + c) mod n, a coprime with n (a fresh c per epoch).
constexpr int kTile = 64;

struct Batch {
    int64_t n;          // data size
    int64_t first;      // first position of this minibatch in the epoch's order
    int64_t count;      // samples in the minibatch
    unsigned long long mul;  // a
    const unsigned long long *shift;  // c (device, per epoch); nullptr: 0
    float scale;        // 1 / count (the mean of the squared errors)
};

__global__ void __launch_bounds__(kTile) k_mlp_grad(const float *feats, const float *targets, Batch bt,
                                                    const float *params, const float *norm, float *grad,
                                                    float *loss_acc) {
    extern __shared__ __align__(16) float sm[];
    float *w = sm;                                  // kMlpParams
    float *sh1 = w + ((kMlpParams + 3) & ~3);       // [kHid][kTile]
    float *sh2 = sh1 + kHid * kTile;                // [kHid][kTile]
    float *sdh2 = sh2 + kHid * kTile;               // [kHid][kTile]
    float *sdh1 = sdh2 + kHid * kTile;              // [kHid][kTile]
    float *sx = sdh1 + kHid * kTile;                // [kFeat][kTile]
    float *sdy = sx + kFeat * kTile;                // [kTile]
    __shared__ float nm[2 * kFeat];
    const int t = threadIdx.x;
    for (int k = t; k < kMlpParams; k += kTile) w[k] = params[k];
    if (t < 2 * kFeat) nm[t] = norm[t];
    __syncthreads();
    const unsigned long long c = bt.shift ? *bt.shift : 0ull;
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < bt.count; base += (int64_t)gridDim.x * kTile) {
        const int64_t q = base + t;
        const bool valid = q < bt.count;
        float x[kFeat];
        float tgt = 0.f;
        if (valid) {
            const unsigned long long pos = (unsigned long long)(bt.first + q);
            const int64_t idx = (int64_t)((bt.mul * (pos % (unsigned long long)bt.n) + c) %
                                          (unsigned long long)bt.n);
#pragma unroll
            for (int k = 0; k < kFeat; ++k) x[k] = (feats[(size_t)idx * kFeat + k] - nm[k]) * nm[kFeat + k];
            tgt = targets[idx];
        } else {
#pragma unroll
            for (int k = 0; k < kFeat; ++k) x[k] = 0.f;
        }
        // forward
        float h1[kHid];
#pragma unroll
        for (int u = 0; u < kHid; ++u) {
            float a = w[kOffB1 + u];
#pragma unroll
            for (int k = 0; k < kFeat; ++k) a = fmaf(w[kOffW1 + u * kFeat + k], x[k], a);
            h1[u] = fmaxf(a, 0.f);
            sh1[u * kTile + t] = h1[u];
        }
        float y = w[kOffB3];
        for (int u = 0; u < kHid; ++u) {
            float a = w[kOffB2 + u];
#pragma unroll
            for (int v = 0; v < kHid; ++v) a = fmaf(w[kOffW2 + u * kHid + v], h1[v], a);
            const float h = fmaxf(a, 0.f);
            sh2[u * kTile + t] = h;
            y = fmaf(w[kOffW3 + u], h, y);
        }
        const float r = valid ? (y - tgt) : 0.f;
        const float dy = 2.f * r * bt.scale;
        sdy[t] = dy;
        float lsum = warp_sum(r * r * bt.scale);
        if (lane_id() == 0 && loss_acc) atomicAdd(loss_acc, lsum);
        // backward through layer 2 and 1 (per sample)
        for (int u = 0; u < kHid; ++u) sdh2[u * kTile + t] = sh2[u * kTile + t] > 0.f ? dy * w[kOffW3 + u] : 0.f;
        for (int v = 0; v < kHid; ++v) {
            float a = 0.f;
            for (int u = 0; u < kHid; ++u) a = fmaf(w[kOffW2 + u * kHid + v], sdh2[u * kTile + t], a);
            sdh1[v * kTile + t] = h1[v] > 0.f ? a : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kFeat; ++k) sx[k * kTile + t] = x[k];
        __syncthreads();
        // parameter gradients: sums over the tile's samples
        for (int p = t; p < kHid * kHid; p += kTile) {
            const int u = p / kHid, v = p % kHid;
            float a = 0.f;
            for (int s = 0; s < kTile; ++s) a = fmaf(sdh2[u * kTile + s], sh1[v * kTile + s], a);
            atomicAdd(grad + kOffW2 + p, a);
        }
        for (int p = t; p < kHid * kFeat; p += kTile) {
            const int u = p / kFeat, k = p % kFeat;
            float a = 0.f;
            for (int s = 0; s < kTile; ++s) a = fmaf(sdh1[u * kTile + s], sx[k * kTile + s], a);
            atomicAdd(grad + kOffW1 + p, a);
        }
        {
            const int u = t;   // kTile == kHid
            float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f;
            for (int s = 0; s < kTile; ++s) {
                gb1 += sdh1[u * kTile + s];
                gb2 += sdh2[u * kTile + s];
                gw3 = fmaf(sdy[s], sh2[u * kTile + s], gw3);
            }
            atomicAdd(grad + kOffB1 + u, gb1);
            atomicAdd(grad + kOffB2 + u, gb2);
            atomicAdd(grad + kOffW3 + u, gw3);
        }
        if (t < 32) {
            float g = sdy[t] + sdy[t + 32];
            g = warp_sum(g);
            if (t == 0) atomicAdd(grad + kOffB3, g);
        }
        __syncthreads();
    }
}

// Adam step on all parameters (then the gradient is cleared and the bf16 copy refreshed).
__global__ void __launch_bounds__(256) k_adam(float *params, float *grad, float *m, float *v, __nv_bfloat16 *wb,
                                              float lr, float b1, float b2, float eps, float wd,
                                              const unsigned long long *stepc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const float step = (float)(*stepc + 1);
    if (p < kMlpParams) {
        const float g = grad[p] + wd * params[p];
        const float mm = b1 * m[p] + (1.f - b1) * g;
        const float vv = b2 * v[p] + (1.f - b2) * g * g;
        m[p] = mm;
        v[p] = vv;
        const float mh = mm / (1.f - powf(b1, step));
        const float vh = vv / (1.f - powf(b2, step));
        const float w = params[p] - lr * mh / (sqrtf(vh) + eps);
        params[p] = w;
        wb[p] = __float2bfloat16(w);
        grad[p] = 0.f;
    }
}

__global__ void k_counter_add(unsigned long long *c, unsigned long long d) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *c += d;
}

// Per-epoch permutation shift: c_e = splitmix(seed, epoch) mod n.
__global__ void k_epoch_shift(unsigned long long *epoch, unsigned long long *shift, unsigned long long seed,
                              unsigned long long n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned long long z = seed + (*epoch + 1ull) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        *shift = n ? z % n : 0ull;
        *epoch += 1ull;
    }
}

// Feature statistics: sums and sums of squares per feature (double).
__global__ void __launch_bounds__(256) k_feat_stats(const float *feats, int64_t n, double *acc) {
    double s[kFeat], q[kFeat];
#pragma unroll
    for (int k = 0; k < kFeat; ++k) s[k] = q[k] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
#pragma unroll
        for (int k = 0; k < kFeat; ++k) {
            const double x = feats[(size_t)i * kFeat + k];
            s[k] += x;
            q[k] += x * x;
        }
#pragma unroll
    for (int k = 0; k < kFeat; ++k) {
        s[k] = warp_sum(s[k]);
        q[k] = warp_sum(q[k]);
        if (lane_id() == 0) {
            atomicAdd(acc + k, s[k]);
            atomicAdd(acc + kFeat + k, q[k]);
        }
    }
}

// ---------------------------------------------------------------------------
// Training samples: rows with at least one product (bound > 0), in row
// order; the target of a row is log1p of its exact count.
__global__ void k_keep_rows(int64_t n, const long long *bound, int *keep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keep[i] = bound[i] > 0 ? 1 : 0;
}

__global__ void k_training_rows(int64_t n, const int *nnz, const int *keep, const int64_t *pos, const float *ftmp,
                                float *feats, float *targets) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && keep[i]) {
        const int64_t p = pos[i];
#pragma unroll
        for (int c = 0; c < kFeat; ++c) feats[p * kFeat + c] = ftmp[i * kFeat + c];
        targets[p] = log1pf((float)nnz[i]);
    }
}

void launch_training_rows(int64_t n, const int *nnz, const long long *bound, const float *ftmp, int *keep,
                          int64_t *pos, long long *total, void *scan, float *feats, float *targets, int sms,
                          cudaStream_t s) {
    (void)sms;
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_keep_rows<<<blocks, 256, 0, s>>>(n, bound, keep);
    launch_scan_rowptr(keep, n, pos, total, scan, s);
    k_training_rows<<<blocks, 256, 0, s>>>(n, nnz, keep, pos, ftmp, feats, targets);
}

void launch_features(const RawOperands &op, const int *row_list, int64_t nrows, float *feats, long long *bound,
                     int *err, int sms, cudaStream_t s) {
    if (nrows <= 0) return;
    const int64_t blocks = (nrows + 7) / 8;
    const int64_t cap = (int64_t)sms * 8;
    k_features<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(op, row_list, nrows, feats, bound, err);
}

void launch_mlp_infer(const float *feats, const long long *bound, const int *row_list, int64_t nrows,
                      const void *wb, const float *norm, float margin, float *y_out, int *cap_out, int sms,
                      cudaStream_t s) {
    if (nrows <= 0) return;
    const int64_t blocks = (nrows + 255) / 256;
    const int64_t cap = (int64_t)sms * 4;
    k_mlp_infer<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(feats, bound, row_list, nrows,
                                                                     (const __nv_bfloat16 *)wb, norm, margin, y_out,
                                                                     cap_out);
}

void launch_mlp_infer_tc(const float *feats, int64_t n, const void *wb, const float *norm, float *y, int sms,
                         cudaStream_t s) {
    if (n <= 0) return;
    static bool attr = false;
    const size_t smem = (size_t)mlp_tc_words(256 / 32) * 4;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 4;
    k_mlp_infer_tc<<<(int)(blocks < cap ? blocks : cap), 256, smem, s>>>(feats, n, (const __nv_bfloat16 *)wb,
                                                                          norm, y);
}

static size_t grad_smem() {
    return (size_t)(((kMlpParams + 3) & ~3) + 4 * kHid * kTile + kFeat * kTile + kTile) * sizeof(float);
}

void launch_mlp_grad(const float *feats, const float *targets, int64_t n, int64_t first, int64_t count,
                     unsigned long long mul, const unsigned long long *shift, const float *params, const float *norm,
                     float *grad, float *loss_acc, int sms, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
        attr = true;
    }
    if (count <= 0) return;
    Batch bt{n, first, count, mul, shift, 1.0f / (float)count};
    const int64_t tiles = (count + kTile - 1) / kTile;
    const int64_t cap = (int64_t)sms * 2;
    k_mlp_grad<<<(int)(tiles < cap ? tiles : cap), kTile, grad_smem(), s>>>(feats, targets, bt, params, norm, grad,
                                                                           loss_acc);
}

void launch_adam(float *params, float *grad, float *m, float *v, void *wb, float lr, float b1, float b2, float eps,
                 float wd, unsigned long long *stepc, cudaStream_t s) {
    k_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(params, grad, m, v, (__nv_bfloat16 *)wb, lr, b1, b2, eps, wd,
                                                    stepc);
    k_counter_add<<<1, 32, 0, s>>>(stepc, 1ull);
}

void launch_epoch_shift(unsigned long long *epoch, unsigned long long *shift, unsigned long long seed,
                        unsigned long long n, cudaStream_t s) {
    k_epoch_shift<<<1, 32, 0, s>>>(epoch, shift, seed, n);
}

__global__ void k_to_bf16(const float *src, __nv_bfloat16 *dst, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16(src[i]);
}

void launch_to_bf16(const float *src, void *dst, int n, cudaStream_t s) {
    if (n > 0) k_to_bf16<<<(n + 255) / 256, 256, 0, s>>>(src, (__nv_bfloat16 *)dst, n);
}

void launch_feat_stats(const float *feats, int64_t n, double *acc, int sms, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 4;
    k_feat_stats<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(feats, n, acc);
}

}  // namespace smash
