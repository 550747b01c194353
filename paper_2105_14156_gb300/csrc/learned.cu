// C ABI of learned sizing: the row-size model, its training on the device,
// and C = A*B sized by its predictions with an exact fallback.
//
// Not part of the paper (its setup phase counts each row exactly). The
// prediction replaces the symbolic pass: rows are hashed once with tables
// sized by the predicted capacity into a staging buffer; rows whose result
// does not fit are recomputed by the exact symbolic + numeric path, so C is
// always the exact product.
#include <cmath>
#include <cstdio>

#include "internal.h"

using namespace smash;
using namespace smash::host;

struct smash_model {
    smash_handle *h = nullptr;
    DevBuf block;
    smash_free_fn free_fn = nullptr;   // the allocator that provided block
    void *ctx = nullptr;
    float *params = nullptr;  // fp32 master weights
    float *grad = nullptr;
    float *m = nullptr;
    float *v = nullptr;
    void *wb = nullptr;        // bf16 inference copy
    float *norm = nullptr;     // mean[6], inv_std[6]
    unsigned long long *ctr = nullptr;  // [0] Adam step, [1] epoch, [2] permutation shift
    float *loss = nullptr;     // [0] current epoch's loss
    double *stats = nullptr;   // feature sums (12)
};

namespace {

constexpr int P = kMlpParams;

uint64_t splitmix(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double normal01(uint64_t &x) {
    const double u1 = ((splitmix(x) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (splitmix(x) >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

int upload_params(smash_model *m, const float *host_params, cudaStream_t s) {
    if (cudaMemcpyAsync(m->params, host_params, sizeof(float) * P, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    launch_to_bf16(m->params, m->wb, P, s);
    return cudaStreamSynchronize(s) == cudaSuccess ? SMASH_OK : SMASH_ERR_CUDA;
}

}  // namespace

extern "C" {

int smash_train_cfg_default(smash_train_cfg *c) {
    if (!c) return SMASH_ERR_INVALID_ARG;
    memset(c, 0, sizeof(*c));
    c->epochs = 8;
    c->batch = 4096;
    c->lr = 2e-3f;
    c->beta1 = 0.9f;
    c->beta2 = 0.999f;
    c->eps = 1e-8f;
    c->weight_decay = 0.f;
    c->seed = 1;
    return SMASH_OK;
}

int smash_model_create(smash_handle *h, smash_model **out, uint64_t seed) {
    if (!h || !out) return SMASH_ERR_INVALID_ARG;
    *out = nullptr;
    DeviceGuard g(h->device);
    smash_model *m = new (std::nothrow) smash_model();
    if (!m) return SMASH_ERR_ALLOC;
    m->h = h;
    size_t need = 0;
    for (size_t part : {4 * (size_t)P, 4 * (size_t)P, 4 * (size_t)P, 4 * (size_t)P, 2 * (size_t)P, (size_t)48,
                        (size_t)32, (size_t)64, (size_t)96})
        carve_size<char>(need, part);
    if (ensure(h, m->block, need, 0, true) != SMASH_OK) {
        delete m;
        return SMASH_ERR_ALLOC;
    }
    m->free_fn = h->free_fn;
    m->ctx = h->ctx;
    cudaDeviceSynchronize();
    Carver c(m->block.ptr);
    m->params = c.take<float>(P);
    m->grad = c.take<float>(P);
    m->m = c.take<float>(P);
    m->v = c.take<float>(P);
    m->wb = c.take<uint16_t>(P);
    m->norm = c.take<float>(12);
    m->ctr = c.take<unsigned long long>(4);
    m->loss = c.take<float>(16);
    m->stats = c.take<double>(12);
    // He initialisation; biases zero; identity normalisation.
    std::vector<float> p(P, 0.f);
    uint64_t x = seed * 0x2545F4914F6CDD1Dull + 17;
    for (int k = 0; k < 64 * 6; ++k) p[k] = (float)(normal01(x) * sqrt(2.0 / 6.0));
    for (int k = 0; k < 64 * 64; ++k) p[448 + k] = (float)(normal01(x) * sqrt(2.0 / 64.0));
    for (int k = 0; k < 64; ++k) p[4608 + k] = (float)(normal01(x) * sqrt(1.0 / 64.0));
    float norm[12];
    for (int k = 0; k < 6; ++k) {
        norm[k] = 0.f;
        norm[6 + k] = 1.f;
    }
    if (cudaMemcpy(m->norm, norm, sizeof(norm), cudaMemcpyHostToDevice) != cudaSuccess ||
        upload_params(m, p.data(), 0) != SMASH_OK) {
        cudaDeviceSynchronize();
        m->free_fn(m->block.ptr, m->ctx);
        delete m;
        return SMASH_ERR_CUDA;
    }
    *out = m;
    return SMASH_OK;
}

int smash_model_destroy(smash_model *m) {
    if (!m) return SMASH_ERR_INVALID_ARG;
    {
        DeviceGuard g(m->h->device);
        cudaDeviceSynchronize();
        if (m->block.ptr) m->free_fn(m->block.ptr, m->ctx);   // with the allocator that provided it
    }
    delete m;
    return SMASH_OK;
}

int smash_model_get(const smash_model *m, float *params, float *norm) {
    if (!m) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(m->h->device);
    cudaDeviceSynchronize();
    if (params && cudaMemcpy(params, m->params, sizeof(float) * P, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SMASH_ERR_CUDA;
    if (norm && cudaMemcpy(norm, m->norm, sizeof(float) * 12, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SMASH_ERR_CUDA;
    return SMASH_OK;
}

int smash_model_set(smash_model *m, const float *params, const float *norm) {
    if (!m) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(m->h->device);
    cudaDeviceSynchronize();
    if (norm && cudaMemcpy(m->norm, norm, sizeof(float) * 12, cudaMemcpyHostToDevice) != cudaSuccess)
        return SMASH_ERR_CUDA;
    if (params) return upload_params(m, params, 0);
    return SMASH_OK;
}

int smash_model_save(const smash_model *m, const char *path) {
    if (!m || !path) return SMASH_ERR_INVALID_ARG;
    std::vector<float> p(P);
    float norm[12];
    int st = smash_model_get(m, p.data(), norm);
    if (st) return st;
    FILE *f = fopen(path, "wb");
    if (!f) return SMASH_ERR_INVALID_ARG;
    const int32_t ver = 1, np = P;
    bool ok = fwrite("SMASHMLP", 1, 8, f) == 8 && fwrite(&ver, 4, 1, f) == 1 && fwrite(&np, 4, 1, f) == 1 &&
              fwrite(p.data(), 4, P, f) == (size_t)P && fwrite(norm, 4, 12, f) == 12;
    ok = (fclose(f) == 0) && ok;
    return ok ? SMASH_OK : SMASH_ERR_INVALID_ARG;
}

int smash_model_load(smash_model *m, const char *path) {
    if (!m || !path) return SMASH_ERR_INVALID_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return SMASH_ERR_INVALID_ARG;
    char magic[8];
    int32_t ver = 0, np = 0;
    std::vector<float> p(P);
    float norm[12];
    const bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "SMASHMLP", 8) == 0 && fread(&ver, 4, 1, f) == 1 &&
                    ver == 1 && fread(&np, 4, 1, f) == 1 && np == P && fread(p.data(), 4, P, f) == (size_t)P &&
                    fread(norm, 4, 12, f) == 12;
    fclose(f);
    if (!ok) return SMASH_ERR_INVALID_ARG;
    return smash_model_set(m, p.data(), norm);
}

int smash_row_features(smash_handle *h, const smash_csr *A, const smash_csr *B, float *feats, void *stream) {
    if (!h || !feats) return SMASH_ERR_INVALID_ARG;
    int st = check_csr(A, false);
    if (st) return st;
    if ((st = check_csr(B, false))) return st;
    if (A->cols != B->rows) return SMASH_ERR_SHAPE_MISMATCH;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const RawOperands op = raw_ops(A, B);
    {
        LaunchTimer lt(h, s, "features", -1, 256, A->rows, A->nnz, 0, 0);
        launch_features(op, nullptr, A->rows, feats, nullptr, (int *)h->err.ptr, h->sms, s);
    }
    return last_cuda_status();
}

int smash_training_rows(smash_handle *h, const smash_csr *A, const smash_csr *B, float *feats, float *targets,
                        int64_t *count, void *stream) {
    if (!h || !feats || !targets || !count) return SMASH_ERR_INVALID_ARG;
    int st = check_csr(A, false);
    if (st) return st;
    if ((st = check_csr(B, false))) return st;
    if (A->cols != B->rows) return SMASH_ERR_SHAPE_MISMATCH;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->rows;
    *count = 0;
    if (n == 0) return SMASH_OK;
    const RawOperands op = raw_ops(A, B);
    // 1. exact nnz(C_i) of every row (the symbolic phase)
    Plan pl;
    if ((st = plan_buffers(h, n, true, s, pl))) return st;
    if (A->nnz > 0 && B->nnz > 0) {
        if ((st = run_symbolic(h, op, n, pl, pl.nnz, s, nullptr, 0))) return st;
    } else if (cudaMemsetAsync(pl.nnz, 0, sizeof(int) * (size_t)n, s) != cudaSuccess) {
        return SMASH_ERR_CUDA;
    }
    // 2. features and bounds of every row; 3. rows with products, in order
    size_t need = 0;
    carve_size<float>(need, (size_t)n * 6);
    carve_size<long long>(need, (size_t)n);
    carve_size<int>(need, (size_t)n);
    carve_size<int64_t>(need, (size_t)n + 1);
    carve_size<long long>(need, 1);
    carve_size<char>(need, scan_scratch_bytes(n));
    if ((st = ensure(h, h->learn, need, s))) return st;
    Carver c(h->learn.ptr);
    float *ftmp = c.take<float>((size_t)n * 6);
    long long *bound = c.take<long long>((size_t)n);
    int *keep = c.take<int>((size_t)n);
    int64_t *pos = c.take<int64_t>((size_t)n + 1);
    long long *total = c.take<long long>(1);
    void *scan = c.take<char>(scan_scratch_bytes(n));
    {
        LaunchTimer lt(h, s, "training_rows", -1, 256, n, A->nnz, 0, 0, 5);
        launch_features(op, nullptr, n, ftmp, bound, (int *)h->err.ptr, h->sms, s);
        launch_training_rows(n, pl.nnz, bound, ftmp, keep, pos, total, scan, feats, targets, h->sms, s);
    }
    if ((st = last_cuda_status())) return st;
    if (read_small(h, 0, total, sizeof(long long), s)) return SMASH_ERR_CUDA;
    st = read_flags(h, s, true);
    *count = h->host[0];
    return st;
}

int smash_mlp_gradient(smash_handle *h, smash_model *m, const float *feats, const float *targets, int64_t n,
                       float *grad, float *loss, void *stream) {
    if (!h || !m || !feats || !targets || !grad || n <= 0) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(m->grad, 0, sizeof(float) * P, s);
    cudaMemsetAsync(m->loss, 0, sizeof(float), s);
    launch_mlp_grad(feats, targets, n, 0, n, 1ull, nullptr, m->params, m->norm, m->grad, m->loss, h->sms, s);
    cudaMemcpyAsync(grad, m->grad, sizeof(float) * P, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(m->grad, 0, sizeof(float) * P, s);
    float lh = 0.f;
    cudaMemcpyAsync(h->host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return SMASH_ERR_CUDA;
    memcpy(&lh, h->host, sizeof(float));
    if (loss) *loss = lh;
    return last_cuda_status();
}

int smash_mlp_predict(smash_handle *h, const smash_model *m, const float *feats, int64_t n, float *y,
                      void *stream) {
    if (!h || !m || !feats || !y || n < 0) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    launch_mlp_infer(feats, nullptr, nullptr, n, m->wb, m->norm, 0.f, y, nullptr, h->sms, (cudaStream_t)stream);
    return last_cuda_status();
}

int smash_mlp_predict_tc(smash_handle *h, const smash_model *m, const float *feats, int64_t n, float *y,
                         void *stream) {
    if (!h || !m || !feats || !y || n < 0) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    launch_mlp_infer_tc(feats, n, m->wb, m->norm, y, h->sms, (cudaStream_t)stream);
    return last_cuda_status();
}

int smash_mlp_train(smash_handle *h, smash_model *m, const float *feats, const float *targets, int64_t n,
                    const smash_train_cfg *cfg_in, float *final_loss, void *stream) {
    if (!h || !m || !feats || !targets || n <= 0 || n >= (1ll << 31)) return SMASH_ERR_INVALID_ARG;
    smash_train_cfg cfg;
    if (cfg_in) cfg = *cfg_in;
    else smash_train_cfg_default(&cfg);
    if (cfg.epochs <= 0 || cfg.batch <= 0 || !(cfg.lr > 0.f)) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t caller = (cudaStream_t)stream;
    // normalisation from the data
    cudaMemsetAsync(m->stats, 0, sizeof(double) * 12, caller);
    launch_feat_stats(feats, n, m->stats, h->sms, caller);
    double acc[12];
    if (cudaMemcpyAsync(acc, m->stats, sizeof(acc), cudaMemcpyDeviceToHost, caller) != cudaSuccess ||
        cudaStreamSynchronize(caller) != cudaSuccess)
        return SMASH_ERR_CUDA;
    float norm[12];
    for (int k = 0; k < 6; ++k) {
        const double mean = acc[k] / (double)n;
        const double var = acc[6 + k] / (double)n - mean * mean;
        norm[k] = (float)mean;
        norm[6 + k] = var > 1e-12 ? (float)(1.0 / sqrt(var)) : 1.f;
    }
    if (cudaMemcpy(m->norm, norm, sizeof(norm), cudaMemcpyHostToDevice) != cudaSuccess) return SMASH_ERR_CUDA;
    // sample order: position q of an epoch reads sample (a*q + c_e) mod n
    uint64_t x = cfg.seed * 0x9E3779B97F4A7C15ull + 3;
    uint64_t a = (splitmix(x) % (uint64_t)n) | 1ull;
    while (gcd64(a, (uint64_t)n) != 1ull) a = (a + 2) % (uint64_t)n ? (a + 2) % (uint64_t)n : 1ull;
    // one epoch as a CUDA graph (captured on a private stream), replayed per epoch
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return SMASH_ERR_CUDA;
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, caller);
    cudaStreamWaitEvent(cs, ev, 0);
    const int64_t steps = (n + cfg.batch - 1) / cfg.batch;
    launch_mlp_grad(feats, targets, n, 0, 0, a, nullptr, m->params, m->norm, m->grad, m->loss, h->sms, cs);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int st = SMASH_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = SMASH_ERR_CUDA;
    if (st == SMASH_OK) {
        cudaMemsetAsync(m->loss, 0, sizeof(float), cs);
        launch_epoch_shift(m->ctr + 1, m->ctr + 2, cfg.seed, (unsigned long long)n, cs);
        for (int64_t k = 0; k < steps; ++k) {
            const int64_t first = k * cfg.batch;
            const int64_t cnt = (n - first) < cfg.batch ? (n - first) : cfg.batch;
            // the loss accumulates sum over batches of each batch's mean; divide by steps below
            launch_mlp_grad(feats, targets, n, first, cnt, a, m->ctr + 2, m->params, m->norm, m->grad, m->loss,
                            h->sms, cs);
            launch_adam(m->params, m->grad, m->m, m->v, m->wb, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps,
                        cfg.weight_decay, m->ctr, cs);
        }
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) st = SMASH_ERR_CUDA;
    }
    if (st == SMASH_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) st = SMASH_ERR_CUDA;
    for (int e = 0; st == SMASH_OK && e < cfg.epochs; ++e)
        if (cudaGraphLaunch(exec, cs) != cudaSuccess) st = SMASH_ERR_CUDA;
    float lh = 0.f;
    if (st == SMASH_OK) {
        cudaMemcpyAsync(h->host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, cs);
        if (cudaStreamSynchronize(cs) != cudaSuccess) st = SMASH_ERR_CUDA;
        memcpy(&lh, h->host, sizeof(float));
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaEventRecord(ev, cs);
    cudaStreamWaitEvent(caller, ev, 0);
    cudaEventDestroy(ev);
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (final_loss) *final_loss = lh / (float)steps;
    return st;
}

int smash_free_csr(smash_handle *h, smash_csr *C) {
    if (!h || !C) return SMASH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    if (C->row_ptr) h->free_fn(C->row_ptr, h->ctx);
    if (C->col_idx) h->free_fn(C->col_idx, h->ctx);
    if (C->val) h->free_fn(C->val, h->ctx);
    C->row_ptr = nullptr;
    C->col_idx = nullptr;
    C->val = nullptr;
    return SMASH_OK;
}

int spgemm_learned(smash_handle *h, const smash_csr *A, const smash_csr *B, smash_dtype dtype,
                   const smash_model *m, float margin, smash_csr *C, smash_learned_stats *stats, void *stream) {
    if (!h || !C || !(margin > -1.f)) return SMASH_ERR_INVALID_ARG;
    if (dtype != SMASH_F32 && dtype != SMASH_F64) return SMASH_ERR_UNSUPPORTED;
    int st = check_csr(A, true);
    if (st) return st;
    if ((st = check_csr(B, true))) return st;
    if (A->cols != B->rows) return SMASH_ERR_SHAPE_MISMATCH;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->rows;
    const int dt = dtype == SMASH_F64 ? 1 : 0;
    const size_t vsz = dt ? 8 : 4;
    memset(&h->stats, 0, sizeof(h->stats));
    smash_learned_stats ls;
    memset(&ls, 0, sizeof(ls));
    ls.rows = n;
    C->rows = n;
    C->cols = B->cols;
    C->nnz = 0;
    C->row_ptr = nullptr;
    C->col_idx = nullptr;
    C->val = nullptr;
    // C's arrays go back to the allocator if the call fails
    struct CGuard {
        smash_handle *h;
        smash_csr *C;
        bool keep = false;
        ~CGuard() {
            if (keep) return;
            cudaDeviceSynchronize();
            cudaGetLastError();
            if (C->row_ptr) h->free_fn(C->row_ptr, h->ctx);
            if (C->col_idx) h->free_fn(C->col_idx, h->ctx);
            if (C->val) h->free_fn(C->val, h->ctx);
            C->row_ptr = nullptr;
            C->col_idx = nullptr;
            C->val = nullptr;
            C->nnz = 0;
        }
    } guard{h, C};
    C->row_ptr = (int64_t *)h->alloc(sizeof(int64_t) * (size_t)(n + 1), h->ctx);
    if (!C->row_ptr) return SMASH_ERR_ALLOC;
    if (n == 0 || A->nnz == 0 || B->nnz == 0) {
        cudaMemsetAsync(C->row_ptr, 0, sizeof(int64_t) * (size_t)(n + 1), s);
        if (stats) *stats = ls;
        const int rc = cudaStreamSynchronize(s) == cudaSuccess ? SMASH_OK : SMASH_ERR_CUDA;
        guard.keep = rc == SMASH_OK;
        return rc;
    }
    const RawOperands op = raw_ops(A, B);
    int *err = (int *)h->err.ptr;
    // the dense rows of this call are counted by this call (no reuse of an
    // earlier symbolic phase's counts), and B is sliced afresh
    h->wcache.valid = false;
    h->plan_cache.valid = false;
    // per-row arrays
    size_t need = 0;
    carve_size<RowGather>(need, (size_t)n);       // planning scratch
    carve_size<int>(need, (size_t)n);             // cap
    carve_size<int64_t>(need, (size_t)n + 1);     // stage_rp
    carve_size<int>(need, (size_t)n);             // row_nnz
    carve_size<uint8_t>(need, (size_t)n);         // ovf
    carve_size<int>(need, (size_t)n);             // overflow list
    carve_size<long long>(need, 4);               // counters
    carve_size<char>(need, scan_scratch_bytes(n));
    if ((st = ensure(h, h->learn, need, s))) return st;
    Carver c(h->learn.ptr);
    RowGather *gather = c.take<RowGather>((size_t)n);
    int *cap = c.take<int>((size_t)n);
    int64_t *stage_rp = c.take<int64_t>((size_t)n + 1);
    int *row_nnz = c.take<int>((size_t)n);
    uint8_t *ovf = c.take<uint8_t>((size_t)n);
    int *list = c.take<int>((size_t)n);
    long long *ctr = c.take<long long>(4);
    void *scan = c.take<char>(scan_scratch_bytes(n));
    cudaMemsetAsync(ctr, 0, 4 * sizeof(long long), s);
    cudaMemsetAsync(row_nnz, 0, sizeof(int) * (size_t)n, s);
    // 1. one planning pass: features, predicted capacity, bin of every row
    Plan pl;
    if ((st = plan_buffers(h, n, false, s, pl))) return st;
    {
        LearnArgs la;
        la.wb = m ? m->wb : nullptr;     // no model: every row sized by its bound
        la.norm = m ? m->norm : nullptr;
        la.margin = margin;
        la.cap = cap;
        la.gather = gather;
        const BinRule rule = num_rule(h, op.ncols, dt);
        {
            LaunchTimer lt(h, s, "learned_gather", -1, 256, n, A->nnz, 0, 0, 2);
            launch_learned_gather(op, rule, pl.bb, la, err, h->sms, s);
        }
        LaunchTimer lt(h, s, "learned_bin", -1, 256, n, 0, 0, 0);
        launch_learned_bin(op, rule, pl.bb, la, h->sms, s);
    }
    {
        LaunchTimer lt(h, s, "bin_scatter", -1, 256, n, 0, 0, 0);
        launch_bin_scatter(n, pl.bb, s);
    }
    if ((st = last_cuda_status())) return st;
    BinPlan bp;
    if ((st = fetch_bins(h, pl, s, bp.counts, bp.offsets, bp.maxsize, bp.stats, bp.sums))) return st;
    // 2. dense rows with column windows write into an arena sized by their
    //    predicted capacities; the other rows get staging ranges
    const int nd = bp.counts[kBinDense];
    const int *drows = pl.bb.rows + bp.offsets[kBinDense];   // valid until the next plan_buffers()
    int cpc = 0, nw = 0, per = 1;
    const bool use_arena = nd > 0 && dense_windows(h, op, dt, bp.sums[16 + kBinDense], cpc, nw, per);
    WinArena ar;
    const int *arena_rows = nullptr;
    if (use_arena) {
        ar.cap = bp.sums[32 + kBinDense] > 0 ? bp.sums[32 + kBinDense] : 1;
        size_t aneed = 0;
        carve_size<unsigned long long>(aneed, 1);
        carve_size<int32_t>(aneed, (size_t)ar.cap);
        carve_size<char>(aneed, (size_t)ar.cap * vsz);
        carve_size<int64_t>(aneed, (size_t)nd * nw);
        carve_size<int>(aneed, (size_t)nd * nw);
        carve_size<int>(aneed, (size_t)nd);
        if ((st = ensure(h, h->arena, aneed, s))) return st;
        Carver ac(h->arena.ptr);
        ar.top = ac.take<unsigned long long>(1);
        ar.ci = ac.take<int32_t>((size_t)ar.cap);
        ar.val = ac.take<char>((size_t)ar.cap * vsz);
        ar.desc_off = ac.take<int64_t>((size_t)nd * nw);
        ar.desc_cnt = ac.take<int>((size_t)nd * nw);
        // the dense rows' list outlives the plan buffers (the fallback's plans
        // reuse them before the arena is compacted)
        int *dcopy = ac.take<int>((size_t)nd);
        if (cudaMemcpyAsync(dcopy, drows, sizeof(int) * (size_t)nd, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return SMASH_ERR_CUDA;
        arena_rows = dcopy;
        cudaMemsetAsync(ar.top, 0, sizeof(unsigned long long), s);
        launch_zero_rows(drows, nd, cap, s);
    }
    {
        LaunchTimer lt(h, s, "scan_rowptr", -1, 512, n, 0, 0, 0, 3);
        launch_scan_rowptr(cap, n, stage_rp, ctr, scan, s);
    }
    if ((st = last_cuda_status())) return st;
    if (read_small(h, 0, ctr, sizeof(long long), s) || cudaStreamSynchronize(s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    const long long staged = h->host[0];
    ls.staged_nnz = staged + (use_arena ? ar.cap : 0);
    size_t sneed = 0;
    carve_size<int32_t>(sneed, (size_t)staged);
    carve_size<char>(sneed, (size_t)staged * vsz);
    if ((st = ensure(h, h->stage, sneed, s))) return st;
    Carver sc(h->stage.ptr);
    int32_t *stage_ci = sc.take<int32_t>((size_t)staged);
    void *stage_val = sc.take<char>((size_t)staged * vsz);
    // 3. one hashing pass with predicted capacities
    NumOut so;
    so.c_rp = stage_rp;
    so.c_ci = stage_ci;
    so.c_val = stage_val;
    so.c_nnz = staged;
    so.row_nnz = row_nnz;
    if ((st = run_bins(h, op, n, dt, so, pl, bp, s, use_arena ? &ar : nullptr, gather))) return st;
    // 4. rows that did not fit
    {
        LaunchTimer lt(h, s, "overflow_list", -1, 256, n, 0, 0, 0);
        launch_overflow_list(row_nnz, n, list, (int *)(ctr + 1), ovf, s);
        if (use_arena) launch_mark_rows(arena_rows, nd, row_nnz, ovf, s);
    }
    if (read_small(h, 0, ctr + 1, sizeof(long long), s) || cudaStreamSynchronize(s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    const int novf = (int)(h->host[0] & 0xffffffff);
    ls.overflow_rows = novf;
    if (novf > 0) {
        Plan ps;
        if ((st = plan_buffers(h, n, true, s, ps))) return st;
        if ((st = run_symbolic(h, op, n, ps, row_nnz, s, list, novf))) return st;
    }
    // 5. exact row pointer of C, then its arrays
    {
        LaunchTimer lt(h, s, "scan_rowptr", -1, 512, n, 0, 0, 0, 3);
        launch_scan_rowptr(row_nnz, n, C->row_ptr, ctr + 2, scan, s);
    }
    if (read_small(h, 0, ctr + 2, sizeof(long long), s) || cudaStreamSynchronize(s) != cudaSuccess)
        return SMASH_ERR_CUDA;
    const long long cnnz = h->host[0];
    C->nnz = cnnz;
    ls.c_nnz = cnnz;
    if (cnnz > 0) {
        C->col_idx = (int32_t *)h->alloc(sizeof(int32_t) * (size_t)cnnz, h->ctx);
        C->val = h->alloc(vsz * (size_t)cnnz, h->ctx);
        if (!C->col_idx || !C->val) return SMASH_ERR_ALLOC;
        {
            // without an arena nearly every row was staged: block copy, its chunk
            // table in the planning scratch (free by now) when it fits there
            int *table = !use_arena && compact_table_bytes(cnnz) <= sizeof(RowGather) * (size_t)n ? (int *)gather
                                                                                                   : nullptr;
            LaunchTimer lt(h, s, "compact_rows", -1, 256, n, 0, 0, cnnz, table ? 2 : 1);
            launch_compact_rows(dt, n, stage_rp, ovf, stage_ci, stage_val, C->row_ptr, C->col_idx, C->val, cnnz,
                                table, h->sms, s);
        }
        if (use_arena) {
            LaunchTimer lt(h, s, "compact_arena", -1, 256, nd, 0, 0, cnnz);
            launch_arena_compact(dt, arena_rows, nd, nw, ar, ovf, C->row_ptr, C->col_idx, C->val, h->sms, s);
        }
        if (novf > 0) {
            Plan pn;
            if ((st = plan_buffers(h, n, false, s, pn))) return st;
            NumOut co;
            co.c_rp = C->row_ptr;
            co.c_ci = C->col_idx;
            co.c_val = C->val;
            co.c_nnz = cnnz;
            if ((st = run_numeric(h, op, n, dt, co, pn, s, list, novf))) return st;
        }
    }
    st = read_flags(h, s, true);
    h->stats.c_nnz = cnnz;
    if (stats) *stats = ls;
    guard.keep = st == SMASH_OK;
    return st;
}

}  // extern "C"
