// Warp rows: the symbolic kernel, float values, and the launch entries.
#include "k_warp.cuh"

namespace smash {

void launch_num_warp_f64(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                         float inv_load, const RowGather *rec, int bulk_copy, const NumOut &out, int *err,
                         cudaStream_t s);

size_t sym_warp_smem(int tbits) {
    return (size_t)kWarpRowWarps * (((size_t)4 << tbits) + sizeof(EntryScratch<float>));
}

void launch_sym_warp(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                     int *nnz_out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    const Operands<float> op = warp_operands<float>(r);
    const size_t smem = sym_warp_smem(hl.tbits);
    const HashCfg hc{hl.hash_kind, hl.colbits};
    if (r.b_nnz < INT_MAX) {
        auto kern = k_sym_warp<int32_t, kWarpRowWarps>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<warp_grid(kern, smem, hl.sms, count), kWarpRowWarps * 32, smem, s>>>(op, rows, count, token,
                                                                                  hl.tbits, hc, nnz_out, err);
    } else {
        auto kern = k_sym_warp<int64_t, kWarpRowWarps>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<warp_grid(kern, smem, hl.sms, count), kWarpRowWarps * 32, smem, s>>>(op, rows, count, token,
                                                                                  hl.tbits, hc, nnz_out, err);
    }
}

size_t num_warp_smem(int dtype, int tbits, float inv_load) {
    const int T = 1 << tbits;
    const int L = warp_lcap(tbits, inv_load);
    if (L > kWarpMaxList) return SIZE_MAX;   // more entries than the write-out's registers hold
    const int NB = warp_buckets(tbits);
    const size_t per = dtype ? warp_row_bytes<double>(T, L, NB) : warp_row_bytes<float>(T, L, NB);
    return (size_t)kWarpRowWarps * per;
}

void launch_num_warp(int dtype, const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                     float inv_load, const RowGather *rec, int bulk_copy, const NumOut &out, int *err,
                     cudaStream_t s) {
    if (count <= 0) return;
    if (dtype) launch_num_warp_f64(r, rows, count, token, hl, inv_load, rec, bulk_copy, out, err, s);
    else num_warp_typed<float>(r, rows, count, token, hl, inv_load, rec, bulk_copy, out, err, s);
}

}  // namespace smash
