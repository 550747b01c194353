// Group rows, float values; also the launch entry for both value types.
#include "k_group.cuh"

namespace smash {

void launch_num_group_f64(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                          float inv_load, const RowGather *rec, const NumOut &out, int *err, cudaStream_t s);

size_t num_group_smem(int dtype, int tbits, float inv_load, int group_shift) {
    const int gs = group_threads_of(tbits, group_shift);
    const int L = group_lcap(tbits, inv_load, gs);
    if (gs < 64 || L > 16 * gs) return SIZE_MAX;   // (one row per block, at most 16 entries per thread)
    return dtype ? group_smem_gs<double>(tbits, L, gs) : group_smem_gs<float>(tbits, L, gs);
}

void launch_num_group(int dtype, const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                      float inv_load, const RowGather *rec, const NumOut &out, int *err, cudaStream_t s) {
    if (count <= 0) return;
    if (dtype) launch_num_group_f64(r, rows, count, token, hl, inv_load, rec, out, err, s);
    else num_group_typed<float>(r, rows, count, token, hl, inv_load, rec, out, err, s);
}

}  // namespace smash
