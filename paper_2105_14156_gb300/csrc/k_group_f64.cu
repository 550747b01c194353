// Group rows, double values.
#include "k_group.cuh"

namespace smash {

void launch_num_group_f64(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                          float inv_load, const RowGather *rec, const NumOut &out, int *err, cudaStream_t s) {
    num_group_typed<double>(r, rows, count, token, hl, inv_load, rec, out, err, s);
}

}  // namespace smash
