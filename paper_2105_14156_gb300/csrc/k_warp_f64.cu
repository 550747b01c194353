// Warp rows, double values.
#include "k_warp.cuh"

namespace smash {

void launch_num_warp_f64(const RawOperands &r, const int *rows, int count, int *token, const HashLaunch &hl,
                         float inv_load, const RowGather *rec, int bulk_copy, const NumOut &out, int *err,
                         cudaStream_t s) {
    num_warp_typed<double>(r, rows, count, token, hl, inv_load, rec, bulk_copy, out, err, s);
}

}  // namespace smash
