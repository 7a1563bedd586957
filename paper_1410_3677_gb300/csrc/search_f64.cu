// FP64 instantiations of the search passes (FSTAT_FP64_PLAIN).
#include "search_launch.cuh"

namespace fstat {
int launch_search_cells_f64(const Plan &p, int band_idx, const BandDev &b, int64_t s0,
                            int64_t c0, int64_t nc, cudaStream_t s, cudaEvent_t mid,
                            const CellBufs &cb) {
    return launch_search_dispatch<double>(p, band_idx, b, s0, c0, nc, s, mid, cb);
}
}  // namespace fstat
