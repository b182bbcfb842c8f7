// Integral-image band scan instantiated for one precision (see scan_impl.cuh).
#include "scan_impl.cuh"

namespace inim {

cudaError_t launch_scan_fp32(const Job* d_jobs, const BlockMap& band, const BlockMap& carry,
                           ScanTile tile, const float* dtex, cudaStream_t s, int phase) {
    return launch_scan_acc<AccF32>(d_jobs, band, carry, tile, dtex, phase, s);
}

}  // namespace inim
