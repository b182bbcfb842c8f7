// Integral-image band scan instantiated for one precision (see scan_impl.cuh).
#include "scan_impl.cuh"

namespace inim {

cudaError_t launch_scan_fix64(const Job* d_jobs, const BlockMap& band, const BlockMap& carry,
                           ScanTile tile, const float* dtex, cudaStream_t s, int phase) {
    return launch_scan_acc<AccFix>(d_jobs, band, carry, tile, dtex, phase, s);
}

}  // namespace inim
