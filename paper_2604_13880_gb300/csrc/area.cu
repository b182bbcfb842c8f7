// Step 7 support (Sec. 4.1, Sec. 3.3): signed shoelace area of every region in
// double, average / maximum cartographic errors eps and xi against the desired
// areas w(v) = s(v) / M (M = total mass in the texture, so that area is
// proportional to mass once the density is equalised), fold-over detection,
// and the stop rule (xi < xi_stop, no improvement of xi within stall_window
// iterations, or max_iters iterations; Sec. 4.1 defaults).
//
// One kernel: a warp per region sums the shoelace terms of the region's edges
// (contiguous in the edge list, coalesced loads) with exact FP32 products and
// compensated FP32 sums (the FP64 pipe of this GPU is narrow; double is used
// only for the per-lane partials and the region areas); the last block of a
// job to finish (atomic ticket) forms the regions' relative errors in FP32,
// reduces them in a fixed order (compensated sum, maximum) and applies the
// stop rule, so the result does not depend on timing.
#include "area_impl.cuh"

namespace inim {

namespace {

__global__ void __launch_bounds__(256) k_areas_errors(const Job* __restrict__ jobs, const int2* __restrict__ bmap,
                                                      int update_state) {
    const int2 m = bmap[blockIdx.x];
    const Job J = jobs[m.x];                  // fixed over a run: read before the wait
    const AreaPre pre = areas_prefetch(J, m.y);
    pdl_start(J.pdl_early != 0);
    tl_begin(J.tl, kTlAreas);
    areas_body(J, m.y, update_state, pre, true);
    tl_end(J.tl, kTlAreas);
    pdl_release();
}

}  // namespace

cudaError_t launch_areas_errors(const Job* d_jobs, const BlockMap& region_blocks, int update_state,
                                cudaStream_t s) {
    return launch_pdl(k_areas_errors, region_blocks.n_blocks, 256, 0, s, d_jobs, (const int2*)region_blocks.d_map,
                      update_state);
}

}  // namespace inim
