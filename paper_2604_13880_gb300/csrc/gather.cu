// Steps 5-6 of the static algorithm (Sec. 4.1): the displacement
// t(x, y; d) - t(x, y; d0) of Eq. (3) at the four pixel centres around every
// vertex, bilinear interpolation, the shape blend and the move.
//
// Per corner pixel (i, j) the eight InIms come from S, T and the 1-D arrays
// through Eq. (1) (see scan_impl.cuh); differences are formed in the
// accumulator type (exact for FIX64, compensated for KAHAN), then scaled to
// ratios of C.  t(.; d0) uses the exact pixel counts of a constant texture
// (closed form) scaled by 1/N^2 (a power of two).  Eq. (2) is linear in the
// eight weights for fixed anchors, so the displacement t(d) - t(d0) is one
// evaluation of Eq. (2) on the weight differences; a constant texture gives
// exactly zero.
#include "gather_impl.cuh"

namespace inim {

namespace {

template <class Acc>
__global__ void __launch_bounds__(256) k_gather_move(const Job* __restrict__ jobs,
                                                     const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const Job& J = jobs[m.x];
    if (!J.st->active) return;
    gather_vertex<Acc>(J, m.y * blockDim.x + threadIdx.x);
}

template <class Acc>
__global__ void __launch_bounds__(256) k_displacement(const Job* __restrict__ job, const float2* xy,
                                                      int n, float2* out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    out[v] = displacement_at<Acc>(*job, xy[v]);
}

template <class Acc>
__global__ void k_finalize_B(const Job* __restrict__ job) {
    // turn the stored complements (w > 0) into B(w) = C - complement
    using T = typename Acc::T;
    const int n = job->n;
    T* B = reinterpret_cast<T*>(job->B);
    const T C = job->ST ? reinterpret_cast<const T*>(job->ST)[2 * ((size_t)n * n - 1)]
                        : reinterpret_cast<const T*>(job->S)[(size_t)n * n - 1];
    for (int w = 1 + blockIdx.x * blockDim.x + threadIdx.x; w <= n - 1; w += gridDim.x * blockDim.x)
        B[w + n - 1] = Acc::sub(C, B[w + n - 1]);
}

}  // namespace

cudaError_t launch_gather(const Job* d_jobs, const BlockMap& vert_blocks, int precision, cudaStream_t s) {
    if (!vert_blocks.n_blocks) return cudaSuccess;
    if (precision == INIM_FIX64) k_gather_move<AccFix><<<vert_blocks.n_blocks, 256, 0, s>>>(d_jobs, vert_blocks.d_map);
    else if (precision == INIM_KAHAN) k_gather_move<AccKahan><<<vert_blocks.n_blocks, 256, 0, s>>>(d_jobs, vert_blocks.d_map);
    else k_gather_move<AccF32><<<vert_blocks.n_blocks, 256, 0, s>>>(d_jobs, vert_blocks.d_map);
    return cudaGetLastError();
}

cudaError_t launch_displacement(const Job* d_job, const float* xy, int n, float* delta, int precision,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int g = (n + 255) / 256;
    const float2* p = reinterpret_cast<const float2*>(xy);
    float2* o = reinterpret_cast<float2*>(delta);
    if (precision == INIM_FIX64) k_displacement<AccFix><<<g, 256, 0, s>>>(d_job, p, n, o);
    else if (precision == INIM_KAHAN) k_displacement<AccKahan><<<g, 256, 0, s>>>(d_job, p, n, o);
    else k_displacement<AccF32><<<g, 256, 0, s>>>(d_job, p, n, o);
    return cudaGetLastError();
}

cudaError_t launch_finalize_B(const Job* d_job, int precision, cudaStream_t s) {
    if (precision == INIM_FIX64) k_finalize_B<AccFix><<<8, 256, 0, s>>>(d_job);
    else if (precision == INIM_KAHAN) k_finalize_B<AccKahan><<<8, 256, 0, s>>>(d_job);
    else k_finalize_B<AccF32><<<8, 256, 0, s>>>(d_job);
    return cudaGetLastError();
}

}  // namespace inim
