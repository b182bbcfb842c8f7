// Step 7 support (Sec. 4.1, Sec. 3.3): signed shoelace area of every region in
// double, average / maximum cartographic errors eps and xi against the desired
// areas w(v) = s(v) / M (M = total mass in the texture, so that area is
// proportional to mass once the density is equalised), fold-over detection,
// and the stop rule (xi < xi_stop, no improvement of xi within stall_window
// iterations, or max_iters iterations; Sec. 4.1 defaults).
#include "inim_internal.cuh"

namespace inim {

namespace {

// one warp per region; 8 regions per block
__global__ void __launch_bounds__(256) k_areas(const Job* __restrict__ jobs, const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const Job& J = jobs[m.x];
    if (!J.st->active) return;
    const int v = m.y * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (v >= J.n_regions) return;
    double acc = 0.0;
    for (int q = J.reg_ring_off[v]; q < J.reg_ring_off[v + 1]; ++q) {
        const int r = J.reg_rings[q];
        const int b = J.ring_off[r], e = J.ring_off[r + 1];
        const int len = e - b;
        for (int k = lane; k < len; k += 32) {
            const float2 p = J.xy[J.ring_idx[b + k]];
            const float2 q2 = J.xy[J.ring_idx[b + (k + 1 == len ? 0 : k + 1)]];
            // products of floats are exact in double
            acc += (double)p.x * (double)q2.y - (double)q2.x * (double)p.y;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) J.areas[v] = 0.5 * acc;
}

// one block per job
__global__ void __launch_bounds__(256) k_errors(const Job* __restrict__ jobs, int update_state) {
    const Job& J = jobs[blockIdx.x];
    JobState* st = J.st;
    if (!st->active) return;
    __shared__ double ssum[8], smax[8];
    __shared__ int sfold[8];
    const double M = st->mass;
    double sum = 0.0, mx = 0.0;
    int fold = 0;
    for (int v = threadIdx.x; v < J.n_regions; v += blockDim.x) {
        const double a = J.areas[v];
        const double o = fabs(a);
        const double w = (double)J.values[v] / M;
        const double den = fmax(o, w);
        const double e = den > 0.0 ? fabs(o - w) / den : 0.0;
        sum += e;
        mx = fmax(mx, e);
        const float s0 = J.sign0[v];
        if (s0 != 0.0f && ((a > 0.0) != (s0 > 0.0f) || a == 0.0)) fold = 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        fold |= __shfl_xor_sync(0xffffffffu, fold, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { ssum[w] = sum; smax[w] = mx; sfold[w] = fold; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, X = 0.0;
        int F = 0;
        for (int k = 0; k < 8; ++k) { S += ssum[k]; X = fmax(X, smax[k]); F |= sfold[k]; }
        const double eps = S / (double)J.n_regions;
        st->eps = eps;
        st->xi = X;
        if (F) st->foldover = 1;
        if (update_state) {
            st->iters += 1;
            if (X < st->best_xi) { st->best_xi = X; st->since = 0; }
            else st->since += 1;
            bool stop = st->iters >= st->max_iters;
            if (st->stop_on_rule) {
                if (st->xi_stop > 0.0f && X < (double)st->xi_stop) stop = true;
                if (st->eps_stop > 0.0f && eps < (double)st->eps_stop) stop = true;
                if (st->stall_window > 0 && st->since >= st->stall_window) stop = true;
            }
            if (st->error != 0) stop = true;
            if (stop) st->active = 0;
        }
    }
}

}  // namespace

cudaError_t launch_areas_errors(const Job* d_jobs, int n_jobs, const BlockMap& region_blocks,
                                int update_state, cudaStream_t s) {
    if (region_blocks.n_blocks) k_areas<<<region_blocks.n_blocks, 256, 0, s>>>(d_jobs, region_blocks.d_map);
    if (update_state >= 0) k_errors<<<n_jobs, 256, 0, s>>>(d_jobs, update_state);
    return cudaGetLastError();
}

}  // namespace inim
