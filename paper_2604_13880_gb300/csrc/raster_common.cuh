// Device helpers shared by the rasteriser and the area kernel (which builds
// the next iteration's row histogram): the exact fixed-point edge setup, the
// per-edge row histogram and the block-level row offsets.
#pragma once

#include "inim_internal.cuh"

namespace inim {

struct EdgeFix {
    long long X0, Y0, X1, Y1;
    int jlo, jhi;
};

__device__ __forceinline__ bool edge_rows(const Job& J, int e, EdgeFix& f) {
    int2 ab = J.edges[e];
    float2 p = J.xy[ab.x];
    float2 q = J.xy[ab.y];
    const float scale = (float)(1 << (J.log2n + kSubBits));
    long long X0 = snap_coord(p.x, scale), Y0 = snap_coord(p.y, scale);
    long long X1 = snap_coord(q.x, scale), Y1 = snap_coord(q.y, scale);
    if (Y1 < Y0) {
        long long t = X0; X0 = X1; X1 = t;
        t = Y0; Y0 = Y1; Y1 = t;
    }
    if (Y1 == Y0) return false;                       // horizontal: never counted
    long long jlo = ceil_div(Y0 - 128, 256);
    long long jhi = ceil_div(Y1 - 128, 256) - 1;
    if (jlo < 0) jlo = 0;
    if (jhi > J.n - 1) jhi = J.n - 1;
    if (jlo > jhi) return false;
    f.X0 = X0; f.Y0 = Y0; f.X1 = X1; f.Y1 = Y1;
    f.jlo = (int)jlo; f.jhi = (int)jhi;
    return true;
}


// crossings per row of one edge (the histogram the keys are scattered by)
__device__ __forceinline__ void row_hist_edge(const Job& J, int e) {
    EdgeFix f;
    if (!edge_rows(J, e, f)) return;
    for (int j = f.jlo; j <= f.jhi; ++j) atomicAdd(&J.row_cnt[j], 1);
}

// Exclusive prefix of the per-row crossing counts of one job, done by one
// block (blockDim >= 256, N <= 4096); clears the counters (reused as fill
// cursors by k_crossings), the pixel counts and the big-row list, and checks
// the key capacity.
__device__ __forceinline__ void row_offsets_block(const Job& J) {
    __shared__ int wsum[32];
    const int n = J.n, nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    const int base = threadIdx.x * per;
    int s = 0;
    for (int k = 0; k < per; ++k) {
        const int idx = base + k;
        if (idx < n) s += __ldcg(J.row_cnt + idx);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int woff = 0, tot = 0;
    for (int k = 0; k < (nt >> 5); ++k) {
        if (k < w) woff += wsum[k];
        tot += wsum[k];
    }
    int run = woff + incl - s;
    for (int k = 0; k < per; ++k) {
        const int idx = base + k;
        if (idx < n) {
            const int v = __ldcg(J.row_cnt + idx);
            J.row_off[idx] = run;
            run += v;
            J.row_cnt[idx] = 0;
        }
    }
    if (threadIdx.x == 0) {
        J.row_off[n] = tot;
        J.st->n_big = 0;
        if (tot > J.key_cap) atomicExch(&J.st->error, INIM_E_CAPACITY);
    }
    for (int v = threadIdx.x; v <= J.n_regions; v += nt) J.counts[v] = 0;
    __syncthreads();
}

}  // namespace inim
