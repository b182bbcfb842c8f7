// Device helpers of the rasteriser (per-step kernels and persistent form):
// the exact fixed-point edge setup, the key emission into fixed-stride row
// buckets and the per-job resets.
#pragma once

#include "inim_internal.cuh"

namespace inim {

// An edge in fixed point (I = long long for any input; I = int when every
// coordinate is below 512 in magnitude: |X| < 2^29 for textures up to 4096^2,
// so that the differences the rule needs stay exact in 32 bits).
template <class I>
struct EdgeFixT {
    I X0, Y0, X1, Y1;
    int jlo, jhi;
};
using EdgeFix = EdgeFixT<long long>;

__device__ __forceinline__ long long snap_t(float x, float scale, long long) { return snap_coord(x, scale); }
__device__ __forceinline__ int snap_t(float x, float scale, int) { return __float2int_rn(x * scale); }
__device__ __forceinline__ long long ceil_div256(long long a) { return ceil_div(a, 256); }
__device__ __forceinline__ int ceil_div256(int a) { return (a + 255) >> 8; }   // |a| < 2^30: exact

template <class I>
__device__ __forceinline__ bool edge_rows_pts(const Job& J, float2 p, float2 q, EdgeFixT<I>& f) {
    const float scale = (float)(1 << (J.log2n + kSubBits));
    I X0 = snap_t(p.x, scale, I{}), Y0 = snap_t(p.y, scale, I{});
    I X1 = snap_t(q.x, scale, I{}), Y1 = snap_t(q.y, scale, I{});
    if (Y1 < Y0) {
        I t = X0; X0 = X1; X1 = t;
        t = Y0; Y0 = Y1; Y1 = t;
    }
    if (Y1 == Y0) return false;                       // horizontal: never counted
    I jlo = ceil_div256(Y0 - 128);
    I jhi = ceil_div256(Y1 - 128) - 1;
    if (jlo < 0) jlo = 0;
    if (jhi > J.n - 1) jhi = J.n - 1;
    if (jlo > jhi) return false;
    f.X0 = X0; f.Y0 = Y0; f.X1 = X1; f.Y1 = Y1;
    f.jlo = (int)jlo; f.jhi = (int)jhi;
    return true;
}


__device__ __forceinline__ bool edge_rows(const Job& J, int e, EdgeFix& f) {
    const int2 ab = J.edges[e];
    return edge_rows_pts(J, J.xy[ab.x], J.xy[ab.y], f);
}

// min(max(ceil(num / den), 0), n) exactly, for den > 0, without a 64-bit
// division: a float estimate of the quotient (only needed in [0, n], n <=
// 4096, where it is off by less than one) corrected by exact int64 products.
__device__ __forceinline__ int clamped_ceil_div(long long num, long long den, int n) {
    if (num <= 0) return 0;                              // ceil <= 0
    if (num > (long long)n * den) return n;              // ceil > n
    long long q = (long long)floorf(__fdiv_rn((float)num, (float)den));
    long long r = num - q * den;
    while (r < 0) { --q; r += den; }
    while (r >= den) { ++q; r -= den; }
    const long long c = q + (r > 0 ? 1 : 0);
    return (int)(c > n ? n : c);
}

// The crossings of a warp's edges (E per lane; slots with valid == false take
// part with no crossings) with the texture rows they span: (region << 16 |
// first counted column) keys appended to the rows' fixed-stride buckets; a
// bucket that would overflow raises the capacity error when its row is
// rasterised.  A stretched edge can span hundreds of rows; instead of one lane
// walking them all, the warp numbers the crossings of its edges with a prefix
// sum (lane-major, then slot) and hands them out 32 at a time: crossing i
// belongs to the last lane whose exclusive prefix is <= i (found by a binary
// search over the lanes' prefixes), which supplies its edges through
// shuffles, and to the slot whose range holds it.  The warp's serial work is
// total / 32 crossings instead of the longest edge's row count; the bucket
// atomics of kCrossPipe rounds go out together, so a warp whose stretched
// edges cross many rows waits for one atomic round trip per 32 * kCrossPipe
// crossings.  I is the fixed-point type of the end points (EdgeFixT).
constexpr int kCrossPipe = 4;

template <int E, class I>
__device__ __forceinline__ void emit_crossings_lane(const Job& J, const bool (&valid)[E], const unsigned (&reg)[E],
                                                    const float2 (&p)[E], const float2 (&q)[E]) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    EdgeFixT<I> f[E];
    int c[E];
    int cnt = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        f[e] = EdgeFixT<I>{};
        c[e] = (valid[e] && edge_rows_pts(J, p[e], q[e], f[e])) ? f[e].jhi - f[e].jlo + 1 : 0;
        cnt += c[e];
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(full, incl, 31);
    // the 64-bit form (far-away end points only) pipelines two rounds: fewer
    // registers beside the 32-bit form in one kernel
    constexpr int PIPE = sizeof(I) == 4 ? kCrossPipe : 2;
    for (int base = 0; base < total; base += 32 * PIPE) {
        // up to PIPE rounds of 32 crossings, then their bucket atomics
        // together (one round trip for the batch), then the key stores
        int jq[PIPE];
        unsigned kq[PIPE];
#pragma unroll
        for (int t = 0; t < PIPE; ++t) {
            jq[t] = -1;
            kq[t] = 0;
            if (base + 32 * t >= total) continue;             // warp-uniform
            const int i = base + 32 * t + lane;
            int owner = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int cand = owner + step;
                if (__shfl_sync(full, excl, cand) <= i) owner = cand;
            }
            const int k = i - __shfl_sync(full, excl, owner);     // index among the owner's crossings
            I X0 = 0, Y0 = 0, X1 = 0, Y1 = 0;
            int j = 0;
            unsigned r = 0;
            int acc = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ce = __shfl_sync(full, c[e], owner);
                const I x0 = __shfl_sync(full, f[e].X0, owner), y0 = __shfl_sync(full, f[e].Y0, owner);
                const I x1 = __shfl_sync(full, f[e].X1, owner), y1 = __shfl_sync(full, f[e].Y1, owner);
                const int jl = __shfl_sync(full, f[e].jlo, owner);
                const unsigned re = __shfl_sync(full, reg[e], owner);
                if (k >= acc && k < acc + ce) {
                    X0 = x0; Y0 = y0; X1 = x1; Y1 = y1;
                    j = jl + (k - acc);
                    r = re;
                }
                acc += ce;
            }
            if (i < total) {
                const I dY = Y1 - Y0, dX = X1 - X0;
                const I Yc = (I)256 * j + 128;
                const long long num = (long long)dX * (long long)(Yc - Y0) + (long long)(X0 - 128) * (long long)dY;
                const int col = clamped_ceil_div(num, 256LL * (long long)dY, J.n);
                jq[t] = j;
                kq[t] = (r << 16) | (unsigned)col;
            }
        }
        int slot[PIPE];
#pragma unroll
        for (int t = 0; t < PIPE; ++t) slot[t] = jq[t] >= 0 ? atomicAdd(&J.row_cnt[jq[t]], 1) : kKeyStride;
#pragma unroll
        for (int t = 0; t < PIPE; ++t)
            if (slot[t] < kKeyStride) J.keys[(size_t)jq[t] * kKeyStride + slot[t]] = kq[t];
    }
}

// emit_crossings_lane in 32-bit fixed point when every end point of the
// warp's edges lies within 512 of the origin (the same keys), else in 64 bits.
template <int E>
__device__ __forceinline__ void emit_crossings_warp(const Job& J, const bool (&valid)[E], const unsigned (&reg)[E],
                                                    const float2 (&p)[E], const float2 (&q)[E]) {
    bool wide = false;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (valid[e])
            wide |= !(fabsf(p[e].x) < 512.0f && fabsf(p[e].y) < 512.0f && fabsf(q[e].x) < 512.0f &&
                      fabsf(q[e].y) < 512.0f);
    if (__any_sync(0xffffffffu, wide)) emit_crossings_lane<E, long long>(J, valid, reg, p, q);
    else emit_crossings_lane<E, int>(J, valid, reg, p, q);
}

// One item of kEdgesPerItem edges of a job (a block of 256 threads; lane
// slot s holds edge item * kEdgesPerItem + s * 256 + threadIdx.x), loading
// the edges and their end points itself.
__device__ __forceinline__ void emit_crossings_item(const Job& J, int item) {
    bool valid[kEdgesPerLane];
    unsigned reg[kEdgesPerLane];
    float2 p[kEdgesPerLane], q[kEdgesPerLane];
#pragma unroll
    for (int s = 0; s < kEdgesPerLane; ++s) {
        const int e = item * kEdgesPerItem + s * 256 + (int)threadIdx.x;
        valid[s] = e < J.n_edges;
        reg[s] = 0;
        p[s] = q[s] = make_float2(0.0f, 0.0f);
        if (valid[s]) {
            const int2 ab = J.edges[e];
            reg[s] = (unsigned)J.edge_region[e];
            p[s] = J.xy[ab.x];
            q[s] = J.xy[ab.y];
        }
    }
    emit_crossings_warp<kEdgesPerLane>(J, valid, reg, p, q);
}

// Per job, while the keys of an iteration are being emitted (one block):
// clear the pixel counts and the big-row list the row rasteriser fills.
__device__ __forceinline__ void reset_raster_block(const Job& J) {
    if (threadIdx.x == 0) J.st->n_big = 0;
    for (int v = threadIdx.x; v <= J.n_regions; v += blockDim.x) J.counts[v] = 0;
    __syncthreads();
}

// Per job, at the start of a run (one block): empty every row bucket.  The
// row rasteriser empties each bucket it reads, so this only guards against
// an earlier run that stopped on an error between emission and rows.
__device__ __forceinline__ void reset_buckets_block(const Job& J) {
    for (int j = threadIdx.x; j < J.n; j += blockDim.x) J.row_cnt[j] = 0;
    reset_raster_block(J);
}

}  // namespace inim
