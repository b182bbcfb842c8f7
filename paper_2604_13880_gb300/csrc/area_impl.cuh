// Device body of step 7 support (Sec. 4.1, Sec. 3.3): signed shoelace area of every region in
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
#pragma once

#include "raster_common.cuh"

namespace inim {


constexpr int kRegionsPerBlock = 8;

// (hi, lo) += x exactly in hi + err, err accumulated into lo (two-sum)
__device__ __forceinline__ void err_pair_add(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
    hi = s;
}

// The relative errors |o - w| / max(o, w) of the job's regions and their mean
// (eps) and maximum (xi).  Every input is loaded at once (the mass of both
// iteration parities, the state the stop rule reads), the per-region errors
// are FP32 (relative error ~1e-7: this GPU's FP64 divisions are slow) and
// their sum a compensated FP32 pair, reduced in a fixed order.
__device__ inline void errors_and_stop(const Job& J, int update_state) {
    __shared__ float shi[kRegionsPerBlock], slo[kRegionsPerBlock], smax[kRegionsPerBlock];
    __shared__ int sfold[kRegionsPerBlock];
    JobState* st = J.st;
    const int area_it = __ldcg(&st->area_it);
    const double m0 = __ldcg(&st->mass_it[0]), m1 = __ldcg(&st->mass_it[1]);
    // thread 0: what the stop rule reads, loaded with the regions' data
    int iters = 0, max_iters = 0, since = 0, stall = 0, stop_rule = 0, err = 0;
    float xi_stop = 0.0f, eps_stop = 0.0f;
    double best_xi = 0.0;
    if (threadIdx.x == 0 && update_state) {
        iters = __ldcg(&st->iters); max_iters = __ldcg(&st->max_iters); since = __ldcg(&st->since);
        stall = __ldcg(&st->stall_window); stop_rule = __ldcg(&st->stop_on_rule); err = __ldcg(&st->error);
        xi_stop = __ldcg(&st->xi_stop); eps_stop = __ldcg(&st->eps_stop); best_xi = __ldcg(&st->best_xi);
    }
    const double M = (area_it & 1) ? m1 : m0;     // this iteration's raster
    const float inv_m = __frcp_rn((float)M);
    float hi = 0.0f, lo = 0.0f, mx = 0.0f;
    int fold = 0;
    for (int v = threadIdx.x; v < J.n_regions; v += blockDim.x) {
        const double a = __ldcg(J.areas + v);
        const float o = (float)fabs(a);
        const float w = __fmul_rn(J.values[v], inv_m);
        const float den = fmaxf(o, w);
        const float e = den > 0.0f ? __fdiv_rn(fabsf(__fsub_rn(o, w)), den) : 0.0f;
        err_pair_add(hi, lo, e);
        mx = fmaxf(mx, e);
        const float s0 = J.sign0[v];
        if (s0 != 0.0f && ((a > 0.0) != (s0 > 0.0f) || a == 0.0)) fold = 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        err_pair_add(hi, lo, h2);
        lo = __fadd_rn(lo, l2);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        fold |= __shfl_xor_sync(0xffffffffu, fold, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { shi[w] = hi; slo[w] = lo; smax[w] = mx; sfold[w] = fold; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float H = 0.0f, L = 0.0f, X = 0.0f;
        int F = 0;
        for (int k = 0; k < kRegionsPerBlock; ++k) {
            err_pair_add(H, L, shi[k]);
            L = __fadd_rn(L, slo[k]);
            X = fmaxf(X, smax[k]);
            F |= sfold[k];
        }
        const double eps = ((double)H + (double)L) / (double)J.n_regions;
        const double xi = (double)X;
        st->eps = eps;
        st->xi = xi;
        st->area_it = area_it + 1;
        if (F) st->foldover = 1;
        if (update_state) {
            iters += 1;
            st->iters = iters;
            if (xi < best_xi) { st->best_xi = xi; since = 0; }
            else since += 1;
            st->since = since;
            bool stop = iters >= max_iters;
            if (stop_rule) {
                if (xi_stop > 0.0f && xi < (double)xi_stop) stop = true;
                if (eps_stop > 0.0f && eps < (double)eps_stop) stop = true;
                if (stall > 0 && since >= stall) stop = true;
            }
            if (err != 0) stop = true;
            if (stop) st->active = 0;
        }
    }
}

// Compensated FP32 accumulation of one shoelace term x_a y_b - x_b y_a: each
// product is split exactly into p + e (e = fma(x, y, -p)) and summed with
// two-sum into a (hi, lo) pair.
__device__ __forceinline__ void shoelace_add(float& hi, float& lo, float2 p, float2 q) {
    const float p1 = __fmul_rn(p.x, q.y), e1p = __fmaf_rn(p.x, q.y, -p1);
    const float p2 = __fmul_rn(q.x, p.y), e2p = __fmaf_rn(q.x, p.y, -p2);
    float s = __fadd_rn(hi, p1);
    float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p1, bb)), e1p));
    hi = s;
    s = __fadd_rn(hi, -p2);
    bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fsub_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(-p2, bb)), e2p));
    hi = s;
}

// The mesh part of one warp's work, fixed over a run and so read before the
// programmatic-launch wait: the region, the lane's first edge, the region's
// end and the lane's first four edges.
struct AreaPre {
    int v, wr, e, e1;
    int2 ab[4];
};

// A block (8 warps) holds 8 >> lw regions, 1 << lw warps each; a warp's lanes
// take every (32 << lw)-th edge of the region.
__device__ __forceinline__ AreaPre areas_prefetch(const Job& J, int item) {
    AreaPre a;
    const int lw = area_warps_log2(J.n_edges, J.n_regions);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stride = 32 << lw;
    a.v = item * (kRegionsPerBlock >> lw) + (warp >> lw);
    a.wr = warp & ((1 << lw) - 1);
    a.e = 0;
    a.e1 = 0;
    if (a.v < J.n_regions) {
        a.e1 = J.reg_edge_off[a.v + 1];
        a.e = J.reg_edge_off[a.v] + a.wr * 32 + lane;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        a.ab[u] = (a.e + u * stride < a.e1) ? __ldg(J.edges + a.e + u * stride) : make_int2(0, 0);
    return a;
}

// update_state: 1 = errors + stop rule, 0 = errors only, -1 = areas only.
// Edges go in groups of four, in order; the next group's edges are loaded
// while the current group's vertices are in flight.  check_active: the job's
// active flag is read with the first vertices (one round trip) and a stopped
// job's block leaves (the same in every thread of the block).
__device__ inline void areas_body(const Job& J, int item, int update_state, const AreaPre& pre,
                                  bool check_active = false) {
    __shared__ double wpart[kRegionsPerBlock];
    const int lw = area_warps_log2(J.n_edges, J.n_regions);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = pre.v, wr = pre.wr;
    const int act = check_active ? J.st->active : 1;
    double acc = 0.0;
    if (v < J.n_regions) {
        float hi = 0.0f, lo = 0.0f;
        const int e1 = pre.e1;
        const int stride = 32 << lw;
        int2 ab[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ab[u] = pre.ab[u];
        for (int e = pre.e; e < e1; e += 4 * stride) {
            float2 p[4], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                p[u] = q[u] = make_float2(0.0f, 0.0f);
                if (e + u * stride < e1) { p[u] = J.xy[ab[u].x]; q[u] = J.xy[ab[u].y]; }
            }
            if (!act) break;
            const int en = e + 4 * stride;
#pragma unroll
            for (int u = 0; u < 4; ++u) ab[u] = (en + u * stride < e1) ? __ldg(J.edges + en + u * stride) : ab[u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e + u * stride < e1) shoelace_add(hi, lo, p[u], q[u]);
        }
        acc = (double)hi + (double)lo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    if (!act) return;
    if (lane == 0) wpart[warp] = acc;
    __syncthreads();
    if (v < J.n_regions && wr == 0 && lane == 0) {
        double a = 0.0;
        for (int k = 0; k < (1 << lw); ++k) a += wpart[warp + k];      // fixed order
        J.areas[v] = 0.5 * a;
    }
    if (update_state < 0) return;
    // the last block of this job reduces the errors
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int rpb = kRegionsPerBlock >> area_warps_log2(J.n_edges, J.n_regions);
        const int nblk = (J.n_regions + rpb - 1) / rpb;
        const int ticket = atomicAdd(&J.st->blocks_done, 1);
        last = (ticket == nblk - 1);
        if (last) J.st->blocks_done = 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    errors_and_stop(J, update_state);
}

__device__ __forceinline__ void areas_item(const Job& J, int item, int update_state) {
    areas_body(J, item, update_state, areas_prefetch(J, item));
}

}  // namespace inim
