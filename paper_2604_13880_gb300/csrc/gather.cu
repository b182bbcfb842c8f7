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

// blocks per SM the register budget aims at: four for FP32 (the sweep's
// chain launches ~4 blocks per SM in one wave), two for the wider sums
template <class Acc>
constexpr int gather_min_blocks() { return sizeof(typename Acc::T) == 4 ? 4 : 2; }

template <class Acc>
__global__ void __launch_bounds__(256, (gather_min_blocks<Acc>())) k_gather_move(const Job* __restrict__ jobs,
                                                                              const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const Job J = jobs[m.x];                  // fixed over a run: read before the wait
    const int v = m.y * blockDim.x + threadIdx.x;
    if constexpr (sizeof(typename Acc::T) == 4) {
        // FP32: the vertex before the wait too (only this kernel writes it,
        // and the previous iteration's move has completed: the kernels in
        // between have passed their waits), so that its corners are known
        // when the wait returns and the active flag, C and the corner sums
        // of the interleaved table go out in one round trip
        const bool has_v = v < J.n_verts;
        const float2 p = has_v ? J.xy[v] : make_float2(0.0f, 0.0f);
        const CornerPos cp = corner_pos(J.n, p);
        pdl_start(J.pdl_early != 0);
        if (!has_v) return;
        if (J.ST) {
            CornerSums<Acc> q[4];
            load_corners<Acc>(J, cp.i0, cp.j0, q);
            const int act = J.st->active;
            const typename Acc::T C = grand_total<Acc>(J);
            if (!act) return;
            tl_begin(J.tl, kTlGather);
            const float2 dlt = displacement_from<Acc>(J, cp, q, C);
            J.xy[v] = make_float2(p.x + J.lam * dlt.x, p.y + J.lam * dlt.y);
            tl_end(J.tl, kTlGather);
        } else {
            const int act = J.st->active;
            const typename Acc::T C = grand_total<Acc>(J);
            if (!act) return;
            tl_begin(J.tl, kTlGather);
            move_vertex<Acc>(J, v, p, C);
            tl_end(J.tl, kTlGather);
        }
    } else {
        // the wider sums of the other precisions: the active flag, the vertex
        // and C in one round trip, then the corners
        pdl_start(J.pdl_early != 0);
        if (v >= J.n_verts) return;
        const int act = J.st->active;
        const float2 p = J.xy[v];
        const typename Acc::T C = grand_total<Acc>(J);
        if (!act) return;
        tl_begin(J.tl, kTlGather);
        move_vertex<Acc>(J, v, p, C);
        tl_end(J.tl, kTlGather);
    }
    pdl_release();
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

// CNN input: mean of log(d / d0) over pool x pool pixel blocks of the label
// texture (the densities are already relative to d0)
__global__ void k_density_pooled(const Job* __restrict__ job, int pool, float* __restrict__ out) {
    const Job& J = *job;
    const int m = J.n / pool;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m * m) return;
    const int bi = q % m, bj = q / m;
    float s = 0.0f;
    for (int dj = 0; dj < pool; ++dj) {
        const uint16_t* row = J.labels + (size_t)(bj * pool + dj) * J.n + bi * pool;
        for (int di = 0; di < pool; ++di) s += logf(fmaxf(J.dens[row[di]], 1e-6f));
    }
    out[q] = s / (float)(pool * pool);
}

// warm start: every vertex moves by the field (m x m cell-centre samples,
// 2 channels, scaled by inv_scale) interpolated bilinearly at its position
__global__ void k_apply_field(const Job* __restrict__ jobs, const int2* __restrict__ bmap, const float* const* fields,
                              int m, float inv_scale) {
    const int2 bm = bmap[blockIdx.x];
    const Job& J = jobs[bm.x];
    const float* f = fields[bm.x];
    if (!f) return;
    const int v = bm.y * blockDim.x + threadIdx.x;
    if (v >= J.n_verts) return;
    float2 p = J.xy[v];
    const float fx = p.x * (float)m - 0.5f, fy = p.y * (float)m - 0.5f;
    const int i0 = min(max((int)floorf(fx), 0), m - 2), j0 = min(max((int)floorf(fy), 0), m - 2);
    const float a = fminf(fmaxf(fx - (float)i0, 0.0f), 1.0f), b = fminf(fmaxf(fy - (float)j0, 0.0f), 1.0f);
    const float* c00 = f + ((size_t)j0 * m + i0) * 2;
    const float* c01 = c00 + 2;
    const float* c10 = c00 + (size_t)m * 2;
    const float* c11 = c10 + 2;
    for (int d = 0; d < 2; ++d) {
        const float val = (1.0f - b) * ((1.0f - a) * c00[d] + a * c01[d]) + b * ((1.0f - a) * c10[d] + a * c11[d]);
        if (d == 0) p.x += inv_scale * val; else p.y += inv_scale * val;
    }
    J.xy[v] = p;
}

}  // namespace

cudaError_t launch_density_pooled(const Job* d_job, int n, int pool, float* out, cudaStream_t s) {
    const int m = n / pool;
    k_density_pooled<<<(m * m + 255) / 256, 256, 0, s>>>(d_job, pool, out);
    return cudaGetLastError();
}

cudaError_t launch_apply_field(const Job* d_jobs, const BlockMap& vert_blocks, const float* const* fields, int m,
                               float inv_scale, cudaStream_t s) {
    if (vert_blocks.n_blocks)
        k_apply_field<<<vert_blocks.n_blocks, 256, 0, s>>>(d_jobs, vert_blocks.d_map, fields, m, inv_scale);
    return cudaGetLastError();
}

cudaError_t launch_gather(const Job* d_jobs, const BlockMap& vert_blocks, int precision, cudaStream_t s) {
    if (!vert_blocks.n_blocks) return cudaSuccess;
    const int2* bm = vert_blocks.d_map;
    if (precision == INIM_FIX64) return launch_pdl(k_gather_move<AccFix>, vert_blocks.n_blocks, 256, 0, s, d_jobs, bm);
    if (precision == INIM_KAHAN) return launch_pdl(k_gather_move<AccKahan>, vert_blocks.n_blocks, 256, 0, s, d_jobs, bm);
    return launch_pdl(k_gather_move<AccF32>, vert_blocks.n_blocks, 256, 0, s, d_jobs, bm);
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
