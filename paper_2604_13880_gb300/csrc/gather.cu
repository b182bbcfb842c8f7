// Steps 5-6 of the static algorithm (Sec. 4.1): the displacement
// t(x, y; d) - t(x, y; d0) of Eq. (3) at the four pixel centres around every
// vertex, bilinear interpolation, the shape blend and the move.
//
// Per corner pixel (i, j) the eight InIms come from S, T and the 1-D arrays
// through Eq. (1) (see scan_impl.cuh); differences are formed in the
// accumulator type (exact for FIX64, compensated for KAHAN), then turned into
// ratios to C and fed to Eq. (2) in float.  t(.; d0) uses the exact pixel
// counts of a constant texture (closed form), through the same Eq. (2) code,
// so that a constant texture gives exactly zero displacement.
#include "scan_impl.cuh"

namespace inim {

namespace {

struct Ratios { float a, b, g, d, at, bt, gt, dt; };

template <class Acc>
__device__ __forceinline__ Ratios corner_ratios(const Job& J, int i, int j) {
    using T = typename Acc::T;
    const int n = J.n;
    const T* S = reinterpret_cast<const T*>(J.S);
    const T* Tt = reinterpret_cast<const T*>(J.T);
    const T* A = reinterpret_cast<const T*>(J.A);
    const T* B = reinterpret_cast<const T*>(J.B);
    const T* RC = reinterpret_cast<const T*>(J.rowcum);
    const T C = S[(size_t)(n - 1) * n + (n - 1)];
    const T a = S[(size_t)j * n + i];
    const T colcum = S[(size_t)(n - 1) * n + i];
    const T rowcum = RC[j];
    const T b = Acc::sub(colcum, a);
    const T d = Acc::sub(rowcum, a);
    const T g = Acc::sub(Acc::sub(Acc::sub(C, a), b), d);
    const T at = Tt[(size_t)j * n + i];
    const T bt = Acc::sub(A[i + j], at);
    const int w = i - j;
    const T Bw = (w <= 0) ? B[w + n - 1] : Acc::sub(C, B[w + n - 1]);
    const T gt = Acc::sub(Bw, bt);
    const T dt = Acc::sub(Acc::sub(Acc::sub(C, at), bt), gt);
    Ratios r;
    r.a = Acc::ratio(a, C); r.b = Acc::ratio(b, C); r.g = Acc::ratio(g, C); r.d = Acc::ratio(d, C);
    r.at = Acc::ratio(at, C); r.bt = Acc::ratio(bt, C); r.gt = Acc::ratio(gt, C); r.dt = Acc::ratio(dt, C);
    return r;
}

// uniform texture: ratios of the exact pixel counts (same code path shape)
__device__ __forceinline__ Ratios uniform_ratios(int i, int j, int n, int precision) {
    Counts8 c = uniform_counts(i, j, n);
    Ratios r;
    if (precision == INIM_FP32) {
        const float C = (float)c.C;
        r.a = (float)c.a / C; r.b = (float)c.b / C; r.g = (float)c.g / C; r.d = (float)c.d / C;
        r.at = (float)c.at / C; r.bt = (float)c.bt / C; r.gt = (float)c.gt / C; r.dt = (float)c.dt / C;
    } else {
        const double C = (double)c.C;
        r.a = (float)((double)c.a / C); r.b = (float)((double)c.b / C);
        r.g = (float)((double)c.g / C); r.d = (float)((double)c.d / C);
        r.at = (float)((double)c.at / C); r.bt = (float)((double)c.bt / C);
        r.gt = (float)((double)c.gt / C); r.dt = (float)((double)c.dt / C);
    }
    return r;
}

__device__ __forceinline__ float2 eq2_ratios(const Ratios& r, int i, int j, int n) {
    const float inv_n = 1.0f / (float)n;
    const float x = ((float)i + 0.5f) * inv_n, y = ((float)j + 0.5f) * inv_n;
    float tx, ty;
    eq2<float>(r.a, r.b, r.g, r.d, r.at, r.bt, r.gt, r.dt, 1.0f, x, y, tx, ty);
    return make_float2(tx, ty);
}

template <class Acc>
__device__ __forceinline__ float2 displacement_at(const Job& J, float2 p) {
    const int n = J.n;
    const float fx = p.x * (float)n - 0.5f;
    const float fy = p.y * (float)n - 0.5f;
    int i0 = (int)floorf(fx), j0 = (int)floorf(fy);
    i0 = min(max(i0, 0), n - 2);
    j0 = min(max(j0, 0), n - 2);
    const float a = fminf(fmaxf(fx - (float)i0, 0.0f), 1.0f);
    const float b = fminf(fmaxf(fy - (float)j0, 0.0f), 1.0f);
    float2 f[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int i = i0 + (c & 1), j = j0 + (c >> 1);
        const float2 t = eq2_ratios(corner_ratios<Acc>(J, i, j), i, j, n);
        const float2 t0 = eq2_ratios(uniform_ratios(i, j, n, J.precision), i, j, n);
        f[c] = make_float2(t.x - t0.x, t.y - t0.y);
    }
    const float2 top = make_float2((1.0f - a) * f[0].x + a * f[1].x, (1.0f - a) * f[0].y + a * f[1].y);
    const float2 bot = make_float2((1.0f - a) * f[2].x + a * f[3].x, (1.0f - a) * f[2].y + a * f[3].y);
    return make_float2((1.0f - b) * top.x + b * bot.x, (1.0f - b) * top.y + b * bot.y);
}

template <class Acc>
__global__ void __launch_bounds__(256) k_gather_move(const Job* __restrict__ jobs,
                                                     const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const Job& J = jobs[m.x];
    if (!J.st->active) return;
    const int v = m.y * blockDim.x + threadIdx.x;
    if (v >= J.n_verts) return;
    float2 p = J.xy[v];
    const float2 dlt = displacement_at<Acc>(J, p);
    p.x += J.lam * dlt.x;
    p.y += J.lam * dlt.y;
    J.xy[v] = p;
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
    const T* S = reinterpret_cast<const T*>(job->S);
    const T C = S[(size_t)(n - 1) * n + (n - 1)];
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
