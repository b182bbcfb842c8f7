// The plain GPU form of one iteration: one unfused kernel per step of the
// static algorithm (Sec. 4.1), every intermediate as a full texture, the field
// precomputed per pixel and interpolated afterwards, exactly in the order the
// paper lists the steps.  It is the comparison point of the fused path and a
// second, independent GPU formulation of the integral images (left wedge by the
// column sweep L(i,j) = L(i-1,j) + D1 + D2 - d instead of the top wedge).
//
//   density   d = dens[label]                                   (step 3)
//   rowscan   R = row prefix of d                               (step 4)
//   colscan   S = column prefix of R
//   diag1     D1(i,j) = d(i,j) + D1(i-1,j-1)
//   diag2     D2(i,j) = d(i,j) + D2(i-1,j+1)
//   lscan     L = row prefix of (D1 + D2 - d)
//   diagsums  anti-diagonal / diagonal sums, then prefix -> A, B
//   field     t(d) - t(d0) per pixel (Eq. 2, Eq. 3)             (step 5)
//   move      bilinear at the vertices, blend, move             (step 6)
#include "inim_internal.cuh"

namespace inim {

namespace {

__global__ void p_density(const Job* __restrict__ job, float* __restrict__ d) {
    const Job& J = *job;
    const size_t np = (size_t)J.n * J.n;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < np; p += (size_t)gridDim.x * blockDim.x)
        d[p] = J.dens[J.labels[p]];
}

// one warp per row: inclusive prefix of src (optionally of a + b - c)
__global__ void p_rowscan(const float* __restrict__ a, const float* __restrict__ b,
                          const float* __restrict__ c, float* __restrict__ out, int n) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float carry = 0.0f;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const size_t p = (size_t)row * n + i0 + lane;
        float v = a[p];
        if (b) v = v + b[p] - c[p];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        v += carry;
        out[p] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

// one thread per column
__global__ void p_colscan(const float* __restrict__ R, float* __restrict__ S, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.0f;
    for (int j = 0; j < n; ++j) {
        acc += R[(size_t)j * n + i];
        S[(size_t)j * n + i] = acc;
    }
}

// one thread per diagonal ray; dir = +1: (i-1, j-1) predecessor, dir = -1: (i-1, j+1)
__global__ void p_diag(const float* __restrict__ d, float* __restrict__ D, int n, int dir) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;   // start index in [0, 2n-1)
    if (q >= 2 * n - 1) return;
    int i, j;
    if (dir > 0) {      // starts on the top row (q < n) or the left column
        if (q < n) { i = q; j = 0; } else { i = 0; j = q - n + 1; }
    } else {            // starts on the bottom row or the left column
        if (q < n) { i = q; j = n - 1; } else { i = 0; j = n - 1 - (q - n + 1); }
    }
    float acc = 0.0f;
    while (i < n && j >= 0 && j < n) {
        acc += d[(size_t)j * n + i];
        D[(size_t)j * n + i] = acc;
        ++i;
        j += dir;
    }
}

// sums along anti-diagonals (i + j = s) and diagonals (i - j = w), one thread each
__global__ void p_diagsums(const float* __restrict__ d, float* __restrict__ ad, float* __restrict__ dd, int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * (2 * n - 1)) return;
    float acc = 0.0f;
    if (q < 2 * n - 1) {
        const int s = q;
        for (int j = max(0, s - n + 1); j <= min(s, n - 1); ++j) acc += d[(size_t)j * n + (s - j)];
        ad[s] = acc;
    } else {
        const int w = q - (2 * n - 1) - (n - 1);      // i - j = w
        for (int j = max(0, -w); j <= min(n - 1, n - 1 - w); ++j) acc += d[(size_t)j * n + (j + w)];
        dd[w + n - 1] = acc;
    }
}

// single block: inclusive prefix of both 1-D arrays (in place)
__global__ void p_prefix2(float* __restrict__ a, float* __restrict__ b, int len) {
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int k = 0; k < len; ++k) { s += a[k]; a[k] = s; }
    } else if (threadIdx.x == 32) {
        float s = 0.0f;
        for (int k = 0; k < len; ++k) { s += b[k]; b[k] = s; }
    }
}

__device__ __forceinline__ float2 eq2_point(float a, float b, float g, float d, float at, float bt,
                                            float gt, float dt, float C, int i, int j, int n) {
    const float inv_n = 1.0f / (float)n;
    const float x = ((float)i + 0.5f) * inv_n, y = ((float)j + 0.5f) * inv_n;
    float tx, ty;
    eq2<float>(a / C, b / C, g / C, d / C, at / C, bt / C, gt / C, dt / C, 1.0f, x, y, tx, ty);
    return make_float2(tx, ty);
}

// step 1: t(.; d0) from the exact counts of a constant texture
__global__ void p_t0(float2* __restrict__ t0, int n) {
    const size_t np = (size_t)n * n;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < np; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % n), j = (int)(p / n);
        const Counts8 c = uniform_counts(i, j, n);
        t0[p] = eq2_point((float)c.a, (float)c.b, (float)c.g, (float)c.d, (float)c.at, (float)c.bt,
                          (float)c.gt, (float)c.dt, (float)c.C, i, j, n);
    }
}

// step 5: displacement per pixel from all eight InIms
__global__ void p_field(const float* __restrict__ S, const float* __restrict__ L, const float* __restrict__ A,
                        const float* __restrict__ B, const float2* __restrict__ t0, float2* __restrict__ fld, int n) {
    const size_t np = (size_t)n * n;
    const float C = S[np - 1];
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < np; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % n), j = (int)(p / n);
        const float a = S[p];
        const float b = S[(size_t)(n - 1) * n + i] - a;
        const float d = S[(size_t)j * n + n - 1] - a;
        const float g = C - a - b - d;
        const float bt = L[p];
        const float at = A[i + j] - bt;
        const float gt = B[i - j + n - 1] - bt;
        const float dt = C - at - bt - gt;
        const float2 t = eq2_point(a, b, g, d, at, bt, gt, dt, C, i, j, n);
        const float2 u = t0[p];
        fld[p] = make_float2(t.x - u.x, t.y - u.y);
    }
}

// step 6: bilinear interpolation of the field at the vertices, blend, move
__global__ void p_move(const Job* __restrict__ job, const float2* __restrict__ fld) {
    const Job& J = *job;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= J.n_verts) return;
    const int n = J.n;
    float2 p = J.xy[v];
    const float fx = p.x * (float)n - 0.5f, fy = p.y * (float)n - 0.5f;
    int i0 = min(max((int)floorf(fx), 0), n - 2);
    int j0 = min(max((int)floorf(fy), 0), n - 2);
    const float a = fminf(fmaxf(fx - (float)i0, 0.0f), 1.0f);
    const float b = fminf(fmaxf(fy - (float)j0, 0.0f), 1.0f);
    const float2 f00 = fld[(size_t)j0 * n + i0], f01 = fld[(size_t)j0 * n + i0 + 1];
    const float2 f10 = fld[(size_t)(j0 + 1) * n + i0], f11 = fld[(size_t)(j0 + 1) * n + i0 + 1];
    const float dx = (1 - b) * ((1 - a) * f00.x + a * f01.x) + b * ((1 - a) * f10.x + a * f11.x);
    const float dy = (1 - b) * ((1 - a) * f00.y + a * f01.y) + b * ((1 - a) * f10.y + a * f11.y);
    p.x += J.lam * dx;
    p.y += J.lam * dy;
    J.xy[v] = p;
}

}  // namespace

cudaError_t plain_alloc(PlainWork& w, int n) {
    const size_t np = (size_t)n * n;
    cudaError_t e = cudaSuccess;
    w.n = n;
    float** tex[] = {&w.d, &w.R, &w.S, &w.D1, &w.D2, &w.L};
    for (float** t : tex) if (e == cudaSuccess) e = cudaMalloc(t, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&w.ad, (2 * n - 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&w.dd, (2 * n - 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&w.t0, np * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&w.fld, np * sizeof(float2));
    if (e == cudaSuccess) {
        p_t0<<<1024, 256>>>(w.t0, n);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    return e;
}

void plain_free(PlainWork& w) {
    void* ptrs[] = {w.d, w.R, w.S, w.D1, w.D2, w.L, w.ad, w.dd, w.t0, w.fld};
    for (void* p : ptrs) if (p) cudaFree(p);
    w = PlainWork{};
}

// everything after the raster and the density table
cudaError_t plain_iteration(const Job* d_job, const Job& h, PlainWork& w, cudaStream_t s) {
    const int n = h.n;
    const int np_blocks = 1024;
    p_density<<<np_blocks, 256, 0, s>>>(d_job, w.d);
    p_rowscan<<<(n + 7) / 8, 256, 0, s>>>(w.d, nullptr, nullptr, w.R, n);
    p_colscan<<<(n + 255) / 256, 256, 0, s>>>(w.R, w.S, n);
    p_diag<<<(2 * n - 1 + 255) / 256, 256, 0, s>>>(w.d, w.D1, n, +1);
    p_diag<<<(2 * n - 1 + 255) / 256, 256, 0, s>>>(w.d, w.D2, n, -1);
    p_rowscan<<<(n + 7) / 8, 256, 0, s>>>(w.D1, w.D2, w.d, w.L, n);
    p_diagsums<<<(2 * (2 * n - 1) + 255) / 256, 256, 0, s>>>(w.d, w.ad, w.dd, n);
    p_prefix2<<<1, 64, 0, s>>>(w.ad, w.dd, 2 * n - 1);
    p_field<<<np_blocks, 256, 0, s>>>(w.S, w.L, w.ad, w.dd, w.t0, w.fld, n);
    p_move<<<(h.n_verts + 255) / 256, 256, 0, s>>>(d_job, w.fld);
    return cudaGetLastError();
}

}  // namespace inim
