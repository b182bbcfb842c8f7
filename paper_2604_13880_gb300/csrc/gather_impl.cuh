// Device bodies of steps 5-6 of the static algorithm (Sec. 4.1): the displacement
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
#pragma once

#include "scan_impl.cuh"

namespace inim {


struct Ratios { float a, b, g, d, at, bt, gt, dt; };

// The eight sums at pixel (i, j) from S, T and the 1-D arrays (Eq. 1),
// formed in the accumulator type, as ratios to C (inv_c = 1 / C).
template <class Acc>
__device__ __forceinline__ Ratios corner_ratios(const Job& J, int i, int j, typename Acc::T C, double inv_c) {
    using T = typename Acc::T;
    const int n = J.n;
    const T* A = reinterpret_cast<const T*>(J.A);
    const T* B = reinterpret_cast<const T*>(J.B);
    const T* RC = reinterpret_cast<const T*>(J.rowcum);
    T a, at, colcum;
    if (J.ST) {
        const T* ST = reinterpret_cast<const T*>(J.ST);
        const size_t p = 2 * ((size_t)j * n + i);
        a = ST[p];
        at = ST[p + 1];
        colcum = ST[2 * ((size_t)(n - 1) * n + i)];
    } else {
        const T* S = reinterpret_cast<const T*>(J.S);
        a = S[(size_t)j * n + i];
        at = reinterpret_cast<const T*>(J.T)[(size_t)j * n + i];
        colcum = S[(size_t)(n - 1) * n + i];
    }
    const T b = Acc::sub(colcum, a);
    const T d = Acc::sub(RC[j], a);
    const T g = Acc::sub(Acc::sub(Acc::sub(C, a), b), d);
    const T bt = Acc::sub(A[i + j], at);
    const int w = i - j;
    const T Bw = (w <= 0) ? B[w + n - 1] : Acc::sub(C, B[w + n - 1]);
    const T gt = Acc::sub(Bw, bt);
    const T dt = Acc::sub(Acc::sub(Acc::sub(C, at), bt), gt);
    Ratios r;
    r.a = Acc::scale(a, inv_c); r.b = Acc::scale(b, inv_c); r.g = Acc::scale(g, inv_c); r.d = Acc::scale(d, inv_c);
    r.at = Acc::scale(at, inv_c); r.bt = Acc::scale(bt, inv_c); r.gt = Acc::scale(gt, inv_c);
    r.dt = Acc::scale(dt, inv_c);
    return r;
}

// #{(i', j') in [0,n)^2 : i' + j' <= s} in 32-bit integers (n <= 4096)
__device__ __forceinline__ int anti_count32(int s, int n) {
    if (s < 0) return 0;
    if (s >= 2 * n - 2) return n * n;
    if (s <= n - 1) return ((s + 1) * (s + 2)) >> 1;
    const int m = 2 * n - 3 - s;
    return n * n - (((m + 1) * (m + 2)) >> 1);
}

// The same eight sums for a constant texture (exact pixel counts, t(.; d0)),
// as ratios to C0 = N^2 = 2^(2k): an exact power-of-two scaling.
__device__ __forceinline__ Ratios uniform_ratios(int i, int j, int n, float inv_c0) {
    const int a = (i + 1) * (j + 1);
    const int b = (i + 1) * (n - 1 - j);
    const int g = (n - 1 - i) * (n - 1 - j);
    const int d = (n - 1 - i) * (j + 1);
    const int m = i + 1;
    const int k1 = min(i, j), k2 = min(i, n - 1 - j);
    const int L = m + (k1 * m - ((k1 * (k1 + 1)) >> 1)) + (k2 * m - ((k2 * (k2 + 1)) >> 1));
    const int at = anti_count32(i + j, n) - L;
    const int gt = anti_count32(i - j + n - 1, n) - L;
    const int dt = n * n - L - at - gt;
    Ratios r;
    r.a = (float)a * inv_c0; r.b = (float)b * inv_c0; r.g = (float)g * inv_c0; r.d = (float)d * inv_c0;
    r.at = (float)at * inv_c0; r.bt = (float)L * inv_c0; r.gt = (float)gt * inv_c0; r.dt = (float)dt * inv_c0;
    return r;
}

// Eq. (3) at one pixel: t(d) - t(d0) = Eq. (2) applied to the difference of
// the weights (Eq. 2 is linear in the eight weights for fixed anchors).
__device__ __forceinline__ float2 delta_at_pixel(const Ratios& r, const Ratios& r0, int i, int j, float inv_n) {
    const float x = ((float)i + 0.5f) * inv_n, y = ((float)j + 0.5f) * inv_n;
    float tx, ty;
    eq2<float>(r.a - r0.a, r.b - r0.b, r.g - r0.g, r.d - r0.d, r.at - r0.at, r.bt - r0.bt, r.gt - r0.gt,
               r.dt - r0.dt, 1.0f, x, y, tx, ty);
    return make_float2(tx, ty);
}

// C = the grand total (the last element of S)
template <class Acc>
__device__ __forceinline__ typename Acc::T grand_total(const Job& J) {
    using T = typename Acc::T;
    const size_t last = (size_t)J.n * J.n - 1;
    return J.ST ? reinterpret_cast<const T*>(J.ST)[2 * last] : reinterpret_cast<const T*>(J.S)[last];
}

// The sums that Eq. (1) turns into the eight InIms at one pixel: S and T at
// the pixel, S at the bottom of its column, S at the end of its row, A(i+j)
// and the stored B entry of w = i - j.
template <class Acc>
struct CornerSums {
    typename Acc::T a, at, colcum, rc, A, Braw;
};

// corner_ratios from sums already loaded (the same arithmetic)
template <class Acc>
__device__ __forceinline__ Ratios ratios_from(const CornerSums<Acc>& q, int w, typename Acc::T C, double inv_c) {
    using T = typename Acc::T;
    const T b = Acc::sub(q.colcum, q.a);
    const T d = Acc::sub(q.rc, q.a);
    const T g = Acc::sub(Acc::sub(Acc::sub(C, q.a), b), d);
    const T bt = Acc::sub(q.A, q.at);
    const T Bw = (w <= 0) ? q.Braw : Acc::sub(C, q.Braw);
    const T gt = Acc::sub(Bw, bt);
    const T dt = Acc::sub(Acc::sub(Acc::sub(C, q.at), bt), gt);
    Ratios r;
    r.a = Acc::scale(q.a, inv_c); r.b = Acc::scale(b, inv_c); r.g = Acc::scale(g, inv_c); r.d = Acc::scale(d, inv_c);
    r.at = Acc::scale(q.at, inv_c); r.bt = Acc::scale(bt, inv_c); r.gt = Acc::scale(gt, inv_c);
    r.dt = Acc::scale(dt, inv_c);
    return r;
}

// Two horizontally adjacent (S, T) pairs of the interleaved table starting at
// element p = 2 (j n + i): one 16-byte load when p is a multiple of 4 (FP32,
// i even), else two 8-byte loads; 64-bit and compensated pairs are 16 bytes
// each.
template <class T>
__device__ __forceinline__ void load_two_pairs(const T* ST, size_t p, T& s0, T& t0, T& s1, T& t1) {
    if constexpr (sizeof(T) == 4) {
        if ((p & 3) == 0) {
            const float4 v = *reinterpret_cast<const float4*>(ST + p);
            s0 = v.x; t0 = v.y; s1 = v.z; t1 = v.w;
        } else {
            const float2 u = *reinterpret_cast<const float2*>(ST + p);
            const float2 v = *reinterpret_cast<const float2*>(ST + p + 2);
            s0 = u.x; t0 = u.y; s1 = v.x; t1 = v.y;
        }
    } else {
        const uint4 u = *reinterpret_cast<const uint4*>(ST + p);
        const uint4 v = *reinterpret_cast<const uint4*>(ST + p + 2);
        s0 = *reinterpret_cast<const T*>(&u.x); t0 = *reinterpret_cast<const T*>(&u.z);
        s1 = *reinterpret_cast<const T*>(&v.x); t1 = *reinterpret_cast<const T*>(&v.z);
    }
}

// The sums of the four corners (i0, j0), (i0 + 1, j0), (i0, j0 + 1),
// (i0 + 1, j0 + 1) from the interleaved table, loaded together: two
// 16-byte rows of (S, T) pairs, the two column ends, the two row ends, three
// consecutive A and three consecutive B entries.
template <class Acc>
__device__ __forceinline__ void load_corners(const Job& J, int i0, int j0, CornerSums<Acc> (&q)[4]) {
    using T = typename Acc::T;
    const int n = J.n;
    const T* ST = reinterpret_cast<const T*>(J.ST);
    const T* A = reinterpret_cast<const T*>(J.A);
    const T* B = reinterpret_cast<const T*>(J.B);
    const T* RC = reinterpret_cast<const T*>(J.rowcum);
    const size_t p0 = 2 * ((size_t)j0 * n + i0);
    const size_t pc = 2 * ((size_t)(n - 1) * n + i0);
    T dummy0, dummy1;
    load_two_pairs<T>(ST, p0, q[0].a, q[0].at, q[1].a, q[1].at);
    load_two_pairs<T>(ST, p0 + 2 * (size_t)n, q[2].a, q[2].at, q[3].a, q[3].at);
    load_two_pairs<T>(ST, pc, q[0].colcum, dummy0, q[1].colcum, dummy1);
    q[2].colcum = q[0].colcum;
    q[3].colcum = q[1].colcum;
    q[0].rc = q[1].rc = RC[j0];
    q[2].rc = q[3].rc = RC[j0 + 1];
    const int s = i0 + j0;
    q[0].A = A[s];
    q[1].A = q[2].A = A[s + 1];
    q[3].A = A[s + 2];
    const int w0 = i0 - j0 + n - 1;             // stored index of w = i0 - j0
    q[0].Braw = q[3].Braw = B[w0];
    q[1].Braw = B[w0 + 1];
    q[2].Braw = B[w0 - 1];
}

// #{(i', j') : i' + j' <= s} (anti_count32) in FP32: every count is an
// integer below 2^24 + 1, so the arithmetic is exact
__device__ __forceinline__ float anti_count_f(int s, int n, float nn) {
    if (s < 0) return 0.0f;
    if (s >= 2 * n - 2) return nn;
    if (s <= n - 1) return (float)(((s + 1) * (s + 2)) >> 1);
    const int m = 2 * n - 3 - s;
    return nn - (float)(((m + 1) * (m + 2)) >> 1);
}

// uniform_ratios of the four corners (i0, j0), (i0 + 1, j0), (i0, j0 + 1),
// (i0 + 1, j0 + 1) with their shared factors and the three distinct values
// of each diagonal count computed once; exact integer counts in FP32, then
// the power-of-two scaling (the same values as uniform_ratios)
__device__ __forceinline__ void uniform_ratios4(int i0, int j0, int n, float inv_c0, Ratios (&r0)[4]) {
    const float nn = (float)n * (float)n;
    const float I[2] = {(float)(i0 + 1), (float)(i0 + 2)};              // i + 1
    const float Ni[2] = {(float)(n - 1 - i0), (float)(n - 2 - i0)};     // n - 1 - i
    const float Jp[2] = {(float)(j0 + 1), (float)(j0 + 2)};             // j + 1
    const float Nj[2] = {(float)(n - 1 - j0), (float)(n - 2 - j0)};     // n - 1 - j
    float A3[3], B3[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        A3[q] = anti_count_f(i0 + j0 + q, n, nn);                        // i + j = i0 + j0 + q
        B3[q] = anti_count_f(i0 - j0 + n - 2 + q, n, nn);                // i - j + n - 1, q = di - dj + 1
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int di = c & 1, dj = c >> 1;
        const int i = i0 + di, j = j0 + dj;
        const float a = I[di] * Jp[dj], b = I[di] * Nj[dj], g = Ni[di] * Nj[dj], d = Ni[di] * Jp[dj];
        const int m = i + 1;
        const int k1 = min(i, j), k2 = min(i, n - 1 - j);
        const float L = (float)(m + (k1 * m - ((k1 * (k1 + 1)) >> 1)) + (k2 * m - ((k2 * (k2 + 1)) >> 1)));
        const float at = A3[di + dj] - L;
        const float gt = B3[di - dj + 1] - L;
        const float dt = nn - L - at - gt;
        Ratios& r = r0[c];
        r.a = a * inv_c0; r.b = b * inv_c0; r.g = g * inv_c0; r.d = d * inv_c0;
        r.at = at * inv_c0; r.bt = L * inv_c0; r.gt = gt * inv_c0; r.dt = dt * inv_c0;
    }
}

// The pixel (i0, j0) whose centre is the top-left of the four around p (kept
// inside the texture) and p's bilinear weights (a, b) towards i0 + 1, j0 + 1.
struct CornerPos {
    int i0, j0;
    float a, b;
};

__device__ __forceinline__ CornerPos corner_pos(int n, float2 p) {
    const float fx = p.x * (float)n - 0.5f;
    const float fy = p.y * (float)n - 0.5f;
    CornerPos c;
    c.i0 = min(max((int)floorf(fx), 0), n - 2);
    c.j0 = min(max((int)floorf(fy), 0), n - 2);
    c.a = fminf(fmaxf(fx - (float)c.i0, 0.0f), 1.0f);
    c.b = fminf(fmaxf(fy - (float)c.j0, 0.0f), 1.0f);
    return c;
}

__device__ __forceinline__ float2 bilinear(const float2 (&f)[4], float a, float b) {
    const float2 top = make_float2((1.0f - a) * f[0].x + a * f[1].x, (1.0f - a) * f[0].y + a * f[1].y);
    const float2 bot = make_float2((1.0f - a) * f[2].x + a * f[3].x, (1.0f - a) * f[2].y + a * f[3].y);
    return make_float2((1.0f - b) * top.x + b * bot.x, (1.0f - b) * top.y + b * bot.y);
}

// The displacement from the interleaved table's corner sums already loaded.
template <class Acc>
__device__ __forceinline__ float2 displacement_from(const Job& J, const CornerPos& cp, const CornerSums<Acc> (&q)[4],
                                                    typename Acc::T C) {
    const int n = J.n;
    const double inv_c = Acc::inv(C);
    const float inv_n = 1.0f / (float)n;
    const float inv_c0 = ldexpf(1.0f, -2 * J.log2n);
    Ratios r0[4];
    uniform_ratios4(cp.i0, cp.j0, n, inv_c0, r0);
    float2 f[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int i = cp.i0 + (c & 1), j = cp.j0 + (c >> 1);
        f[c] = delta_at_pixel(ratios_from<Acc>(q[c], i - j, C, inv_c), r0[c], i, j, inv_n);
    }
    return bilinear(f, cp.a, cp.b);
}

template <class Acc>
__device__ __forceinline__ float2 displacement_at_c(const Job& J, float2 p, typename Acc::T C) {
    const int n = J.n;
    const CornerPos cp = corner_pos(n, p);
    if (J.ST) {
        CornerSums<Acc> q[4];
        load_corners<Acc>(J, cp.i0, cp.j0, q);
        return displacement_from<Acc>(J, cp, q, C);
    }
    const double inv_c = Acc::inv(C);
    const float inv_n = 1.0f / (float)n;
    const float inv_c0 = ldexpf(1.0f, -2 * J.log2n);
    float2 f[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int i = cp.i0 + (c & 1), j = cp.j0 + (c >> 1);
        f[c] = delta_at_pixel(corner_ratios<Acc>(J, i, j, C, inv_c), uniform_ratios(i, j, n, inv_c0), i, j, inv_n);
    }
    return bilinear(f, cp.a, cp.b);
}

template <class Acc>
__device__ __forceinline__ float2 displacement_at(const Job& J, float2 p) {
    return displacement_at_c<Acc>(J, p, grand_total<Acc>(J));
}

// the blend of Sec. 4.1 step 6 and the move, from the vertex p and C loaded
template <class Acc>
__device__ __forceinline__ void move_vertex(const Job& J, int v, float2 p, typename Acc::T C) {
    const float2 dlt = displacement_at_c<Acc>(J, p, C);
    p.x += J.lam * dlt.x;
    p.y += J.lam * dlt.y;
    J.xy[v] = p;
}

template <class Acc>
__device__ __forceinline__ void gather_vertex(const Job& J, int v) {
    if (v >= J.n_verts) return;
    move_vertex<Acc>(J, v, J.xy[v], grand_total<Acc>(J));
}

}  // namespace inim
