// Geographic quality measures of a cartogram against its original map
// (Sec. 3.3), on the label rasters of both (background = n_regions) and on
// their vertex arrays:
//   topology distortion  tau = 1 - |E_c & E_m| / |E_c | E_m| over region
//                        adjacencies (4-neighbouring pixels of two regions),
//                        kept as R x R bitmaps (bit u R + v, u < v);
//   shape distortion     per region, the normalised symmetric difference of
//                        its two pixel sets minimised over whole-pixel
//                        translations = (|m| + |c| - 2 o) / (|m| + |c| - o) at
//                        the largest overlap o, found by brute force over
//                        every translation of the region's bit-packed
//                        bounding-box masks (one thread per translation);
//   relative position    R = 1 / (pi |V| (|V| - 1)) sum over ordered pairs of
//   error                the angle between the pair's barycentre vectors in
//                        the cartogram and in the map; barycentres are the
//                        area centroids of the region polygons (shoelace
//                        moments in double).
// The host part (raster, workspace, bounding-box layout) is inim_quality.
#include <climits>

#include "inim_internal.cuh"

namespace inim {

namespace {

constexpr int kQThreads = kQualityChunk;   // one translation a thread in k_correlate

// marks the pair (a, b) of different regions in the bitmap (read first: most
// boundary pixels repeat a pair that is already set)
__device__ __forceinline__ void mark_pair(uint32_t* bits, int R, int a, int b) {
    if (b >= R || b == a) return;
    const unsigned long long k = (unsigned long long)min(a, b) * (unsigned long long)R + (unsigned long long)max(a, b);
    const uint32_t m = 1u << (k & 31);
    uint32_t* w = bits + (k >> 5);
    if (!(__ldcg(w) & m)) atomicOr(w, m);
}

__global__ void __launch_bounds__(kQThreads) k_adjacency(const uint16_t* __restrict__ lab, int log2n, int R,
                                                         uint32_t* __restrict__ bits) {
    const int n = 1 << log2n;
    const long long p = (long long)blockIdx.x * kQThreads + threadIdx.x;
    if (p >= (long long)n * n) return;
    const int i = (int)(p & (n - 1)), j = (int)(p >> log2n);
    const int a = lab[p];
    if (a >= R) return;
    if (i + 1 < n) mark_pair(bits, R, a, lab[p + 1]);
    if (j + 1 < n) mark_pair(bits, R, a, lab[p + n]);
}

// out[0..3] += popcount of a, b, a & b, a | b
__global__ void __launch_bounds__(kQThreads) k_pair_counts(const uint32_t* __restrict__ a,
                                                           const uint32_t* __restrict__ b, long long nw,
                                                           unsigned long long* __restrict__ out) {
    unsigned long long c[4] = {0, 0, 0, 0};
    for (long long w = (long long)blockIdx.x * kQThreads + threadIdx.x; w < nw; w += (long long)gridDim.x * kQThreads) {
        const uint32_t x = a[w], y = b[w];
        c[0] += __popc(x);
        c[1] += __popc(y);
        c[2] += __popc(x & y);
        c[3] += __popc(x | y);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int k = 16; k > 0; k >>= 1) c[q] += __shfl_xor_sync(0xffffffffu, c[q], k);
        if ((threadIdx.x & 31) == 0 && c[q]) atomicAdd(out + q, c[q]);
    }
}

__global__ void k_fill_box(int* box, int R) {
    const int v = blockIdx.x * kQThreads + threadIdx.x;
    if (v >= R) return;
    box[4 * v + 0] = INT_MAX;
    box[4 * v + 1] = -1;
    box[4 * v + 2] = INT_MAX;
    box[4 * v + 3] = -1;
}

// box[v] = (x_min, x_max, y_min, y_max) of region v's pixels; an extreme
// pixel always has a neighbour of another label (or the texture edge) on
// that side, so only such pixels update it
__global__ void __launch_bounds__(kQThreads) k_bbox(const uint16_t* __restrict__ lab, int log2n, int R,
                                                    int* __restrict__ box) {
    const int n = 1 << log2n;
    const long long p = (long long)blockIdx.x * kQThreads + threadIdx.x;
    if (p >= (long long)n * n) return;
    const int i = (int)(p & (n - 1)), j = (int)(p >> log2n);
    const int v = lab[p];
    if (v >= R) return;
    if (i == 0 || lab[p - 1] != v) atomicMin(box + 4 * v + 0, i);
    if (i == n - 1 || lab[p + 1] != v) atomicMax(box + 4 * v + 1, i);
    if (j == 0 || lab[p - n] != v) atomicMin(box + 4 * v + 2, j);
    if (j == n - 1 || lab[p + n] != v) atomicMax(box + 4 * v + 3, j);
}

// region v's pixels of raster `which` as bits of its bounding-box mask
// (row-major, W words a row); regions without a layout (W = 0) are skipped
__global__ void __launch_bounds__(kQThreads) k_pack(const uint16_t* __restrict__ lab, int log2n, int R,
                                                    const QRegion* __restrict__ reg, int which,
                                                    uint32_t* __restrict__ masks) {
    const int n = 1 << log2n;
    const long long p = (long long)blockIdx.x * kQThreads + threadIdx.x;
    if (p >= (long long)n * n) return;
    const int v = lab[p];
    if (v >= R) return;
    const int W = reg[v].W[which];
    if (W == 0) return;
    const int x = (int)(p & (n - 1)) - reg[v].x0[which], y = (int)(p >> log2n) - reg[v].y0[which];
    atomicOr(masks + reg[v].off[which] + (long long)y * W + (x >> 5), 1u << (x & 31));
}

// One thread per translation (dx, dy) of the cartogram mask against the map
// mask: o = sum over rows y of popcount(M[y] & C[y + dy] shifted by dx);
// items[b] = (region, chunk of kQThreads translations).  The block's largest
// overlap goes to omax[region].
__global__ void __launch_bounds__(kQThreads) k_correlate(const int2* __restrict__ items,
                                                         const QRegion* __restrict__ reg,
                                                         const uint32_t* __restrict__ mm,
                                                         const uint32_t* __restrict__ mc, int* __restrict__ omax) {
    const int2 it = items[blockIdx.x];
    const QRegion g = reg[it.x];
    const int wm = g.w[0], hm = g.h[0], wc = g.w[1], hc = g.h[1], Wm = g.W[0], Wc = g.W[1];
    const int nx = wm + wc - 1;
    const long long ntr = (long long)nx * (hm + hc - 1);
    const long long t = (long long)it.y * kQThreads + threadIdx.x;
    int o = 0;
    if (t < ntr) {
        const int dx = (int)(t % nx) - (wm - 1), dy = (int)(t / nx) - (hm - 1);
        const int y_lo = max(0, -dy), y_hi = min(hm, hc - dy);
        for (int y = y_lo; y < y_hi; ++y) {
            const uint32_t* mr = mm + g.off[0] + (long long)y * Wm;
            const uint32_t* cr = mc + g.off[1] + (long long)(y + dy) * Wc;
            for (int k = 0; k < Wm; ++k) {
                const int s = 32 * k + dx;            // cartogram column under bit 0 of word k
                const int w0 = s >> 5;                // floor(s / 32)
                const uint32_t lo = (w0 >= 0 && w0 < Wc) ? __ldg(cr + w0) : 0u;
                const uint32_t hi = (w0 + 1 >= 0 && w0 + 1 < Wc) ? __ldg(cr + w0 + 1) : 0u;
                o += __popc(__ldg(mr + k) & __funnelshift_r(lo, hi, s & 31));
            }
        }
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) o = max(o, __shfl_xor_sync(0xffffffffu, o, k));
    if ((threadIdx.x & 31) == 0 && o > 0) atomicMax(omax + it.x, o);
}

// per-region shape distortion (1 for a region missing from either raster)
// and out = (sum over regions present in both, their number); one block
__global__ void __launch_bounds__(1024) k_shape_final(const int* __restrict__ cm, const int* __restrict__ cc,
                                                      const int* __restrict__ omax, int R, double* __restrict__ per,
                                                      double* __restrict__ out) {
    __shared__ double ws[32];
    __shared__ int wc[32];
    double s = 0.0;
    int c = 0;
    for (int v = threadIdx.x; v < R; v += 1024) {
        const int am = cm[v], ac = cc[v];
        double val = 1.0;
        if (am > 0 && ac > 0) {
            const int o = omax[v];
            val = (double)(am + ac - 2 * o) / (double)(am + ac - o);
            s += val;
            c += 1;
        }
        per[v] = val;
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, k);
        c += __shfl_xor_sync(0xffffffffu, c, k);
    }
    if ((threadIdx.x & 31) == 0) { ws[threadIdx.x >> 5] = s; wc[threadIdx.x >> 5] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int m = 0;
        for (int w = 0; w < 32; ++w) { t += ws[w]; m += wc[w]; }
        out[0] = t;
        out[1] = (double)m;
    }
}

// area centroid of every region: one warp per region over all its rings,
// C = sum (p + q) cross(p, q) / (3 sum cross(p, q))
__global__ void __launch_bounds__(kQThreads) k_barycentres(const int* __restrict__ reg_ring_off,
                                                           const int* __restrict__ reg_rings,
                                                           const int* __restrict__ ring_off,
                                                           const int* __restrict__ ring_idx,
                                                           const float2* __restrict__ xy, int R,
                                                           double2* __restrict__ bary) {
    const int v = (int)((blockIdx.x * kQThreads + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (v >= R) return;                                   // uniform over the warp
    double a2 = 0.0, cx = 0.0, cy = 0.0;
    for (int q = reg_ring_off[v]; q < reg_ring_off[v + 1]; ++q) {
        const int r = reg_rings[q];
        const int b = ring_off[r], len = ring_off[r + 1] - b;
        for (int k = lane; k < len; k += 32) {
            const float2 p = xy[ring_idx[b + k]];
            const float2 nq = xy[ring_idx[b + (k + 1 == len ? 0 : k + 1)]];
            const double px = p.x, py = p.y, qx = nq.x, qy = nq.y;
            const double c = __dsub_rn(__dmul_rn(px, qy), __dmul_rn(qx, py));
            a2 += c;
            cx += (px + qx) * c;
            cy += (py + qy) * c;
        }
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        a2 += __shfl_xor_sync(0xffffffffu, a2, k);
        cx += __shfl_xor_sync(0xffffffffu, cx, k);
        cy += __shfl_xor_sync(0xffffffffu, cy, k);
    }
    if (lane == 0) bary[v] = make_double2(cx / (3.0 * a2), cy / (3.0 * a2));
}

// sum over unordered pairs u < v of |angle(b_c(u, v), b_m(u, v))| (the
// ordered pair (v, u) negates both vectors and has the same angle), per
// block into partial[]
__global__ void __launch_bounds__(kQThreads) k_rel_pos(const double2* __restrict__ bm, const double2* __restrict__ bc,
                                                       int R, double* __restrict__ partial) {
    __shared__ double ws[kQThreads / 32];
    double s = 0.0;
    const long long np = (long long)R * R;
    for (long long k = (long long)blockIdx.x * kQThreads + threadIdx.x; k < np; k += (long long)gridDim.x * kQThreads) {
        const int u = (int)(k / R), v = (int)(k % R);
        if (v <= u) continue;
        const double mx = bm[v].x - bm[u].x, my = bm[v].y - bm[u].y;
        const double cx = bc[v].x - bc[u].x, cy = bc[v].y - bc[u].y;
        const double cr = __dsub_rn(__dmul_rn(cx, my), __dmul_rn(cy, mx));
        const double dt = __dadd_rn(__dmul_rn(cx, mx), __dmul_rn(cy, my));
        s += fabs(atan2(cr, dt));
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kQThreads / 32; ++w) t += ws[w];
        partial[blockIdx.x] = t;
    }
}

// out = 2 sum(partial) / (pi R (R - 1)); one block of 32 threads
__global__ void k_rel_pos_final(const double* __restrict__ partial, int nb, int R, double* __restrict__ out) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += partial[b];
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if (threadIdx.x == 0) out[0] = R < 2 ? 0.0 : 2.0 * s / (3.14159265358979323846 * (double)R * (double)(R - 1));
}

unsigned pixel_blocks(int log2n) { return (unsigned)(((1ll << (2 * log2n)) + kQThreads - 1) / kQThreads); }

}  // namespace

cudaError_t launch_adjacency(const uint16_t* lab, int log2n, int R, uint32_t* bits, cudaStream_t s) {
    k_adjacency<<<pixel_blocks(log2n), kQThreads, 0, s>>>(lab, log2n, R, bits);
    return cudaGetLastError();
}

cudaError_t launch_pair_counts(const uint32_t* a, const uint32_t* b, long long nw, unsigned long long* out,
                               cudaStream_t s) {
    const long long want = (nw + kQThreads - 1) / kQThreads;
    const unsigned grid = (unsigned)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
    k_pair_counts<<<grid, kQThreads, 0, s>>>(a, b, nw, out);
    return cudaGetLastError();
}

cudaError_t launch_bbox(const uint16_t* lab, int log2n, int R, int* box, cudaStream_t s) {
    k_fill_box<<<(R + kQThreads - 1) / kQThreads, kQThreads, 0, s>>>(box, R);
    k_bbox<<<pixel_blocks(log2n), kQThreads, 0, s>>>(lab, log2n, R, box);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint16_t* lab, int log2n, int R, const QRegion* reg, int which, uint32_t* masks,
                        cudaStream_t s) {
    k_pack<<<pixel_blocks(log2n), kQThreads, 0, s>>>(lab, log2n, R, reg, which, masks);
    return cudaGetLastError();
}

cudaError_t launch_correlate(const int2* items, int n_items, const QRegion* reg, const uint32_t* mm,
                             const uint32_t* mc, int* omax, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    k_correlate<<<(unsigned)n_items, kQThreads, 0, s>>>(items, reg, mm, mc, omax);
    return cudaGetLastError();
}

cudaError_t launch_shape_final(const int* cm, const int* cc, const int* omax, int R, double* per, double* out,
                               cudaStream_t s) {
    k_shape_final<<<1, 1024, 0, s>>>(cm, cc, omax, R, per, out);
    return cudaGetLastError();
}

cudaError_t launch_barycentres(const int* reg_ring_off, const int* reg_rings, const int* ring_off,
                               const int* ring_idx, const float2* xy, int R, double2* bary, cudaStream_t s) {
    const unsigned grid = (unsigned)(((long long)R * 32 + kQThreads - 1) / kQThreads);
    k_barycentres<<<grid, kQThreads, 0, s>>>(reg_ring_off, reg_rings, ring_off, ring_idx, xy, R, bary);
    return cudaGetLastError();
}

int rel_pos_blocks() { return 152 * 4; }

cudaError_t launch_rel_pos(const double2* bm, const double2* bc, int R, double* partial, double* out,
                           cudaStream_t s) {
    const int nb = rel_pos_blocks();
    k_rel_pos<<<nb, kQThreads, 0, s>>>(bm, bc, R, partial);
    k_rel_pos_final<<<1, 32, 0, s>>>(partial, nb, R, out);
    return cudaGetLastError();
}

}  // namespace inim
