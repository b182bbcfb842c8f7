// Step 2 of the static algorithm (Sec. 4.1): rasterise the current region
// polygons into a label texture and count the pixel area o(v) of every region.
//
// Exact integer rule (shared reading with the oracle): vertices snap to
// X = rint(x 2^(k+8)); pixel (i, j) has its centre at (256 i + 128, 256 j + 128);
// an edge ordered so that Y0 < Y1 counts for a centre iff Y0 <= Yc < Y1 and
// (Xc - X0)(Y1 - Y0) >= (X1 - X0)(Yc - Y0).  For the centres of row j that is
// exactly the columns i >= c with
//   c = ceil(((X1 - X0)(Yc - Y0) + (X0 - 128)(Y1 - Y0)) / (256 (Y1 - Y0))).
// A pixel is inside region v iff v's crossing count is odd; inside several
// regions it takes the smallest id and the overlap flag is raised.
//
// Kernels (edge-parallel, then row-parallel; no per-pixel atomics):
//   k_row_hist     per edge: crossings per row
//   k_row_offsets  per job: exclusive prefix over rows, clears counters
//   k_crossings    per edge: scatter (region << 16 | c) keys into row buckets
//   k_raster_rows  per row: sort keys, pair them into spans, turn the spans
//                  into an XOR/coverage difference array, prefix it, write
//                  the labels of the whole row once with vector stores, and
//                  add span lengths to the pixel counts.
#include "inim_internal.cuh"

namespace inim {

namespace {

constexpr int kRowThreads = 256;
constexpr int kRowKeyCap = 2048;   // crossings one row can hold in shared memory

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

__global__ void k_row_hist(const Job* __restrict__ jobs, const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const Job& J = jobs[m.x];
    if (!J.st->active) return;
    const int e = m.y * blockDim.x + threadIdx.x;
    if (e >= J.n_edges) return;
    EdgeFix f;
    if (!edge_rows(J, e, f)) return;
    for (int j = f.jlo; j <= f.jhi; ++j) atomicAdd(&J.row_cnt[j], 1);
}

// one block of 1024 threads per job
__global__ void k_row_offsets(const Job* __restrict__ jobs) {
    const Job& J = jobs[blockIdx.x];
    if (!J.st->active) return;
    __shared__ int wsum[32];
    const int n = J.n;
    const int per = (n + blockDim.x - 1) / blockDim.x;   // <= 4
    const int base = threadIdx.x * per;
    int loc[4];
    int s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int v = (k < per && base + k < n) ? J.row_cnt[base + k] : 0;
        loc[k] = s;
        s += v;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int woff = 0, tot = 0;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) {
        if (k < w) woff += wsum[k];
        tot += wsum[k];
    }
    const int excl = woff + incl - s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k < per && base + k < n) {
            J.row_off[base + k] = excl + loc[k];
            J.row_cnt[base + k] = 0;            // reused as the fill cursor
        }
    }
    if (threadIdx.x == 0) {
        J.row_off[n] = tot;
        if (tot > J.key_cap) atomicExch(&J.st->error, INIM_E_CAPACITY);
    }
    for (int v = threadIdx.x; v <= J.n_regions; v += blockDim.x) J.counts[v] = 0;
}

__global__ void k_crossings(const Job* __restrict__ jobs, const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const Job& J = jobs[m.x];
    if (!J.st->active) return;
    const int e = m.y * blockDim.x + threadIdx.x;
    if (e >= J.n_edges) return;
    EdgeFix f;
    if (!edge_rows(J, e, f)) return;
    const unsigned reg = (unsigned)J.edge_region[e] << 16;
    const long long dY = f.Y1 - f.Y0;
    const long long dX = f.X1 - f.X0;
    const long long den = 256 * dY;
    for (int j = f.jlo; j <= f.jhi; ++j) {
        const long long Yc = 256LL * j + 128;
        long long c = ceil_div(dX * (Yc - f.Y0) + (f.X0 - 128) * dY, den);
        if (c < 0) c = 0;
        if (c > J.n) c = J.n;
        const int slot = atomicAdd(&J.row_cnt[j], 1);
        const int idx = J.row_off[j] + slot;
        if (idx < J.key_cap) J.keys[idx] = reg | (unsigned)c;
    }
}

template <int CPT>
__device__ __forceinline__ void store_labels(uint16_t* dst, const uint16_t (&lab)[CPT]) {
    if constexpr (CPT == 16) {
        uint4 a, b;
        a.x = lab[0] | (lab[1] << 16); a.y = lab[2] | (lab[3] << 16);
        a.z = lab[4] | (lab[5] << 16); a.w = lab[6] | (lab[7] << 16);
        b.x = lab[8] | (lab[9] << 16); b.y = lab[10] | (lab[11] << 16);
        b.z = lab[12] | (lab[13] << 16); b.w = lab[14] | (lab[15] << 16);
        reinterpret_cast<uint4*>(dst)[0] = a;
        reinterpret_cast<uint4*>(dst)[1] = b;
    } else if constexpr (CPT == 8) {
        uint4 a;
        a.x = lab[0] | (lab[1] << 16); a.y = lab[2] | (lab[3] << 16);
        a.z = lab[4] | (lab[5] << 16); a.w = lab[6] | (lab[7] << 16);
        reinterpret_cast<uint4*>(dst)[0] = a;
    } else if constexpr (CPT == 4) {
        uint2 a;
        a.x = lab[0] | (lab[1] << 16); a.y = lab[2] | (lab[3] << 16);
        reinterpret_cast<uint2*>(dst)[0] = a;
    } else if constexpr (CPT == 2) {
        reinterpret_cast<unsigned*>(dst)[0] = lab[0] | (lab[1] << 16);
    } else {
        dst[0] = lab[0];
    }
}

struct RowShared {
    unsigned keys[kRowKeyCap];
    unsigned sorted[kRowKeyCap];
    unsigned diff[4097];          // low 16 bits: XOR of (v+1); high 16 bits: coverage delta
    unsigned wx[kRowThreads / 32];
    unsigned wc[kRowThreads / 32];
};

template <int CPT>
__device__ void raster_row(const Job& J, int j, RowShared& sh) {
    const int n = J.n;
    const int R = J.n_regions;
    const int tid = threadIdx.x;
    const int k0 = J.row_off[j];
    const int k1 = J.row_off[j + 1];
    const int cnt = k1 - k0;
    const bool bad = (k1 > J.key_cap) || (cnt > kRowKeyCap);
    if (bad) {   // capacity error already (or now) flagged; write background
        if (tid == 0) { atomicExch(&J.st->error, INIM_E_CAPACITY); J.row_cnt[j] = 0; }
        uint16_t lab[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) lab[k] = (uint16_t)R;
        store_labels<CPT>(J.labels + (size_t)j * n + tid * CPT, lab);
        return;
    }
    for (int k = tid; k < cnt; k += blockDim.x) sh.keys[k] = J.keys[k0 + k];
    for (int k = tid; k <= n; k += blockDim.x) sh.diff[k] = 0u;
    __syncthreads();
    // rank sort (ties broken by position): sorted by (region, column)
    for (int e = tid; e < cnt; e += blockDim.x) {
        const unsigned key = sh.keys[e];
        int rank = 0;
        for (int k = 0; k < cnt; ++k) {
            const unsigned o = sh.keys[k];
            rank += (o < key) || (o == key && k < e);
        }
        sh.sorted[rank] = key;
    }
    __syncthreads();
    // consecutive pairs of one region are its spans [a, b)
    const int nspan = cnt >> 1;
    for (int p = tid; p < nspan; p += blockDim.x) {
        const unsigned ka = sh.sorted[2 * p], kb = sh.sorted[2 * p + 1];
        const unsigned a = ka & 0xffffu, b = kb & 0xffffu, v = ka >> 16;
        if (a < b) {
            atomicXor(&sh.diff[a], v + 1u);
            atomicXor(&sh.diff[b], v + 1u);
            atomicAdd(&sh.diff[a], 1u << 16);
            atomicAdd(&sh.diff[b], 0xffff0000u);
        }
    }
    __syncthreads();
    // prefix (XOR on the low half, sum on the high half) over the row
    const int i0 = tid * CPT;
    unsigned px[CPT], pc[CPT];
    unsigned ax = 0, ac = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const unsigned w = sh.diff[i0 + k];
        ax ^= (w & 0xffffu);
        ac += (w >> 16);
        px[k] = ax;
        pc[k] = ac;
    }
    const int lane = tid & 31, wid = tid >> 5;
    unsigned ix = ax, ic = ac;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned tx = __shfl_up_sync(0xffffffffu, ix, o);
        const unsigned tc = __shfl_up_sync(0xffffffffu, ic, o);
        if (lane >= o) { ix ^= tx; ic += tc; }
    }
    if (lane == 31) { sh.wx[wid] = ix; sh.wc[wid] = ic; }
    __syncthreads();
    unsigned ox = ix ^ ax, oc = ic - ac;          // exclusive within the warp
    for (int w = 0; w < wid; ++w) { ox ^= sh.wx[w]; oc += sh.wc[w]; }
    uint16_t lab[CPT];
    int over = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const unsigned c = (oc + pc[k]) & 0xffffu;
        const unsigned x = (ox ^ px[k]) & 0xffffu;
        if (c == 0) lab[k] = (uint16_t)R;
        else if (c == 1) lab[k] = (uint16_t)(x - 1);
        else { over = 1; lab[k] = 0xffffu; }
    }
    const int any_over = __syncthreads_or(over);
    if (any_over) {
        // slow path (fold-over): smallest region id among the covering spans,
        // counts from the resolved labels
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            if (lab[k] == 0xffffu) {
                const unsigned i = (unsigned)(i0 + k);
                unsigned best = 0xffffu;
                for (int p = 0; p < nspan; ++p) {
                    const unsigned ka = sh.sorted[2 * p], kb = sh.sorted[2 * p + 1];
                    if ((ka & 0xffffu) <= i && i < (kb & 0xffffu) && (ka >> 16) < best) best = ka >> 16;
                }
                lab[k] = (uint16_t)best;
            }
            if (lab[k] != (uint16_t)R) atomicAdd(&J.counts[lab[k]], 1);
        }
        if (tid == 0) atomicExch(&J.st->overlap, 1);
    } else {
        for (int p = tid; p < nspan; p += blockDim.x) {
            const unsigned ka = sh.sorted[2 * p], kb = sh.sorted[2 * p + 1];
            const int a = (int)(ka & 0xffffu), b = (int)(kb & 0xffffu);
            if (a < b) atomicAdd(&J.counts[ka >> 16], b - a);
        }
    }
    store_labels<CPT>(J.labels + (size_t)j * n + i0, lab);
    if (tid == 0) J.row_cnt[j] = 0;     // ready for the next iteration
}

__global__ void __launch_bounds__(kRowThreads) k_raster_rows(const Job* __restrict__ jobs,
                                                            const int2* __restrict__ bmap) {
    __shared__ RowShared sh;
    const int2 m = bmap[blockIdx.x];
    const Job& J = jobs[m.x];
    if (!J.st->active) return;
    const int j = m.y;
    switch (J.n / kRowThreads) {
        case 1: raster_row<1>(J, j, sh); break;
        case 2: raster_row<2>(J, j, sh); break;
        case 4: raster_row<4>(J, j, sh); break;
        case 8: raster_row<8>(J, j, sh); break;
        default: raster_row<16>(J, j, sh); break;
    }
}

// per job: d0, density table, background count, total mass, fixed-point scale
__global__ void k_density_table(const Job* __restrict__ jobs) {
    const Job& J = jobs[blockIdx.x];
    if (!J.st->active) return;
    __shared__ double ss[32];
    __shared__ long long so[32];
    const int R = J.n_regions;
    double s = 0.0;
    long long o = 0;
    int bad = 0;
    for (int v = threadIdx.x; v < R; v += blockDim.x) {
        const float sv = J.values[v];
        if (!(sv >= 0.0f) || isinf(sv)) bad = 1;           // values must be finite, >= 0
        const int c = J.counts[v];
        if (c > 0) { s += (double)sv; o += c; }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&J.st->error, INIM_E_VALUE);
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, k);
        o += __shfl_xor_sync(0xffffffffu, o, k);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { ss[w] = s; so[w] = o; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0;
        long long O = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { S += ss[k]; O += so[k]; }
        ss[0] = S;
        so[0] = O;
    }
    __syncthreads();
    const double sum_s = ss[0];
    const long long sum_o = so[0];
    const long long npx = (long long)J.n * J.n;
    const long long o_bg = npx - sum_o;
    const bool empty = (sum_o == 0);
    const double d0 = empty ? 1.0 : sum_s / (double)sum_o;
    for (int v = threadIdx.x; v < R; v += blockDim.x) {
        const int c = J.counts[v];
        J.dens[v] = (c > 0 && !empty) ? (float)((double)J.values[v] / ((double)c * d0)) : 0.0f;
    }
    if (threadIdx.x == 0) {
        J.dens[R] = empty ? 1.0f : J.bdv_scale;
        J.counts[R] = (int)o_bg;
        JobState* st = J.st;
        st->d0 = d0;
        st->bdv_abs = (double)J.bdv_scale * d0;
        st->mass = empty ? 1.0 : sum_s + st->bdv_abs * (double)o_bg;
        // all InIm magnitudes are <= C' = sum_o + bdv * o_bg (relative units)
        const double cbound = empty ? (double)npx : ((double)sum_o + (double)J.bdv_scale * (double)o_bg);
        int e = 0;
        frexp(cbound * 1.0001 + 1.0, &e);   // cbound < 2^e
        int fb = 61 - e;
        st->fix_bits = fb < 0 ? 0 : fb;
    }
}

}  // namespace

cudaError_t launch_raster(const Job* d_jobs, const BlockMap& edge_blocks, const BlockMap& job_blocks,
                          const BlockMap& row_blocks, cudaStream_t s) {
    if (edge_blocks.n_blocks) k_row_hist<<<edge_blocks.n_blocks, 256, 0, s>>>(d_jobs, edge_blocks.d_map);
    k_row_offsets<<<job_blocks.n_blocks, 1024, 0, s>>>(d_jobs);
    if (edge_blocks.n_blocks) k_crossings<<<edge_blocks.n_blocks, 256, 0, s>>>(d_jobs, edge_blocks.d_map);
    k_raster_rows<<<row_blocks.n_blocks, kRowThreads, 0, s>>>(d_jobs, row_blocks.d_map);
    return cudaGetLastError();
}

cudaError_t launch_density_table(const Job* d_jobs, int n_jobs, cudaStream_t s) {
    k_density_table<<<n_jobs, 256, 0, s>>>(d_jobs);
    return cudaGetLastError();
}

}  // namespace inim
