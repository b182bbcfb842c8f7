// Device bodies of the rasteriser (Sec. 4.1 step 2) and of the density table
// (step 3), shared by the per-step kernels (raster.cu) and the persistent
// kernel (persistent.cu).  See raster.cu for the rule.
#pragma once

#include "raster_common.cuh"

namespace inim {


constexpr int kRowThreads = 256;
constexpr int kRowKeyCap = kKeyStride;   // crossings one row can hold in shared memory

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
// RowShared plus the density table's reduction arrays in one block of shared
// memory: [RowShared, padded to 16][32 doubles][32 long longs]
constexpr size_t kRowSharedPadded = (sizeof(RowShared) + 15) & ~size_t(15);
constexpr size_t kTableSmem = kRowSharedPadded + 32 * sizeof(double) + 32 * sizeof(long long);

template <int CPT>
__device__ inline void raster_row(const Job& J, int j, RowShared& sh) {
    const int n = J.n;
    const int R = J.n_regions;
    const int tid = threadIdx.x;
    const uint32_t* bucket = J.keys + (size_t)j * kKeyStride;
    const int cnt = __ldcg(J.row_cnt + j);
    __syncthreads();                      // every thread has read the count before it is reset
    const bool bad = cnt > kRowKeyCap;
    if (bad) {   // bucket overflow: flag the capacity error, write background
        if (tid == 0) { atomicExch(&J.st->error, INIM_E_CAPACITY); J.row_cnt[j] = 0; }
        uint16_t lab[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) lab[k] = (uint16_t)R;
        store_labels<CPT>(J.labels + (size_t)j * n + tid * CPT, lab);
        return;
    }
    for (int k = tid; k < cnt; k += blockDim.x) sh.keys[k] = bucket[k];
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
        }
        // counts as run lengths over this thread's CPT pixels
        unsigned cur = lab[0];
        int run = 0;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            if (lab[k] != cur) {
                if (cur != (unsigned)R) atomicAdd(&J.counts[cur], run);
                cur = lab[k];
                run = 0;
            }
            ++run;
        }
        if (cur != (unsigned)R) atomicAdd(&J.counts[cur], run);
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

// Rows with more crossings than a warp holds in registers, one block per job
// (usually none): the block-per-row path.
__device__ inline void raster_big_rows(const Job& J, RowShared& sh) {
    const int nbig = __ldcg(&J.st->n_big);
    for (int q = 0; q < nbig; ++q) {
        const int j = J.big_rows[q];
        switch (J.n / kRowThreads) {
            case 1: raster_row<1>(J, j, sh); break;
            case 2: raster_row<2>(J, j, sh); break;
            case 4: raster_row<4>(J, j, sh); break;
            case 8: raster_row<8>(J, j, sh); break;
            default: raster_row<16>(J, j, sh); break;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// warp-per-row rasteriser (the common case: <= 256 crossings in a row)
// ---------------------------------------------------------------------------
constexpr int kWarpsPerBlock = 8;

// ascending bitonic sort of KPL*32 keys, lane l holding elements [l*KPL, l*KPL+KPL)
template <int KPL>
__device__ __forceinline__ void warp_bitonic(unsigned (&k)[KPL], int lane) {
    constexpr int NT = KPL * 32;
#pragma unroll
    for (int size = 2; size <= NT; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= KPL) {
                const int lmask = stride / KPL;
#pragma unroll
                for (int e = 0; e < KPL; ++e) {
                    const int idx = lane * KPL + e;
                    const unsigned other = __shfl_xor_sync(0xffffffffu, k[e], lmask);
                    const bool up = (idx & size) == 0;
                    const bool lower = (idx & stride) == 0;
                    const unsigned mn = min(k[e], other), mx = max(k[e], other);
                    k[e] = (lower == up) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int e = 0; e < KPL; ++e) {
                    const int p = e ^ stride;
                    if (p > e) {
                        const int idx = lane * KPL + e;
                        const bool up = (idx & size) == 0;
                        const unsigned a = k[e], b = k[p];
                        if (up ? (a > b) : (a < b)) { k[e] = b; k[p] = a; }
                    }
                }
            }
        }
    }
}

// Paint the span [a, b) of one region into the row copy, only over pixels that
// are still background; returns how many of this lane's pixels of the span
// were painted already (a pixel inside two regions).
__device__ __forceinline__ int paint_span(uint16_t* row, unsigned R, unsigned ka, unsigned kb, int lane) {
    const int a = (int)(ka & 0xffffu), b = (int)(kb & 0xffffu);
    const uint16_t v = (uint16_t)(ka >> 16);
    int over = 0;
    for (int i = a + lane; i < b; i += 32) {
        if (row[i] == (uint16_t)R) row[i] = v;
        else ++over;
    }
    __syncwarp();
    return over;
}

// One row: keys sorted by (region, column) give each region's spans as
// consecutive pairs.  The spans are painted into a shared-memory copy of the
// row in sorted order, writing only still-background pixels, so a pixel in
// several regions keeps the smallest id.  Overlap <=> the summed span lengths
// exceed the painted pixel count.
template <int KPL>
__device__ inline void raster_row_warp(const Job& J, int j, int cnt, uint16_t* row, int lane) {
    const int n = J.n;
    const unsigned R = (unsigned)J.n_regions;
    const uint32_t* bucket = J.keys + (size_t)j * kKeyStride;
    unsigned key[KPL];
#pragma unroll
    for (int e = 0; e < KPL; ++e) {
        const int idx = lane * KPL + e;
        key[e] = idx < cnt ? bucket[idx] : 0xffffffffu;
    }
    // background fill of the row copy
    const unsigned bg2 = R | (R << 16);
    const uint4 bg8 = make_uint4(bg2, bg2, bg2, bg2);
    for (int i = lane; i < (n >> 3); i += 32) reinterpret_cast<uint4*>(row)[i] = bg8;
    warp_bitonic<KPL>(key, lane);
    __syncwarp();
    // paint spans in sorted order, noting pixels that were painted already
    int my_over = 0;
    if constexpr (KPL == 1) {
        // pair p is (lane 2p, lane 2p + 1)
        for (int p = 0; 2 * p + 1 < cnt; ++p)
            my_over += paint_span(row, R, __shfl_sync(0xffffffffu, key[0], 2 * p),
                                  __shfl_sync(0xffffffffu, key[0], 2 * p + 1), lane);
    } else {
        const int src_lanes = (cnt + KPL - 1) / KPL;
        for (int src = 0; src < src_lanes; ++src) {
#pragma unroll
            for (int t = 0; t < KPL / 2; ++t) {
                const unsigned ka = __shfl_sync(0xffffffffu, key[2 * t], src);
                const unsigned kb = __shfl_sync(0xffffffffu, key[2 * t + 1], src);
                if (src * KPL + 2 * t + 1 >= cnt) continue;          // padding (warp-uniform)
                my_over += paint_span(row, R, ka, kb, lane);
            }
        }
    }
    if (!__any_sync(0xffffffffu, my_over != 0)) {
        // no overlap: counts from the spans held by this lane
        if constexpr (KPL == 1) {
            const unsigned kb = __shfl_down_sync(0xffffffffu, key[0], 1);
            if ((lane & 1) == 0 && lane + 1 < cnt) {
                const int a = (int)(key[0] & 0xffffu), b = (int)(kb & 0xffffu);
                if (a < b) atomicAdd(&J.counts[key[0] >> 16], b - a);
            }
        } else {
#pragma unroll
            for (int t = 0; t < KPL / 2; ++t) {
                const int idx = lane * KPL + 2 * t;
                if (idx + 1 < cnt) {
                    const int a = (int)(key[2 * t] & 0xffffu), b = (int)(key[2 * t + 1] & 0xffffu);
                    if (a < b) atomicAdd(&J.counts[key[2 * t] >> 16], b - a);
                }
            }
        }
    } else {
        // fold-over in this row: counts from the resolved labels, as run
        // lengths over each lane's n/32 contiguous pixels (one atomic per run
        // instead of one per pixel on a few hot counters)
        const int per = n >> 5;
        const int p0 = lane * per;
        unsigned cur = row[p0];
        int run = 0;
        for (int i = p0; i < p0 + per; ++i) {
            const unsigned l = row[i];
            if (l != cur) {
                if (cur != R) atomicAdd(&J.counts[cur], run);
                cur = l;
                run = 0;
            }
            ++run;
        }
        if (cur != R) atomicAdd(&J.counts[cur], run);
        if (lane == 0) atomicExch(&J.st->overlap, 1);
    }
    // write the row
    uint4* dst = reinterpret_cast<uint4*>(J.labels + (size_t)j * n);
    const uint4* srcv = reinterpret_cast<const uint4*>(row);
    for (int i = lane; i < (n >> 3); i += 32) dst[i] = srcv[i];
    if (lane == 0) J.row_cnt[j] = 0;     // ready for the next iteration
}

// rows [first_row, first_row + 8) of one job, one warp each; rows_smem holds
// 8 * N u16 (the row copies)
__device__ __forceinline__ void raster_rows_item(const Job& J, int first_row, uint16_t* rows_smem) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = first_row + warp;
    if (warp >= kWarpsPerBlock || j >= J.n) return;
    uint16_t* row = rows_smem + (size_t)warp * J.n;
    const int cnt = J.row_cnt[j];
    __syncwarp();                                    // every lane has the count before lane 0 resets it
    if (cnt > kKeyStride) {                          // bucket overflow
        if (lane == 0) { atomicExch(&J.st->error, INIM_E_CAPACITY); J.row_cnt[j] = 0; }
        return;
    }
    if (cnt <= 32) raster_row_warp<1>(J, j, cnt, row, lane);
    else if (cnt <= 2 * 32) raster_row_warp<2>(J, j, cnt, row, lane);
    else if (cnt <= 4 * 32) raster_row_warp<4>(J, j, cnt, row, lane);
    else if (cnt <= 8 * 32) raster_row_warp<8>(J, j, cnt, row, lane);
    else if (lane == 0) {                            // big row: handled by k_raster_big
        const int q = atomicAdd(&J.st->n_big, 1);
        J.big_rows[q] = j;
    }
}

// per job (a block of 256 threads): the big rows, then d0, density table,
// background count, total mass, fixed-point scale
__device__ inline void density_table_body(const Job& J, RowShared& rsh, double* ss, long long* so) {
    raster_big_rows(J, rsh);
    const int R = J.n_regions;
    double s = 0.0;
    long long o = 0;
    int bad = 0;
    for (int v = threadIdx.x; v < R; v += blockDim.x) {
        const float sv = J.values[v];
        if (!(sv >= 0.0f) || isinf(sv)) bad = 1;           // values must be finite, >= 0
        const int c = __ldcg(J.counts + v);
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
        const int c = __ldcg(J.counts + v);
        J.dens[v] = (c > 0 && !empty) ? (float)((double)J.values[v] / ((double)c * d0)) : 0.0f;
    }
    if (threadIdx.x == 0) {
        J.dens[R] = empty ? 1.0f : J.bdv_scale;
        J.counts[R] = (int)o_bg;
        JobState* st = J.st;
        st->d0 = d0;
        st->bdv_abs = (double)J.bdv_scale * d0;
        st->mass = empty ? 1.0 : sum_s + st->bdv_abs * (double)o_bg;
        st->mass_it[st->raster_it & 1] = st->mass;
        st->raster_it += 1;
        // all InIm magnitudes are <= C' = sum_o + bdv * o_bg (relative units)
        const double cbound = empty ? (double)npx : ((double)sum_o + (double)J.bdv_scale * (double)o_bg);
        int e = 0;
        frexp(cbound * 1.0001 + 1.0, &e);   // cbound < 2^e
        int fb = 61 - e;
        st->fix_bits = fb < 0 ? 0 : fb;
    }
}


}  // namespace inim
