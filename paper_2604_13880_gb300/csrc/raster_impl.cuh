// Device bodies of the rasteriser (Sec. 4.1 step 2) and of the density table
// (step 3), shared by the per-step kernels (raster.cu) and the persistent
// kernel (persistent.cu).  See raster.cu for the rule.
#pragma once

#include "raster_common.cuh"
#include "table.cuh"

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
// RowShared in dynamic shared memory, padded to 16 bytes
constexpr size_t kRowSharedPadded = (sizeof(RowShared) + 15) & ~size_t(15);

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

// Shared-memory bytes one warp of the row rasteriser uses for a row of n
// pixels: a u32 difference array of n entries and a bit mask of n bits.
__host__ __device__ constexpr size_t row_warp_bytes(int n) { return (size_t)n * 4 + (size_t)n / 8; }

// Span [a, b) of region v as two events of a difference array: +w at a,
// -w at b, w = 2^17 + v - R (mod 2^32).  The prefix sum at pixel i is then
// P = sum over the spans covering i of w, and with Q = R + P:
//   no span:   Q = R                  (the background label)
//   one span:  Q = 2^17 + v           (low half v)
//   c >= 2:    P >= c (2^17 - R) >= 2^17 (R <= 65534), so Q >= 2^17 + R.
// So the label is the low half of Q, and a pixel is inside two or more spans
// exactly when P >= 2^17 (no wrap: c < 2^14).  An end at b = n lies past the
// last pixel and is dropped.
__device__ __forceinline__ void mark_span(unsigned* diff, unsigned ka, unsigned kb, unsigned n, unsigned R) {
    const unsigned a = ka & 0xffffu, b = kb & 0xffffu;
    if (a < b) {
        const unsigned w = 0x20000u + (ka >> 16) - R;
        atomicAdd(&diff[a], w);
        if (b < n) atomicAdd(&diff[b], 0u - w);
    }
}

// One round of the striped prefix over a row: pixels [256r, 256r + 256),
// lane l holding [256r + 8l, 256r + 8l + 8).  Returns the eight inclusive
// prefixes (from `carry`, the prefix before the round) and advances carry.
struct Round8 { unsigned p[8]; };

__device__ __forceinline__ Round8 prefix_round(const unsigned* diff, int r, int lane, unsigned& carry) {
    const uint4* src = reinterpret_cast<const uint4*>(diff) + 64 * r + 2 * lane;
    const uint4 a = src[0], b = src[1];
    Round8 t;
    t.p[0] = a.x;
    t.p[1] = t.p[0] + a.y;
    t.p[2] = t.p[1] + a.z;
    t.p[3] = t.p[2] + a.w;
    t.p[4] = t.p[3] + b.x;
    t.p[5] = t.p[4] + b.y;
    t.p[6] = t.p[5] + b.z;
    t.p[7] = t.p[6] + b.w;
    unsigned incl = t.p[7];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    const unsigned base = carry + incl - t.p[7];
    carry += __shfl_sync(0xffffffffu, incl, 31);
#pragma unroll
    for (int k = 0; k < 8; ++k) t.p[k] += base;
    return t;
}

// Fold-over in this row: the label pass wrote a meaningless label at each
// pixel inside c >= 2 spans, and the span lengths counted it c times.  Such a
// pixel takes the smallest covering region id.  Three steps:
//  (a) a second striped prefix pass marks those pixels in the row bit mask;
//      each pixel's word of the difference array is read by its owner lane
//      only, which resets a marked word at once to ~0: the array now holds a
//      running minimum per marked pixel;
//  (b) each lane, for each of its own spans, takes the minimum with its
//      region over the marked pixels the span covers, and gives back one
//      count per such pixel;
//  (c) lanes, one 32-pixel word of the mask each, write the resolved labels
//      and count them once.
template <int KPL>
__device__ __forceinline__ void resolve_overlaps_warp(const Job& J, int j, int cnt, const unsigned (&key)[KPL],
                                                      unsigned* diff, unsigned* bits, int lane) {
    const int n = J.n;
    unsigned carry = 0;
    for (int r = 0; r < (n >> 8); ++r) {
        const Round8 t = prefix_round(diff, r, lane, carry);
        unsigned m8 = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) m8 |= (t.p[k] >= 0x20000u ? 1u : 0u) << k;
        const int i0 = 256 * r + 8 * lane;
        for (unsigned h = m8; h; h &= h - 1u) diff[i0 + __ffs(h) - 1] = 0xffffffffu;
        // lanes 4q .. 4q+3 make up mask word 8r + q
        unsigned m = m8 << (8 * (lane & 3));
        m |= __shfl_xor_sync(0xffffffffu, m, 1);
        m |= __shfl_xor_sync(0xffffffffu, m, 2);
        if ((lane & 3) == 0) bits[8 * r + (lane >> 2)] = m;
    }
    __syncwarp();
    // (b) this lane's spans
    auto take = [&](unsigned ka, unsigned kb) {
        const int a = (int)(ka & 0xffffu), b = (int)(kb & 0xffffu);
        if (a >= b) return;
        const unsigned v = ka >> 16;
        int taken = 0;
        for (int w = a >> 5; w <= ((b - 1) >> 5); ++w) {
            const int lo = max(a - (w << 5), 0), hi = min(b - (w << 5), 32);
            const unsigned range = (hi - lo == 32) ? 0xffffffffu : (((1u << (hi - lo)) - 1u) << lo);
            const unsigned hit = bits[w] & range;
            taken += __popc(hit);
            for (unsigned h = hit; h; h &= h - 1u) atomicMin(&diff[(w << 5) + __ffs(h) - 1], v);
        }
        if (taken) atomicAdd(&J.counts[v], -taken);
    };
    if constexpr (KPL == 1) {
        const unsigned kb = __shfl_down_sync(0xffffffffu, key[0], 1);
        if ((lane & 1) == 0 && lane + 1 < cnt) take(key[0], kb);
    } else {
#pragma unroll
        for (int t = 0; t < KPL / 2; ++t)
            if (lane * KPL + 2 * t + 1 < cnt) take(key[2 * t], key[2 * t + 1]);
    }
    __syncwarp();
    // (c) the resolved labels, counted as runs of equal labels
    uint16_t* lab = J.labels + (size_t)j * n;
    unsigned cur = 0xffffffffu;
    int run = 0;
    for (int w = lane; w < (n >> 5); w += 32) {
        for (unsigned h = bits[w]; h; h &= h - 1u) {
            const int i = (w << 5) + __ffs(h) - 1;
            const unsigned v = diff[i];
            lab[i] = (uint16_t)v;
            if (v != cur) {
                if (run) atomicAdd(&J.counts[cur], run);
                cur = v;
                run = 0;
            }
            ++run;
        }
    }
    if (run) atomicAdd(&J.counts[cur], run);
    if (lane == 0) atomicExch(&J.st->overlap, 1);
}

// One row: keys sorted by (region, column) give each region's spans as
// consecutive pairs.  Each lane enters its own spans into the warp's
// difference array; a striped prefix pass (rounds of 256 pixels, 8 per lane,
// a warp scan per round) then yields every label, stored as one contiguous
// 512-byte write per round, and, from the largest prefix, whether any pixel
// lies in two spans.  The cost does not grow with the number of spans.  Such
// pixels are then resolved by resolve_overlaps_warp.  Keys are taken striped
// (lane l holds bucket slots l, l + 32, ...): the sort's input order is free,
// and s0, s1 are slots lane and 32 + lane, read with the row's count.
template <int KPL>
__device__ __forceinline__ void raster_row_warp(const Job& J, int j, int cnt, unsigned s0, unsigned s1,
                                                unsigned* diff, int lane) {
    const int n = J.n;
    const unsigned R = (unsigned)J.n_regions;
    const uint32_t* bucket = J.keys + (size_t)j * kKeyStride;
    unsigned key[KPL];
#pragma unroll
    for (int e = 0; e < KPL; ++e) {
        const int idx = e * 32 + lane;
        const unsigned raw = e == 0 ? s0 : (e == 1 ? s1 : (idx < cnt ? bucket[idx] : 0u));
        key[e] = idx < cnt ? raw : 0xffffffffu;
    }
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int i = lane; i < (n >> 2); i += 32) reinterpret_cast<uint4*>(diff)[i] = z;
    warp_bitonic<KPL>(key, lane);
    __syncwarp();
    if constexpr (KPL == 1) {
        const unsigned kb = __shfl_down_sync(0xffffffffu, key[0], 1);
        if ((lane & 1) == 0 && lane + 1 < cnt) mark_span(diff, key[0], kb, (unsigned)n, R);
    } else {
#pragma unroll
        for (int t = 0; t < KPL / 2; ++t)
            if (lane * KPL + 2 * t + 1 < cnt) mark_span(diff, key[2 * t], key[2 * t + 1], (unsigned)n, R);
    }
    __syncwarp();
    // Q = R + P: labels are its low halves (byte-permute packs two), and the
    // largest Q tells whether a pixel lies in two or more spans
    unsigned carry = R, qmax = 0;
    uint4* dst = reinterpret_cast<uint4*>(J.labels + (size_t)j * n) + lane;
#pragma unroll 2
    for (int r = 0; r < (n >> 8); ++r) {
        const Round8 q = prefix_round(diff, r, lane, carry);
        qmax = max(qmax, max(max(max(q.p[0], q.p[1]), max(q.p[2], q.p[3])),
                             max(max(q.p[4], q.p[5]), max(q.p[6], q.p[7]))));
        dst[32 * r] = make_uint4(__byte_perm(q.p[0], q.p[1], 0x5410), __byte_perm(q.p[2], q.p[3], 0x5410),
                                 __byte_perm(q.p[4], q.p[5], 0x5410), __byte_perm(q.p[6], q.p[7], 0x5410));
    }
    const bool over = qmax >= 0x20000u + R;
    // counts from the spans held by this lane
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
    if (__any_sync(0xffffffffu, over)) {
        __syncwarp();
        resolve_overlaps_warp<KPL>(J, j, cnt, key, diff, diff + n, lane);
    }
    if (lane == 0) J.row_cnt[j] = 0;     // ready for the next iteration
}

// Item first_row / 8 = q of one job's n / 8 row items: rows q + w n / 8,
// w = 0 .. 7, one warp each (rows spread over the texture, so that the rows
// a stretched region makes long are shared out over the items instead of
// filling a few); rows_smem holds 8 * row_warp_bytes(N) bytes.  With
// check_active the job's active flag is read together with the row's count
// and first key slots (one round trip).  A row with more crossings than a
// warp holds is returned (local_big: the caller's block rasterises it) or
// appended to the job's big-row list.  Returns that row or -1, the same on
// every lane.
__device__ __forceinline__ int raster_rows_item(const Job& J, int first_row, unsigned* rows_smem,
                                                bool check_active = false, bool local_big = false) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = first_row / kWarpsPerBlock + warp * (J.n / kWarpsPerBlock);
    if (warp >= kWarpsPerBlock || j >= J.n) return -1;
    unsigned* diff = rows_smem + (size_t)warp * (row_warp_bytes(J.n) / 4);
    const uint32_t* bucket = J.keys + (size_t)j * kKeyStride;
    const int act = check_active ? J.st->active : 1;
    const int cnt = J.row_cnt[j];
    const unsigned s0 = bucket[lane], s1 = bucket[32 + lane];     // slots past cnt are ignored
    __syncwarp();                                    // every lane has the count before lane 0 resets it
    if (!act) return -1;
    if (cnt <= 32) raster_row_warp<1>(J, j, cnt, s0, s1, diff, lane);
    else if (cnt <= 2 * 32) raster_row_warp<2>(J, j, cnt, s0, s1, diff, lane);
    else if (cnt <= 4 * 32) raster_row_warp<4>(J, j, cnt, s0, s1, diff, lane);
    else if (cnt <= 8 * 32) raster_row_warp<8>(J, j, cnt, s0, s1, diff, lane);
    else if (local_big) return j;                    // the block path (raster_row), by the caller
    else if (lane == 0) {                            // big row: left to density_table_body (persistent form)
        const int q = atomicAdd(&J.st->n_big, 1);
        J.big_rows[q] = j;
    }
    return -1;
}

// dynamic shared memory of the row kernel: the warps' row scratch, reused by
// the block path
__host__ __device__ constexpr size_t rows_smem_bytes(int max_n) {
    return kWarpsPerBlock * row_warp_bytes(max_n) > kRowSharedPadded ? kWarpsPerBlock * row_warp_bytes(max_n)
                                                                     : kRowSharedPadded;
}

// One row by the whole block (256 threads): the block path for rows with
// more crossings than a warp holds (up to kRowKeyCap; more raise the
// capacity error in raster_row).
__device__ __forceinline__ void raster_row_block(const Job& J, int j, RowShared& sh) {
    switch (J.n / kRowThreads) {
        case 1: raster_row<1>(J, j, sh); break;
        case 2: raster_row<2>(J, j, sh); break;
        case 4: raster_row<4>(J, j, sh); break;
        case 8: raster_row<8>(J, j, sh); break;
        default: raster_row<16>(J, j, sh); break;
    }
}

// The rows of the job's big-row list (rows with more crossings than a warp
// holds, left by the persistent kernel's row phase), one block per job.
__device__ inline void raster_big_rows(const Job& J, RowShared& sh) {
    const int nbig = __ldcg(&J.st->n_big);
    for (int q = 0; q < nbig; ++q) {
        raster_row_block(J, J.big_rows[q], sh);
        __syncthreads();
    }
}

// per job (a block of 256 threads): the big rows left by the row kernel,
// then the density table and the job's per-iteration state (table.cuh)
__device__ inline void density_table_body(const Job& J, RowShared& rsh) {
    raster_big_rows(J, rsh);
    region_table(J, J.dens, true);
}


}  // namespace inim
