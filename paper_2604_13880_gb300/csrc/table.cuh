// The region density table of Sec. 4.1 step 3, built by one block from the
// pixel counts o(v) of the raster and the values s(v):
//   d0 = sum_{o(v) > 0} s(v) / sum_v o(v)          (area-weighted mean density)
//   dens(v) = s(v) / (o(v) d0) for o(v) > 0, else 0;
//   dens(R) = bdv_scale, or bdv_value / d0 for a given background value
//   (value units per pixel: the dynamic-area background of Eq. (Mb))
// (an empty map, sum o = 0: d0 = 1 and dens(R) = 1).  Used by the density
// kernel and, fused, by every band block of the scan's first phase, so it
// keeps its dependent chain short: every region's value and count are loaded
// once (and kept in registers), sum s is a compensated FP32 pair (hi, lo)
// (two-sum; relative error ~R 2^-48), sum o an integer (<= N^2 <= 2^24), d0 a
// compensated FP32 quotient and the entries s(v) / (o(v) d0) in FP32.  The
// job state in double (d0, total mass M = sum s + bdv d0 o_bg) is written
// afterwards by table_state, off the table's path.
//
// Any block size gives bit-identical results, so that every block (and every
// scan tile) holds the same table: the regions are dealt to 256 virtual
// threads (region v to v mod 256), each summing its regions in order; a
// shuffle tree reduces each virtual warp of 32, and the 8 warp sums are added
// in order.  Block sizes: multiples of 32 that divide 256, or >= 256.
#pragma once

#include "inim_internal.cuh"

namespace inim {

// regions of a virtual thread kept in registers between the sums and the
// table (a map with more regions loads the rest again)
constexpr int kTableSlots = kFusedTableMax / 256;

struct TableSums {
    float hi, lo;    // sum of s(v) over regions with pixels, hi + lo
    int o;           // pixels inside regions
    float d0;        // (hi + lo) / o, 1 for an empty map
    float dbg;       // background entry dens(R)
    int fix_bits;
    int bad;         // a value is negative, NaN or infinite
};

// (hi, lo) += x exactly in hi + err, err accumulated into lo (two-sum)
__device__ __forceinline__ void pair_add(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// Fraction bits of the fixed-point InIms: every InIm magnitude is at most
// C' = sum o + dens(R) o_bg (in units of d0), and C' < 2^e leaves 61 - e
// (the factor 1.0001 covers the FP32 rounding of C').
__device__ __forceinline__ int table_fix_bits(const Job& J, int o, float dbg) {
    const int npx = J.n * J.n;
    const float cbound = o == 0 ? (float)npx : __fadd_rn((float)o, __fmul_rn(dbg, (float)(npx - o)));
    int e = 0;
    frexpf(__fadd_rn(__fmul_rn(cbound, 1.0001f), 1.0f), &e);
    const int fb = 61 - e;
    return fb < 0 ? 0 : fb;
}

__device__ inline void table_state(const Job& J, const TableSums& t, int raster_it);

// The table into `table` (R + 1 entries, shared or global memory; the caller
// synchronises before reading it).  lead: also publish it to J.dens (unless
// `table` is J.dens) and write the job state (table_state, thread 0, after
// the table).  Returns the sums (the same in every thread).
__device__ inline TableSums region_table(const Job& J, float* table, bool lead) {
    __shared__ float wh[8], wl[8];
    __shared__ int wo[8];
    __shared__ TableSums tot;
    const int R = J.n_regions;
    const int nt = (int)blockDim.x, tid = (int)threadIdx.x, lane = tid & 31;
    int bad = 0;
    // the lead's iteration counter, loaded with the regions' data (not after
    // the table, where a dependent round trip would delay the lead block)
    const int raster_it = (lead && tid == 0) ? __ldcg(&J.st->raster_it) : 0;
    // with >= 256 threads, thread t holds the first kTableSlots regions of
    // virtual thread t (v = t + 256 q) for the table below
    const bool cache = nt >= 256;
    float s_c[kTableSlots];
    int c_c[kTableSlots];
    for (int vt0 = 0; vt0 < 256; vt0 += nt) {
        const int vt = vt0 + tid;                         // virtual thread
        float hi = 0.0f, lo = 0.0f;
        int o = 0;
        if (vt < 256) {
#pragma unroll
            for (int q = 0; q < kTableSlots; ++q) {
                const int v = vt + 256 * q;
                float sv = 0.0f;
                int c = 0;
                if (v < R) {
                    sv = J.values[v];
                    c = __ldcg(J.counts + v);
                    if (!(sv >= 0.0f) || isinf(sv)) bad = 1;
                    if (c > 0) { pair_add(hi, lo, sv); o += c; }
                }
                s_c[q] = sv;
                c_c[q] = c;
            }
            for (int v = vt + 256 * kTableSlots; v < R; v += 256) {
                const float sv = J.values[v];
                if (!(sv >= 0.0f) || isinf(sv)) bad = 1;
                const int c = __ldcg(J.counts + v);
                if (c > 0) { pair_add(hi, lo, sv); o += c; }
            }
        }
#pragma unroll
        for (int k = 16; k > 0; k >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, k), l2 = __shfl_xor_sync(0xffffffffu, lo, k);
            o += __shfl_xor_sync(0xffffffffu, o, k);
            pair_add(hi, lo, h2);
            lo = __fadd_rn(lo, l2);
        }
        if (vt < 256 && lane == 0) { wh[vt >> 5] = hi; wl[vt >> 5] = lo; wo[vt >> 5] = o; }
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        TableSums t;
        t.hi = 0.0f;
        t.lo = 0.0f;
        t.o = 0;
        for (int w = 0; w < 8; ++w) {
            pair_add(t.hi, t.lo, wh[w]);
            t.lo = __fadd_rn(t.lo, wl[w]);
            t.o += wo[w];
        }
        if (t.o == 0) {
            t.d0 = 1.0f;
        } else {
            const float of = (float)t.o;                  // exact: o <= 2^24
            const float q = __fdiv_rn(t.hi, of);
            const float r = __fadd_rn(__fmaf_rn(-q, of, t.hi), t.lo);
            t.d0 = __fadd_rn(q, __fdiv_rn(r, of));
        }
        t.dbg = t.o == 0 ? 1.0f : (J.bdv_value > 0.0f ? __fdiv_rn(J.bdv_value, t.d0) : J.bdv_scale);
        t.fix_bits = table_fix_bits(J, t.o, t.dbg);
        t.bad = bad;
        tot = t;
    }
    __syncthreads();
    const TableSums t = tot;
    const bool empty = (t.o == 0);
    const bool publish = lead && table != J.dens;
    auto entry = [&](int v, float sv, int c) {
        const float dv = (c > 0 && !empty) ? __fdiv_rn(sv, __fmul_rn((float)c, t.d0)) : 0.0f;
        table[v] = dv;
        if (publish) J.dens[v] = dv;
    };
    if (cache) {
        if (tid < 256) {
#pragma unroll
            for (int q = 0; q < kTableSlots; ++q)
                if (tid + 256 * q < R) entry(tid + 256 * q, s_c[q], c_c[q]);
            for (int v = tid + 256 * kTableSlots; v < R; v += 256) entry(v, J.values[v], __ldcg(J.counts + v));
        }
    } else {
        for (int v = tid; v < R; v += nt) entry(v, J.values[v], __ldcg(J.counts + v));
    }
    if (tid == 0) {
        table[R] = t.dbg;
        if (publish) J.dens[R] = t.dbg;
        if (lead) table_state(J, t, raster_it);
    }
    return t;
}

// The job's per-iteration state from the table's sums (one thread): value
// error, background pixel count, d0 and background value, total mass (and
// its copy by iteration parity, for the area kernel that may run next to the
// next iteration's table) and the fixed-point bits.
__device__ inline void table_state(const Job& J, const TableSums& t, int raster_it) {
    if (t.bad) atomicExch(&J.st->error, INIM_E_VALUE);
    const long long o_bg = (long long)J.n * J.n - t.o;
    J.counts[J.n_regions] = (int)o_bg;
    JobState* st = J.st;
    const bool empty = (t.o == 0);
    const double s = (double)t.hi + (double)t.lo;
    const double d0 = empty ? 1.0 : s / (double)t.o;
    const double bdv_abs = J.bdv_value > 0.0f ? (double)J.bdv_value : (double)J.bdv_scale * d0;
    const double mass = empty ? 1.0 : s + bdv_abs * (double)o_bg;
    st->d0 = d0;
    st->bdv_abs = bdv_abs;
    st->mass = mass;
    st->mass_it[raster_it & 1] = mass;
    st->raster_it = raster_it + 1;
    st->fix_bits = t.fix_bits;
}

}  // namespace inim
