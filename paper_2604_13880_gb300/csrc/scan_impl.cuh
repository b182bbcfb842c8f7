// Steps 3-4 of the static algorithm (Sec. 4.1): density texture and integral
// images (Sec. 3.1), fused into one reduce-then-scan over full-width row bands.
//
// Stored per pixel: S = alpha (2-D inclusive prefix) and T = alpha_t (top
// wedge: the pixels (i', j') with j' < j and i - (j - j') < i' <= i + (j - j')).
// The other six InIms follow from S, T and the 1-D arrays A, B, rowcum through
// Eq. (1):  beta = S(i, N-1) - S, delta = S(N-1, j) - S, gamma = C - the rest;
// beta_t = A(i+j) - T, gamma_t = B(i-j) - beta_t, delta_t = C - the rest.
//
// Both S and T are causal from the top, so one top-down sweep over rows gives
// them.  With R(i, j) the row prefix of d:
//   S(i, j)  = S(i, j-1) + R(i, j)
//   E1(x, j) = R(x, j) + E1(x+1, j-1)     (R(x >= N) = row total)
//   E2(x, j) = R(x, j) + E2(x-1, j-1)     (R(x < 0) = 0)
//   T(i, j)  = E1(i+1, j-1) - E2(i-1, j-1)
// E1 / E2 sum R along the two upward diagonal rays; their difference is the
// mass of the wedge.  Special values: A(s) = E1(0, s) for s < N and
// A(s) = E1(s-N+1, N-1) beyond; B(w) = E2(w+N-1, N-1) for w <= 0, and for
// w > 0 the complement sum_{i'-j' > w} d = S(N-1, r) - E2(N-1, r), r = N-1-w.
//
// Parallel form (reduce-then-scan over bands of H rows, no inter-block waits):
//   phase 1  per band: band-local S, E1, E2 of the band's last row (zero carry)
//   phase 2  per column / diagonal: carries into every band
//            Sc_b(i) = sum of earlier bands' S aggregates
//            E1c_{b+1}(x) = E1loc_b(x) + E1c_b(x+H)   (x+H >= N: rowcum)
//            E2c_{b+1}(x) = E2loc_b(x) + E2c_b(x-H)   (x-H < 0: 0)
//   phase 3  per band: recompute the rows, add the carries, write S, T, A, B.
// Each thread owns CPT contiguous columns of the full-width band; the row
// prefix is a thread-serial scan plus one warp scan plus a block exclusive
// offset (one __syncthreads per row, double-buffered).
#pragma once

#include "inim_internal.cuh"
#include "tma.cuh"
#include "table.cuh"

namespace inim {

// ---------------------------------------------------------------------------
// accumulator types of the three precisions
// ---------------------------------------------------------------------------
struct AccF32 {
    using T = float;
    static __device__ __forceinline__ T zero() { return 0.0f; }
    static __device__ __forceinline__ T from(float d, float) { return d; }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T shfl_up(T v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
    static __device__ __forceinline__ T shfl_down(T v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
    static __device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    static __device__ __forceinline__ float ratio(T a, T c) { return a / c; }
    static __device__ __forceinline__ double inv(T c) { return (double)(1.0f / c); }
    static __device__ __forceinline__ float scale(T a, double inv_c) { return a * (float)inv_c; }
};

struct AccFix {   // 64-bit fixed point, exact sums
    using T = long long;
    static __device__ __forceinline__ T zero() { return 0; }
    static __device__ __forceinline__ T from(float d, float scale) { return __float2ll_rn(d * scale); }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T shfl_up(T v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
    static __device__ __forceinline__ T shfl_down(T v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
    static __device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    static __device__ __forceinline__ float ratio(T a, T c) { return (float)((double)a / (double)c); }
    static __device__ __forceinline__ double inv(T c) { return 1.0 / (double)c; }
    static __device__ __forceinline__ float scale(T a, double inv_c) { return (float)((double)a * inv_c); }
};

struct AccKahan {   // compensated float pairs: value = hi + lo
    using T = float2;
    static __device__ __forceinline__ T zero() { return make_float2(0.0f, 0.0f); }
    static __device__ __forceinline__ T from(float d, float) { return make_float2(d, 0.0f); }
    static __device__ __forceinline__ T add(T a, T b) {
        // two-sum of the high parts, then fold in the low parts and renormalise
        float s = __fadd_rn(a.x, b.x);
        float bb = __fsub_rn(s, a.x);
        float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
        e = __fadd_rn(e, __fadd_rn(a.y, b.y));
        float hi = __fadd_rn(s, e);
        float lo = __fsub_rn(e, __fsub_rn(hi, s));
        return make_float2(hi, lo);
    }
    static __device__ __forceinline__ T sub(T a, T b) { return add(a, make_float2(-b.x, -b.y)); }
    static __device__ __forceinline__ T shfl_up(T v, int o) {
        return make_float2(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o));
    }
    static __device__ __forceinline__ T shfl_down(T v, int o) {
        return make_float2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
    }
    static __device__ __forceinline__ T shfl(T v, int src) {
        return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
    }
    static __device__ __forceinline__ float ratio(T a, T c) {
        return (float)(((double)a.x + (double)a.y) / ((double)c.x + (double)c.y));
    }
    static __device__ __forceinline__ double inv(T c) { return 1.0 / ((double)c.x + (double)c.y); }
    static __device__ __forceinline__ float scale(T a, double inv_c) {
        return (float)(((double)a.x + (double)a.y) * inv_c);
    }
};

// ---------------------------------------------------------------------------
// density source: labels + per-region table, or a given float texture
// ---------------------------------------------------------------------------
// raw labels of CPT columns (packed u16 pairs)
template <int CPT>
struct LabelWords { unsigned w[(CPT + 1) / 2]; };

template <int CPT>
__device__ __forceinline__ LabelWords<CPT> load_labels(const Job& J, int j, int i0) {
    LabelWords<CPT> L;
    const uint16_t* src = J.labels + (size_t)j * J.n + i0;
    if constexpr (CPT % 8 == 0) {
#pragma unroll
        for (int q = 0; q < CPT / 8; ++q) {
            const uint4 v = reinterpret_cast<const uint4*>(src)[q];
            L.w[4 * q] = v.x; L.w[4 * q + 1] = v.y; L.w[4 * q + 2] = v.z; L.w[4 * q + 3] = v.w;
        }
    } else if constexpr (CPT == 4) {
        const uint2 v = *reinterpret_cast<const uint2*>(src);
        L.w[0] = v.x; L.w[1] = v.y;
    } else if constexpr (CPT == 2) {
        L.w[0] = *reinterpret_cast<const unsigned*>(src);
    } else {
        L.w[0] = src[0];
    }
    return L;
}

template <int CPT>
__device__ __forceinline__ void labels_to_density(const LabelWords<CPT>& L, const float* __restrict__ table,
                                                  float (&d)[CPT]) {
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const unsigned lab = (k & 1) ? (L.w[k >> 1] >> 16) : (L.w[k >> 1] & 0xffffu);
        d[k] = table[lab];
    }
}

template <int CPT>
__device__ __forceinline__ void load_density(const Job& J, const float* __restrict__ dtex, int j,
                                             int i0, float (&d)[CPT]) {
    const size_t base = (size_t)j * J.n + i0;
    if (dtex) {
        if constexpr (CPT % 4 == 0) {
#pragma unroll
            for (int k = 0; k < CPT; k += 4) {
                float4 v = *reinterpret_cast<const float4*>(dtex + base + k);
                d[k] = v.x; d[k + 1] = v.y; d[k + 2] = v.z; d[k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < CPT; ++k) d[k] = dtex[base + k];
        }
        return;
    }
    uint16_t lab[CPT];
    const uint16_t* src = J.labels + base;
    if constexpr (CPT == 8) {
        uint4 v = *reinterpret_cast<const uint4*>(src);
        unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) { lab[2 * k] = w[k] & 0xffffu; lab[2 * k + 1] = w[k] >> 16; }
    } else if constexpr (CPT == 4) {
        uint2 v = *reinterpret_cast<const uint2*>(src);
        lab[0] = v.x & 0xffffu; lab[1] = v.x >> 16; lab[2] = v.y & 0xffffu; lab[3] = v.y >> 16;
    } else if constexpr (CPT == 2) {
        unsigned v = *reinterpret_cast<const unsigned*>(src);
        lab[0] = v & 0xffffu; lab[1] = v >> 16;
    } else {
#pragma unroll
        for (int k = 0; k < CPT; ++k) lab[k] = src[k];
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) d[k] = __ldg(J.dens + lab[k]);
}

template <class Acc, int CPT>
__device__ __forceinline__ void store_row(typename Acc::T* dst, const typename Acc::T (&v)[CPT]) {
    using T = typename Acc::T;
    if constexpr (sizeof(T) == 4 && CPT % 4 == 0) {
#pragma unroll
        for (int k = 0; k < CPT; k += 4)
            reinterpret_cast<float4*>(dst)[k / 4] = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    } else if constexpr (sizeof(T) == 8 && CPT % 2 == 0) {
#pragma unroll
        for (int k = 0; k < CPT; k += 2) {
            T pair[2] = {v[k], v[k + 1]};
            reinterpret_cast<uint4*>(dst)[k / 2] = *reinterpret_cast<const uint4*>(pair);
        }
    } else {
#pragma unroll
        for (int k = 0; k < CPT; ++k) dst[k] = v[k];
    }
}

// interleaved (S, T) pairs of CPT pixels
template <class Acc, int CPT>
__device__ __forceinline__ void store_row_pairs(typename Acc::T* dst, const typename Acc::T (&a)[CPT],
                                                const typename Acc::T (&b)[CPT]) {
    using T = typename Acc::T;
    if constexpr (sizeof(T) == 4 && CPT % 2 == 0) {
#pragma unroll
        for (int k = 0; k < CPT; k += 2)
            reinterpret_cast<float4*>(dst)[k / 2] = make_float4(a[k], b[k], a[k + 1], b[k + 1]);
    } else if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) reinterpret_cast<float2*>(dst)[k] = make_float2(a[k], b[k]);
    } else {
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            T pair[2] = {a[k], b[k]};
            reinterpret_cast<uint4*>(dst)[k] = *reinterpret_cast<const uint4*>(pair);
        }
    }
}

constexpr int kDensSmem = 4096;     // region tables up to this size live in shared memory

template <class Acc, int NT>
struct ScanShared {
    typename Acc::T wtot[2][NT / 32];
    typename Acc::T e1first[2][NT];
    typename Acc::T e2last[2][NT];
    float dens[kDensSmem];
};

// Label rows staged by bulk copies: a ring of DEPTH rows in shared memory, one
// mbarrier per slot; row r lives in slot r % DEPTH and completes the slot's
// barrier phase r / DEPTH.
template <int DEPTH>
struct LabelRing {
    uint16_t* rows;            // [DEPTH][N] (dynamic shared memory)
    uint64_t* bars;            // [DEPTH]
};
constexpr int kLabelDepth = 4;

template <int CPT>
__device__ __forceinline__ LabelWords<CPT> smem_labels(const uint16_t* row, int i0) {
    LabelWords<CPT> L;
    const uint16_t* src = row + i0;
    if constexpr (CPT % 8 == 0) {
#pragma unroll
        for (int q = 0; q < CPT / 8; ++q) {
            const uint4 v = reinterpret_cast<const uint4*>(src)[q];
            L.w[4 * q] = v.x; L.w[4 * q + 1] = v.y; L.w[4 * q + 2] = v.z; L.w[4 * q + 3] = v.w;
        }
    } else if constexpr (CPT == 4) {
        const uint2 v = *reinterpret_cast<const uint2*>(src);
        L.w[0] = v.x; L.w[1] = v.y;
    } else if constexpr (CPT == 2) {
        L.w[0] = *reinterpret_cast<const unsigned*>(src);
    } else {
        L.w[0] = src[0];
    }
    return L;
}

// phase 1 (PHASE == 1) or phase 3 (PHASE == 3) of one band, by a block of NT
// threads; the caller provides the shared memory.  DEPTH > 0: the label rows
// arrive through a ring of bulk copies issued DEPTH rows ahead (ring must
// then be set); DEPTH == 0: each thread loads its labels two rows ahead.
// fuse_table (phase 1 from labels, R + 1 <= kDensSmem): the block builds this
// iteration's density table itself (table.cuh); band 0 publishes it with the
// job state.  keep_fix_bits >= 0: the table is still in sh.dens from this
// block's phase 1 (or in J.dens for more than kDensSmem - 1 regions) and the
// fixed-point bits are given.  fix_bits_out receives the bits used.  Returns
// false (in every thread) when a staged row never arrived.
template <class Acc, int CPT, int NT, int PHASE, int DEPTH = 0>
__device__ inline bool scan_band_body(const Job& J, int band, const float* __restrict__ dtex, ScanShared<Acc, NT>& sh,
                                      LabelRing<DEPTH> ring = {}, bool fuse_table = false, int keep_fix_bits = -1,
                                      int* fix_bits_out = nullptr) {
    using T = typename Acc::T;
    const int n = J.n, H = J.H, nb = J.nb;
    const int j0 = band * H;
    const int rows = min(H, n - j0);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int i0 = tid * CPT;

    T Sacc[CPT], E1[CPT], E2[CPT];
    T e1edge = Acc::zero();             // band-local E1 beyond the right edge
#pragma unroll
    for (int k = 0; k < CPT; ++k) { Sacc[k] = Acc::zero(); E1[k] = Acc::zero(); E2[k] = Acc::zero(); }

    // phase 3 carries
    const T* cS = nullptr;
    const T* c1 = nullptr;
    const T* c2 = nullptr;
    T w1[CPT], w2[CPT];
    T rc_above = Acc::zero();           // rowcum(j0 - 1) = E1 beyond the edge at row j0-1
    if constexpr (PHASE == 3) {
        const T* carry = reinterpret_cast<const T*>(J.carry);
        cS = carry + (size_t)band * n;
        c1 = carry + (size_t)(nb + band) * n;
        c2 = carry + (size_t)(2 * nb + band) * n;
        rc_above = cS[n - 1];
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            Sacc[k] = cS[i0 + k];
            const int x1 = i0 + k + 1;              // E1c at i + r + 1, r = 0
            w1[k] = x1 < n ? c1[x1] : rc_above;
            const int x2 = i0 + k - 1;              // E2c at i - r - 1, r = 0
            w2[k] = x2 >= 0 ? c2[x2] : Acc::zero();
        }
    }

    T* Sout = reinterpret_cast<T*>(J.S);
    T* Tout = reinterpret_cast<T*>(J.T);
    T* STout = reinterpret_cast<T*>(J.ST);
    T* Aout = reinterpret_cast<T*>(J.A);
    T* Bout = reinterpret_cast<T*>(J.B);
    T* RCout = reinterpret_cast<T*>(J.rowcum);

    // density source: a given texture, or labels through the region table
    // (in shared memory when it fits); labels arrive DEPTH rows ahead through
    // the ring, or two rows ahead in registers
    const bool from_labels = (dtex == nullptr);
    constexpr bool kRing = DEPTH > 0;
    const bool use_ring = kRing && from_labels;
    constexpr unsigned kRowBytes = 2u * CPT * NT;
    if constexpr (kRing) {
        if (tid == 0) {
            for (int q = 0; q < DEPTH; ++q) mbar_init(ring.bars + q, 1);
            mbar_init_fence();
        }
        __syncthreads();
        if (use_ring && tid == 0)
            for (int q = 0; q < DEPTH && q < rows; ++q)
                tma_load_1d(ring.rows + q * (CPT * NT), J.labels + (size_t)(j0 + q) * n, kRowBytes, ring.bars + q);
    }
    const float* table = J.dens;
    int fix_bits;
    if (keep_fix_bits >= 0) {
        fix_bits = keep_fix_bits;
        if (from_labels && J.n_regions + 1 <= kDensSmem) table = sh.dens;
    } else if (PHASE == 1 && from_labels && fuse_table) {
        fix_bits = region_table(J, sh.dens, band == 0).fix_bits;
        table = sh.dens;
        __syncthreads();
    } else {
        if (from_labels && J.n_regions + 1 <= kDensSmem) {
            for (int v = tid; v <= J.n_regions; v += NT) sh.dens[v] = J.dens[v];
            table = sh.dens;
            __syncthreads();
        }
        fix_bits = J.st->fix_bits;
    }
    if (fix_bits_out) *fix_bits_out = fix_bits;
    const float qscale = ldexpf(1.0f, fix_bits);   // fixed-point unit (FIX64 only)
    LabelWords<CPT> lw0{}, lw1{};
    float dn[CPT];
    if (from_labels) {
        if (!use_ring) {
            lw0 = load_labels<CPT>(J, j0, i0);
            if (rows > 1) lw1 = load_labels<CPT>(J, j0 + 1, i0);
        }
    } else {
        load_density<CPT>(J, dtex, j0, i0, dn);
    }
    for (int r = 0; r < rows; ++r) {
        const int j = j0 + r;
        float d[CPT];
        bool row_ok = true;
        if (use_ring) {
            const int q = r % DEPTH;
            row_ok = mbar_wait(ring.bars + q, (unsigned)(r / DEPTH) & 1u);
            labels_to_density<CPT>(smem_labels<CPT>(ring.rows + q * (CPT * NT), i0), table, d);
        } else if (from_labels) {
            labels_to_density<CPT>(lw0, table, d);
            lw0 = lw1;
            if (r + 2 < rows) lw1 = load_labels<CPT>(J, j + 2, i0);
        } else {
#pragma unroll
            for (int k = 0; k < CPT; ++k) d[k] = dn[k];
            if (r + 1 < rows) load_density<CPT>(J, dtex, j + 1, i0, dn);   // prefetch
        }

        // thread-local inclusive prefix
        T p[CPT];
        T run = Acc::zero();
#pragma unroll
        for (int k = 0; k < CPT; ++k) { run = Acc::add(run, Acc::from(d[k], qscale)); p[k] = run; }
        // warp inclusive scan of the thread totals
        T incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = Acc::shfl_up(incl, o);
            if (lane >= o) incl = Acc::add(incl, t);
        }
        const int buf = r & 1;
        if (lane == 31) sh.wtot[buf][wid] = incl;
        sh.e1first[buf][tid] = E1[0];
        sh.e2last[buf][tid] = E2[CPT - 1];
        if (__syncthreads_or(!row_ok)) {
            // a staged row never arrived: record it, drain the copies still
            // in flight (bounded), leave the band unfinished
            if (tid == 0) {
                atomicExch(&J.st->error, INIM_E_TIMEOUT);
                for (int rr = r; rr < rows && rr < r + DEPTH; ++rr)
                    mbar_wait(ring.bars + rr % (DEPTH > 0 ? DEPTH : 1), (unsigned)(rr / (DEPTH > 0 ? DEPTH : 1)) & 1u);
            }
            return false;
        }
        // every thread has read this row's slot: refill it DEPTH rows ahead
        if (use_ring && tid == 0 && r + DEPTH < rows) {
            fence_proxy_async_smem();
            tma_load_1d(ring.rows + (r % DEPTH) * (CPT * NT), J.labels + (size_t)(j + DEPTH) * n, kRowBytes,
                        ring.bars + r % DEPTH);
        }
        T off = Acc::sub(incl, run);          // exclusive within the warp
        T rowtot = Acc::zero();
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) {
            const T t = sh.wtot[buf][w];
            if (w < wid) off = Acc::add(off, t);
            rowtot = Acc::add(rowtot, t);
        }
        const T nbr1 = (tid + 1 < NT) ? sh.e1first[buf][tid + 1] : e1edge;     // E1(i0+CPT, j-1) local
        const T nbr2 = (tid > 0) ? sh.e2last[buf][tid - 1] : Acc::zero();      // E2(i0-1, j-1) local

        T Tv[CPT];
        T R[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) R[k] = Acc::add(off, p[k]);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const T e1p = (k + 1 < CPT) ? E1[k + 1] : nbr1;   // E1 local at (i+1, j-1)
            const T e2p = (k > 0) ? E2[k - 1] : nbr2;          // E2 local at (i-1, j-1)
            if constexpr (PHASE == 3) Tv[k] = Acc::sub(Acc::add(e1p, w1[k]), Acc::add(e2p, w2[k]));
            Sacc[k] = Acc::add(Sacc[k], R[k]);
            // E1 / E2 need the old neighbours: build the new rows in p and R
            p[k] = Acc::add(R[k], e1p);       // new E1[k]
            R[k] = Acc::add(R[k], e2p);       // new E2[k]
        }
#pragma unroll
        for (int k = 0; k < CPT; ++k) E1[k] = p[k];
#pragma unroll
        for (int k = 0; k < CPT; ++k) E2[k] = R[k];
        e1edge = Acc::add(e1edge, rowtot);

        if constexpr (PHASE == 3) {
            const size_t rowbase = (size_t)j * n + i0;
            if (STout) {
                store_row_pairs<Acc, CPT>(STout + 2 * rowbase, Sacc, Tv);
            } else {
                store_row<Acc, CPT>(Sout + rowbase, Sacc);
                store_row<Acc, CPT>(Tout + rowbase, Tv);
            }
            if (tid == 0) Aout[j] = Acc::add(E1[0], w1[0]);                      // A(j) = E1(0, j)
            if (tid == NT - 1) {
                RCout[j] = Sacc[CPT - 1];                                       // S(N-1, j)
                if (j < n - 1)                                                  // w = N-1-j > 0
                    Bout[2 * n - 2 - j] = Acc::sub(Sacc[CPT - 1], Acc::add(E2[CPT - 1], w2[CPT - 1]));
            }
            if (j == n - 1) {
#pragma unroll
                for (int k = 0; k < CPT; ++k) {
                    Aout[i0 + k + n - 1] = Acc::add(E1[k], w1[k]);               // A(x+N-1) = E1(x, N-1)
                    Bout[i0 + k] = Acc::add(E2[k], w2[k]);                       // B(x-N+1) = E2(x, N-1)
                }
            }
            // slide the carry windows to row r + 1
            const int rn = r + 1;
#pragma unroll
            for (int k = 0; k < CPT - 1; ++k) w1[k] = w1[k + 1];
            {
                const int x1 = i0 + CPT - 1 + rn + 1;
                w1[CPT - 1] = x1 < n ? c1[x1] : rc_above;
            }
#pragma unroll
            for (int k = CPT - 1; k > 0; --k) w2[k] = w2[k - 1];
            {
                const int x2 = i0 - rn - 1;
                w2[0] = x2 >= 0 ? c2[x2] : Acc::zero();
            }
        }
    }
    if constexpr (PHASE == 1) {
        T* agg = reinterpret_cast<T*>(J.agg);
        store_row<Acc, CPT>(agg + (size_t)band * n + i0, Sacc);
        store_row<Acc, CPT>(agg + (size_t)(nb + band) * n + i0, E1);
        store_row<Acc, CPT>(agg + (size_t)(2 * nb + band) * n + i0, E2);
    }
    return true;
}

template <class Acc, int CPT, int NT, int PHASE>
__global__ void __launch_bounds__(NT) k_scan_band(const Job* __restrict__ jobs,
                                                  const int2* __restrict__ bmap,
                                                  const float* __restrict__ dtex) {
    __shared__ ScanShared<Acc, NT> sh;
    __shared__ uint64_t bars[kLabelDepth];
    extern __shared__ __align__(128) unsigned char scan_ring[];     // [kLabelDepth][CPT * NT] u16
    const int2 m = bmap[blockIdx.x];
    const Job J = jobs[m.x];                  // fixed over a run: read before the wait
    pdl_start(J.pdl_early != 0);
    if (!J.st->active) return;
    tl_begin(J.tl, PHASE == 1 ? kTlScan1 : kTlScan3);
    LabelRing<kLabelDepth> ring{reinterpret_cast<uint16_t*>(scan_ring), bars};
    scan_band_body<Acc, CPT, NT, PHASE, kLabelDepth>(J, m.y, dtex, sh, ring, J.fuse_table != 0);
    tl_end(J.tl, PHASE == 1 ? kTlScan1 : kTlScan3);
    pdl_release();
}

// phase 2: carries.  Each carry is an exclusive prefix sum over the bands b'
// of a value that depends only on (b', q):
//   Sc_b(i)  = sum_{b'<b} aggS_{b'}(i)                                  q = i
//   E1c_b(x) = sum_{b'<b} f1(b', q - (b'+1) H),  x = q - b H,  f1(b', x') =
//              aggE1_{b'}(x') for x' < N, else the band's row-sum total
//   E2c_b(x) = sum_{b'<b} f2(b', q + (b'+1) H),  x = q + b H,  f2 = aggE2 or 0
// One thread per q walks the bands in order; the loads of kU bands are
// issued together before their sums so that they overlap.
constexpr int kCarryU = 16;
__host__ __device__ __forceinline__ int carry_qspace(int n, int nb, int H) {
    return n + 2 * (n + (nb - 1) * H);
}

// One thread's carry chain (kind, q) as a walk over the bands: the term of
// band b sits at column xp = x0 + b dx of the band's aggregate row, index
// x0 + b (N + dx) in the kind's block (zero outside [0, N), except for kind
// 1 past the right edge, where it is the band's row total S(N-1) in the
// kind-0 block); the carry of band b goes to column q + b dx, index
// q + b (N + dx) of the kind's carry block.  dx = 0, -H, +H and
// x0 = q + dx for kinds 0, 1, 2.
template <class Acc>
struct CarryChain {
    using T = typename Acc::T;
    const T* agg;
    T* c;
    int n, kind, q, x0, dx, base;
    __device__ __forceinline__ CarryChain(const Job& J, int kind_, int q_)
        : n(J.n), kind(kind_), q(q_) {
        base = (kind < 0 ? 0 : kind) * J.nb * n;
        agg = reinterpret_cast<const T*>(J.agg);
        c = reinterpret_cast<T*>(J.carry) + base;
        dx = kind == 1 ? -J.H : (kind == 2 ? J.H : 0);
        x0 = q + dx;
    }
    // offset of band b's term in the aggregates, -1 for a zero term
    __device__ __forceinline__ int term_off(int b) const {
        const int xp = x0 + b * dx;
        if ((unsigned)xp < (unsigned)n) return base + x0 + b * (n + dx);
        if (kind == 1 && xp >= n) return b * n + n - 1;
        return -1;
    }
    __device__ __forceinline__ T term(int b) const {
        const int o = term_off(b);
        return o >= 0 ? agg[o] : Acc::zero();
    }
    __device__ __forceinline__ void store(int b, T v) const {
        const int x = q + b * dx;
        if ((unsigned)x < (unsigned)n) c[q + b * (n + dx)] = v;
    }
};

// q in [0, N + 2 span) -> (kind, q within the kind); kind -1 past the end
__device__ __forceinline__ int carry_kind(int& q, int n, int nb, int H) {
    const int span = n + (nb - 1) * H;
    if (q < n) return 0;
    if ((q -= n) < span) return 1;
    if ((q -= span) < span) { q -= (nb - 1) * H; return 2; }
    return -1;
}

template <class Acc>
__device__ inline void scan_carry_body(const Job& J, int q) {
    using T = typename Acc::T;
    const int nb = J.nb;
    const int kind = carry_kind(q, J.n, nb, J.H);
    if (kind < 0) return;
    const CarryChain<Acc> ch(J, kind, q);
    T acc = Acc::zero();
    for (int b0 = 0; b0 < nb; b0 += kCarryU) {
        T v[kCarryU];
#pragma unroll
        for (int u = 0; u < kCarryU; ++u) v[u] = (b0 + u < nb) ? ch.term(b0 + u) : Acc::zero();
#pragma unroll
        for (int u = 0; u < kCarryU; ++u) {
            if (b0 + u < nb) {
                ch.store(b0 + u, acc);
                acc = Acc::add(acc, v[u]);
            }
        }
    }
}

template <class Acc>
__global__ void __launch_bounds__(256) k_scan_carry(const Job* __restrict__ jobs,
                                                    const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const Job J = jobs[m.x];                  // fixed over a run: read before the wait
    pdl_start(J.pdl_early != 0);
    if (!J.st->active) return;
    tl_begin(J.tl, kTlCarry);
    scan_carry_body<Acc>(J, m.y * blockDim.x + threadIdx.x);
    tl_end(J.tl, kTlCarry);
}

// Two-level form of the same carries, for many short bands: a block covers
// 32 consecutive q (the lanes, so loads and stores stay coalesced) times 8
// groups of consecutive bands (the warps).  Each thread sums the terms of its
// group's bands, the 8 group totals are scanned in shared memory, and each
// thread then writes the exclusive prefixes of its own bands.  The same sums
// as the serial walk, associated by group, with 1/8 of its dependent chain.
// Up to 128 bands a thread's terms (at most 16) are loaded in one round and
// kept in registers across the barrier; beyond, they are loaded in rounds of
// kCarryUG and loaded again (L1 hits) for the prefixes.
constexpr int kCarryGroups = 8;
constexpr int kCarryUG = 8;               // loads in flight per thread in the grouped form

// q values per carry block: the grouped form pays off for a small
// (latency-bound) batch once there are many bands (its dependent chain is
// nb / 8 loads instead of nb); a large batch has parallelism enough for the
// serial walk, which moves fewer blocks.
__host__ __device__ inline int carry_q_per_block(int nb, int size_class) {
    return (size_class == 0 && nb >= 32) ? 32 : 256;
}

template <class Acc>
__global__ void __launch_bounds__(32 * kCarryGroups) k_scan_carry_grouped(const Job* __restrict__ jobs,
                                                                const int2* __restrict__ bmap) {
    using T = typename Acc::T;
    constexpr int G = kCarryGroups;
    __shared__ T tot[G][32];
    const int2 m = bmap[blockIdx.x];
    const Job J = jobs[m.x];                  // fixed over a run: read before the wait
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int nb = J.nb;
    int q = m.y * 32 + lane;
    const int kind = carry_kind(q, J.n, nb, J.H);
    const CarryChain<Acc> ch(J, kind, q);
    const int cb = (nb + G - 1) / G;
    const int b_lo = min(nb, g * cb), b_hi = min(nb, b_lo + cb);
    constexpr int HOLD = 128 / G;             // terms a thread keeps in registers across the barrier
    pdl_start(J.pdl_early != 0);
    tl_begin(J.tl, kTlCarry);
    // the active flag is read with the terms (one round trip); the same in
    // every thread of the block
    const int act = J.st->active;
    T s = Acc::zero();
    T v[HOLD];
    if (cb <= HOLD) {
        // all terms of the group in one round of loads, kept for the prefix pass
#pragma unroll
        for (int u = 0; u < HOLD; ++u) v[u] = (kind >= 0 && b_lo + u < b_hi) ? ch.term(b_lo + u) : Acc::zero();
#pragma unroll
        for (int u = 0; u < HOLD; ++u) s = Acc::add(s, v[u]);
    } else if (kind >= 0) {
        for (int b0 = b_lo; b0 < b_hi; b0 += kCarryUG) {
            T w[kCarryUG];
#pragma unroll
            for (int u = 0; u < kCarryUG; ++u) w[u] = (b0 + u < b_hi) ? ch.term(b0 + u) : Acc::zero();
#pragma unroll
            for (int u = 0; u < kCarryUG; ++u) if (b0 + u < b_hi) s = Acc::add(s, w[u]);
        }
    }
    if (!act) {
        tl_end(J.tl, kTlCarry);
        return;
    }
    tot[g][lane] = s;
    __syncthreads();
    if (kind < 0) return;
    T acc = Acc::zero();
    for (int k = 0; k < g; ++k) acc = Acc::add(acc, tot[k][lane]);
    if (cb <= HOLD) {
#pragma unroll
        for (int u = 0; u < HOLD; ++u) {
            if (b_lo + u < b_hi) {
                ch.store(b_lo + u, acc);
                acc = Acc::add(acc, v[u]);
            }
        }
    } else {
        // the terms again (this thread's own loads: L1 hits), now with their carries
        for (int b0 = b_lo; b0 < b_hi; b0 += kCarryUG) {
            T w[kCarryUG];
#pragma unroll
            for (int u = 0; u < kCarryUG; ++u) w[u] = (b0 + u < b_hi) ? ch.term(b0 + u) : Acc::zero();
#pragma unroll
            for (int u = 0; u < kCarryUG; ++u) {
                if (b0 + u < b_hi) {
                    ch.store(b0 + u, acc);
                    acc = Acc::add(acc, w[u]);
                }
            }
        }
    }
    tl_end(J.tl, kTlCarry);
    pdl_release();
}

// the carry kernel of a group: the serial walk, or the grouped form
template <class Acc>
cudaError_t launch_carry(const Job* d_jobs, const BlockMap& carry, cudaStream_t s) {
    const int2* cm = carry.d_map;
    if (carry.q_per_block != 32) return launch_pdl(k_scan_carry<Acc>, carry.n_blocks, 256, 0, s, d_jobs, cm);
    return launch_pdl(k_scan_carry_grouped<Acc>, carry.n_blocks, 32 * kCarryGroups, 0, s, d_jobs, cm);
}

// phase 1 of a row-serial tile: the binned form (scan_agg.cuh) for up to 8
// columns a thread, the row-serial form beyond
template <class Acc, int CPT, int NT>
cudaError_t launch_scan_phase1(const Job* d_jobs, const BlockMap& band, const float* dtex, size_t ring_bytes,
                               cudaStream_t s);

// ---------------------------------------------------------------------------
// launch: one (CPT, NT) instantiation per tile shape, N = CPT * NT
// ---------------------------------------------------------------------------
template <class Acc, int CPT, int NT>
cudaError_t launch_scan_tile(const Job* d_jobs, const BlockMap& band, const BlockMap& carry,
                             const float* dtex, int phase, cudaStream_t s) {
    const int2* bm = band.d_map;
    const int2* cm = carry.d_map;
    constexpr size_t ring_bytes = (size_t)kLabelDepth * CPT * NT * 2;
    static bool attr_set = false;                  // per instantiation: allow the ring above 48 KB in total
    cudaError_t e = cudaSuccess;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_scan_band<Acc, CPT, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_scan_band<Acc, CPT, NT, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (phase == 0 || phase == 1) e = launch_scan_phase1<Acc, CPT, NT>(d_jobs, band, dtex, ring_bytes, s);
    if (e == cudaSuccess && (phase == 0 || phase == 2)) {
        e = launch_carry<Acc>(d_jobs, carry, s);
    }
    if (e == cudaSuccess && (phase == 0 || phase == 3))
        e = launch_pdl(k_scan_band<Acc, CPT, NT, 3>, band.n_blocks, NT, ring_bytes, s, d_jobs, bm, dtex);
    return e;
}

template <class Acc, int N, int H>
cudaError_t launch_scan_pb(const Job* d_jobs, const BlockMap& band, const BlockMap& carry, const float* dtex,
                           int phase, cudaStream_t s);

template <class Acc, int CPT, int NT>
cudaError_t launch_scan_fused_tile(const Job* d_jobs, const BlockMap& band, cudaStream_t s);

// phase 0: the whole scan (the single-pass kernel for a fused tile); 1, 2, 3:
// one phase of the three-kernel form (nothing for a fused tile); 4: only the
// single-pass kernel of a fused tile (for stage timing)
template <class Acc>
cudaError_t launch_scan_acc(const Job* d_jobs, const BlockMap& band, const BlockMap& carry,
                            ScanTile tile, const float* dtex, int phase, cudaStream_t s) {
    const bool fused = tile.fused && tile.cpt > 0 && dtex == nullptr;
    if (phase == 4 && !fused) return cudaSuccess;
    if (fused) {
        if (phase != 0 && phase != 4) return cudaSuccess;
        switch (tile.cpt * 10000 + tile.nt) {
            case 2 * 10000 + 128: return launch_scan_fused_tile<Acc, 2, 128>(d_jobs, band, s);
            case 4 * 10000 + 128: return launch_scan_fused_tile<Acc, 4, 128>(d_jobs, band, s);
            case 2 * 10000 + 256: return launch_scan_fused_tile<Acc, 2, 256>(d_jobs, band, s);
            case 8 * 10000 + 128: return launch_scan_fused_tile<Acc, 8, 128>(d_jobs, band, s);
            case 4 * 10000 + 256: return launch_scan_fused_tile<Acc, 4, 256>(d_jobs, band, s);
            case 8 * 10000 + 256: return launch_scan_fused_tile<Acc, 8, 256>(d_jobs, band, s);
            case 4 * 10000 + 512: return launch_scan_fused_tile<Acc, 4, 512>(d_jobs, band, s);
            case 8 * 10000 + 512: return launch_scan_fused_tile<Acc, 8, 512>(d_jobs, band, s);
            case 16 * 10000 + 64: return launch_scan_fused_tile<Acc, 16, 64>(d_jobs, band, s);
            case 32 * 10000 + 32: return launch_scan_fused_tile<Acc, 32, 32>(d_jobs, band, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (tile.cpt == 0) {                          // parallel-rows form
        switch (tile.n * 100 + tile.H) {
            case 1024 * 100 + 8: return launch_scan_pb<Acc, 1024, 8>(d_jobs, band, carry, dtex, phase, s);
            case 1024 * 100 + 16: return launch_scan_pb<Acc, 1024, 16>(d_jobs, band, carry, dtex, phase, s);
            case 512 * 100 + 8: return launch_scan_pb<Acc, 512, 8>(d_jobs, band, carry, dtex, phase, s);
            case 512 * 100 + 16: return launch_scan_pb<Acc, 512, 16>(d_jobs, band, carry, dtex, phase, s);
            default: return cudaErrorInvalidValue;
        }
    }
    const int key = tile.cpt * 10000 + tile.nt;
    switch (key) {
        case 2 * 10000 + 128: return launch_scan_tile<Acc, 2, 128>(d_jobs, band, carry, dtex, phase, s);
        case 4 * 10000 + 128: return launch_scan_tile<Acc, 4, 128>(d_jobs, band, carry, dtex, phase, s);
        case 2 * 10000 + 256: return launch_scan_tile<Acc, 2, 256>(d_jobs, band, carry, dtex, phase, s);
        case 8 * 10000 + 128: return launch_scan_tile<Acc, 8, 128>(d_jobs, band, carry, dtex, phase, s);
        case 4 * 10000 + 256: return launch_scan_tile<Acc, 4, 256>(d_jobs, band, carry, dtex, phase, s);
        case 8 * 10000 + 256: return launch_scan_tile<Acc, 8, 256>(d_jobs, band, carry, dtex, phase, s);
        case 4 * 10000 + 512: return launch_scan_tile<Acc, 4, 512>(d_jobs, band, carry, dtex, phase, s);
        case 8 * 10000 + 512: return launch_scan_tile<Acc, 8, 512>(d_jobs, band, carry, dtex, phase, s);
        case 16 * 10000 + 64: return launch_scan_tile<Acc, 16, 64>(d_jobs, band, carry, dtex, phase, s);
        case 32 * 10000 + 32: return launch_scan_tile<Acc, 32, 32>(d_jobs, band, carry, dtex, phase, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace inim

#include "scan_pb.cuh"
#include "scan_fused.cuh"
#include "scan_agg.cuh"

namespace inim {

template <class Acc, int CPT, int NT>
cudaError_t launch_scan_phase1(const Job* d_jobs, const BlockMap& band, const float* dtex, size_t ring_bytes,
                               cudaStream_t s) {
    if constexpr (CPT <= 8) {
        using L = AggLayout<Acc, CPT, NT>;
        static bool attr_set = false;
        if (!attr_set) {
            const cudaError_t e = cudaFuncSetAttribute(k_scan_band_agg<Acc, CPT, NT>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kBytes);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        return launch_pdl(k_scan_band_agg<Acc, CPT, NT>, band.n_blocks, NT, L::kBytes, s, d_jobs, band.d_map, dtex);
    } else {
        return launch_pdl(k_scan_band<Acc, CPT, NT, 1>, band.n_blocks, NT, ring_bytes, s, d_jobs, band.d_map, dtex);
    }
}

}  // namespace inim
