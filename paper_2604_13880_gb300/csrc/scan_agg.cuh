// Phase 1 of the row-serial band scan (scan_impl.cuh) without row prefixes:
// the band's aggregates at its last row with zero carries are sums of the
// band's densities d(x', r) over pixel sets that the ray recurrences cover,
//   S(x)  = sum_{x' <= x} c(x'),           c(x') = sum_r d(x', r)
//   E1(x) = sum_{t <= x + H - 1} D1(t),    D1(t) = sum_{x' + r = t} d(x', r)
//   E2(x) = sum_{t <= x} D2(t),            D2(t) = sum_{x' - r + H - 1 = t} d(x', r)
// (r = 0 .. H-1 the band's rows).  A block takes the band in sub-bands of
// 8 rows: each thread bins the densities of its CPT columns (its column sums,
// and the diagonal bins of the sub-band in a window of CPT + 7), the partial
// bins are added across threads in thread order into the band's bins (a
// sub-band's bins sit at a shift of 8 s for D1 and H - 8 - 8 s for D2), and
// three block scans give the prefixes.  Two block barriers per sub-band,
// against one per row for the recurrences; the same values in 64-bit fixed
// point, other roundings in FP32.  Labels are read straight from global
// memory, a sub-band ahead.
#pragma once

// included at the end of scan_impl.cuh (uses its helpers)

namespace inim {

constexpr int kAggSub = 8;                 // rows of a sub-band

template <class Acc, int CPT, int NT>
struct AggLayout {
    using T = typename Acc::T;
    static constexpr int NBW = CPT + kAggSub - 1;                    // a thread's diagonal bins
    static constexpr int N = CPT * NT;
    static constexpr int MMAX = N + 63;                              // band bins for H <= 64
    static constexpr size_t kPart = (size_t)2 * NT * NBW * sizeof(T);
    static constexpr size_t kBins = (size_t)2 * MMAX * sizeof(T);
    static constexpr size_t kBytes = kPart + kBins;
};

// inclusive block scan of V values per thread (thread order, then value
// order); returns the exclusive offset of this thread's first value
template <class Acc, int NT, int V>
__device__ __forceinline__ void block_scan3(typename Acc::T (&a)[V], typename Acc::T (&b)[V],
                                            typename Acc::T (&c)[V], typename Acc::T (*wt)[NT / 32]) {
    using T = typename Acc::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int u = 1; u < V; ++u) {
        a[u] = Acc::add(a[u - 1], a[u]);
        b[u] = Acc::add(b[u - 1], b[u]);
        c[u] = Acc::add(c[u - 1], c[u]);
    }
    T i1 = a[V - 1], i2 = b[V - 1], i3 = c[V - 1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y1 = Acc::shfl_up(i1, o), y2 = Acc::shfl_up(i2, o), y3 = Acc::shfl_up(i3, o);
        if (lane >= o) { i1 = Acc::add(i1, y1); i2 = Acc::add(i2, y2); i3 = Acc::add(i3, y3); }
    }
    if (lane == 31) { wt[0][warp] = i1; wt[1][warp] = i2; wt[2][warp] = i3; }
    __syncthreads();
    T o1 = Acc::shfl_up(i1, 1), o2 = Acc::shfl_up(i2, 1), o3 = Acc::shfl_up(i3, 1);
    if (lane == 0) { o1 = Acc::zero(); o2 = Acc::zero(); o3 = Acc::zero(); }
    for (int w = 0; w < warp; ++w) {
        o1 = Acc::add(wt[0][w], o1);
        o2 = Acc::add(wt[1][w], o2);
        o3 = Acc::add(wt[2][w], o3);
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
        a[u] = Acc::add(o1, a[u]);
        b[u] = Acc::add(o2, b[u]);
        c[u] = Acc::add(o3, c[u]);
    }
}

// blocks per SM the register budget aims at: four 256-thread blocks for FP32
// and up to 4 columns a thread (the 72-solve batch's tile), else the default
template <class Acc, int CPT, int NT>
constexpr int agg_min_blocks() { return (sizeof(typename Acc::T) == 4 && CPT <= 4) ? 1024 / NT : 1; }

template <class Acc, int CPT, int NT>
__global__ void __launch_bounds__(NT, (agg_min_blocks<Acc, CPT, NT>())) k_scan_band_agg(const Job* __restrict__ jobs, const int2* __restrict__ bmap,
                                                      const float* __restrict__ dtex) {
    using T = typename Acc::T;
    using L = AggLayout<Acc, CPT, NT>;
    constexpr int NBW = L::NBW, SB = kAggSub;
    constexpr int MSB = L::N + SB - 1;                               // diagonal bins of a sub-band
    constexpr int BPS = (MSB + NT - 1) / NT;                         // of them per thread
    constexpr int BPB = (L::MMAX + NT - 1) / NT;                     // band bins per thread (upper bound)
    extern __shared__ __align__(16) unsigned char agg_smem[];
    T* P1 = reinterpret_cast<T*>(agg_smem);                          // [NT][NBW] partial D1 bins
    T* P2 = P1 + NT * NBW;                                           // [NT][NBW] partial D2 bins
    T* B1 = reinterpret_cast<T*>(agg_smem + L::kPart);              // [M] band D1 bins, then prefixes
    T* B2 = B1 + L::MMAX;
    __shared__ float dens[kDensSmem];
    __shared__ T wt[3][NT / 32];

    const int2 m = bmap[blockIdx.x];
    const Job J = jobs[m.x];                  // fixed over a run: read before the wait
    const int n = L::N, H = J.H, nb = J.nb, band = m.y, j0 = band * H;
    const int M = n + H - 1;
    const int tid = threadIdx.x;
    const int i0 = tid * CPT;
    const bool from_labels = (dtex == nullptr);
    for (int g = tid; g < M; g += NT) { B1[g] = Acc::zero(); B2[g] = Acc::zero(); }
    pdl_start(J.pdl_early != 0);
    tl_begin(J.tl, kTlScan1);
    // the first sub-band's labels, the active flag and the table's loads go out together
    LabelWords<CPT> lw[SB];
#pragma unroll
    for (int r = 0; r < SB; ++r)
        if (from_labels && r < H) lw[r] = load_labels<CPT>(J, j0 + r, i0);
    const int act = J.st->active;
    const float* table = J.dens;
    int fix_bits;
    if (from_labels && J.fuse_table) {
        fix_bits = region_table(J, dens, band == 0 && act).fix_bits;
        table = dens;
    } else {
        if (from_labels && J.n_regions + 1 <= kDensSmem) {
            for (int v = tid; v <= J.n_regions; v += NT) dens[v] = J.dens[v];
            table = dens;
        }
        fix_bits = J.st->fix_bits;
    }
    __syncthreads();                          // the table, the zeroed bins
    if (!act) {
        tl_end(J.tl, kTlScan1);
        return;
    }
    const float qscale = ldexpf(1.0f, fix_bits);   // fixed-point unit (FIX64 only)

    T cs[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) cs[k] = Acc::zero();
    const int nsb = (H + SB - 1) / SB;
    for (int s = 0; s < nsb; ++s) {
        T b1[NBW], b2[NBW];
#pragma unroll
        for (int q = 0; q < NBW; ++q) { b1[q] = Acc::zero(); b2[q] = Acc::zero(); }
#pragma unroll
        for (int r = 0; r < SB; ++r) {
            const int rb = s * SB + r;                                // row within the band
            if (rb < H) {
                float d[CPT];
                if (from_labels) labels_to_density<CPT>(lw[r], table, d);
                else load_density<CPT>(J, dtex, j0 + rb, i0, d);
#pragma unroll
                for (int k = 0; k < CPT; ++k) {
                    const T v = Acc::from(d[k], qscale);
                    cs[k] = Acc::add(cs[k], v);
                    b1[k + r] = Acc::add(b1[k + r], v);
                    b2[k + SB - 1 - r] = Acc::add(b2[k + SB - 1 - r], v);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NBW; ++q) { P1[tid * NBW + q] = b1[q]; P2[tid * NBW + q] = b2[q]; }
        // the next sub-band's labels, in flight across the barrier and the combine
        if (from_labels && s + 1 < nsb) {
#pragma unroll
            for (int r = 0; r < SB; ++r) {
                const int rb = (s + 1) * SB + r;
                if (rb < H) lw[r] = load_labels<CPT>(J, j0 + rb, i0);
            }
        }
        __syncthreads();
        // this thread's sub-band bins: the partials of the threads whose windows
        // hold them, in thread order, into the band's bins
        const int o1 = SB * s, o2 = H - SB - SB * s;                 // shifts of the two families
#pragma unroll
        for (int u = 0; u < BPS; ++u) {
            const int g = tid * BPS + u;
            if (g < MSB) {
                // at most NTB threads hold bin g: t_hi - NTB + 1 .. t_hi, in order
                constexpr int NTB = (NBW + CPT - 1) / CPT;
                const int t_lo = g >= NBW ? (g - NBW) / CPT + 1 : 0;
                const int t_hi = min(NT - 1, g / CPT);
                T a = Acc::zero(), b = Acc::zero();
#pragma unroll
                for (int v = 0; v < NTB; ++v) {
                    const int t = t_hi - (NTB - 1) + v;
                    if (t >= t_lo) {
                        a = Acc::add(a, P1[t * NBW + g - t * CPT]);
                        b = Acc::add(b, P2[t * NBW + g - t * CPT]);
                    }
                }
                if (g + o1 < M) B1[g + o1] = Acc::add(B1[g + o1], a);
                if (g + o2 >= 0 && g + o2 < M) B2[g + o2] = Acc::add(B2[g + o2], b);
            }
        }
        __syncthreads();
    }
    // prefixes of the band's bins (BPB per thread, in place) and of the column sums
    T f1[BPB], f2[BPB], fc[BPB];
#pragma unroll
    for (int u = 0; u < BPB; ++u) {
        const int g = tid * BPB + u;
        f1[u] = g < M ? B1[g] : Acc::zero();
        f2[u] = g < M ? B2[g] : Acc::zero();
        fc[u] = u < CPT ? cs[u] : Acc::zero();     // BPB >= CPT: the column sums ride along
    }
    static_assert(BPB >= CPT, "column sums fit the scan's values per thread");
    block_scan3<Acc, NT, BPB>(f1, f2, fc, wt);
    __syncthreads();                          // every bin read before the prefixes overwrite them
#pragma unroll
    for (int u = 0; u < BPB; ++u) {
        const int g = tid * BPB + u;
        if (g < M) { B1[g] = f1[u]; B2[g] = f2[u]; }
    }
    __syncthreads();
    T Sagg[CPT], a1[CPT], a2[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        Sagg[k] = fc[k];
        a1[k] = B1[i0 + k + H - 1];           // E1(x) = P1(x + H - 1)
        a2[k] = B2[i0 + k];                   // E2(x) = P2(x)
    }
    tl_end(J.tl, kTlScan1);
    pdl_release();
    T* agg = reinterpret_cast<T*>(J.agg);
    store_row<Acc, CPT>(agg + (size_t)band * n + i0, Sagg);
    store_row<Acc, CPT>(agg + (size_t)(nb + band) * n + i0, a1);
    store_row<Acc, CPT>(agg + (size_t)(2 * nb + band) * n + i0, a2);
}

}  // namespace inim
