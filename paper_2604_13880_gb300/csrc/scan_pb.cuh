// Parallel-rows form of the band scan (phases 1 and 3 of scan_impl.cuh) for
// short bands: the same outputs, computed with few block barriers.
//
//   stage  all H label rows of the band arrive by bulk copies at once (and,
//          in phase 3, the band's three carry rows);
//   A      each warp takes whole rows: a lane owns contiguous columns of a
//          row segment, so a row's prefix R(x, r) is a lane-serial scan plus
//          one warp scan per segment (shuffles only); R and the row totals go
//          to shared memory;
//   B      after one barrier each thread owns N/256 columns.
//          Phase 1: the band's aggregates with zero carries are direct sums
//          over its rows, S(x) = sum_r R(x, r), E1(x) = sum_r R'(x + H-1-r, r),
//          E2(x) = sum_r R'(x - (H-1-r), r) (R'(x >= N) = row total,
//          R'(x < 0) = 0): no thread needs another's results.
//          Phase 3: the thread walks the H rows with the full rays
//            E1(x, r) = R'(x, r) + E1(x + 1, r - 1)
//            E2(x, r) = R'(x, r) + E2(x - 1, r - 1)
//          started from the carries; the neighbouring value each row needs
//          comes by a shuffle inside a warp and through shared memory across
//          warps (one barrier per row); S accumulates R down its columns and
//          T = E1(i + 1, r - 1) - E2(i - 1, r - 1).
// Phase 1 stores the band's aggregates, phase 3 S, T and the 1-D arrays with
// the same carries and layout as the row-serial form.
#pragma once

// included at the end of scan_impl.cuh (uses its helpers)

namespace inim {

constexpr int kPbThreads = 256;
constexpr int kPbDens = 2048;            // region tables up to this size live in shared memory
static_assert(kFusedTableMax <= kPbDens && kFusedTableMax <= kDensSmem, "fused tables fit in shared memory");

// shared-memory layout (dynamic): R rows padded by one element per 32 (or
// N/32) columns, so that a lane's contiguous run and a thread's column group
// both map to distinct banks
template <class Acc, int N, int H>
struct PbLayout {
    using T = typename Acc::T;
    static constexpr int CW = N / 32;                   // columns per lane in stage A
    static constexpr int kRowStride = N + N / CW;       // padded row of R
    // phase 1 uses the R region for its bins: two [256][CB + H - 1] partial
    // tables and the column sums, later the three prefix arrays
    static constexpr int CB = N / kPbThreads;
    static constexpr size_t kBins = ((size_t)2 * kPbThreads * (CB + H - 1) + N) * sizeof(T);
    static constexpr size_t kRrows = (size_t)H * kRowStride * sizeof(T);
    static constexpr size_t kR = kRrows > kBins ? kRrows : kBins;
    static constexpr size_t kTot = 16 * sizeof(T);
    static constexpr size_t kDens = (size_t)kPbDens * sizeof(float);
    static constexpr size_t kRing = (size_t)H * N * 2;
    static constexpr size_t kCarry = (size_t)3 * N * sizeof(T);     // phase 3: S, E1, E2 carries
    static constexpr size_t kBytes = kR + kTot + kDens + kRing + kCarry;
    static __device__ __forceinline__ int at(int x) { return x + x / CW; }
};

template <class Acc, int N, int H, int PHASE>
__global__ void __launch_bounds__(kPbThreads, (H <= 8 ? 3 : 1)) k_scan_band_pb(const Job* __restrict__ jobs,
                                                             const int2* __restrict__ bmap,
                                                             const float* __restrict__ dtex) {
    using T = typename Acc::T;
    using L = PbLayout<Acc, N, H>;
    constexpr int CW = L::CW;
    constexpr int CB = N / kPbThreads;                 // columns per thread in stage B
    static_assert(H % 8 == 0 && CW % 8 == 0 && CB >= 1, "tile");
    extern __shared__ __align__(128) unsigned char pb_smem[];
    T* Rs = reinterpret_cast<T*>(pb_smem);
    T* rowtot = reinterpret_cast<T*>(pb_smem + L::kR);
    float* dens = reinterpret_cast<float*>(pb_smem + L::kR + L::kTot);
    uint16_t* ring = reinterpret_cast<uint16_t*>(pb_smem + L::kR + L::kTot + L::kDens);
    T* csm = reinterpret_cast<T*>(pb_smem + L::kR + L::kTot + L::kDens + L::kRing);   // [3][N]
    __shared__ uint64_t bars[H + 1];                      // label rows, then the carry rows

    const int2 m = bmap[blockIdx.x];
    const Job J = jobs[m.x];                  // fixed over a run: read before the wait
    const int band = m.y, nb = J.nb, j0 = band * H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool from_labels = (dtex == nullptr);
    if (tid == 0) {
        for (int q = 0; q <= H; ++q) mbar_init(bars + q, 1);
        mbar_init_fence();
        // Phase 3's label rows before the wait: the row kernel that wrote
        // them has completed (phase 1 and the carries, launched after it,
        // have passed their waits before this grid could start).
        if (PHASE == 3 && from_labels)
            for (int q = 0; q < H; ++q)
                tma_load_1d(ring + q * N, J.labels + (size_t)(j0 + q) * N, 2u * N, bars + q);
    }
    __syncthreads();
    pdl_start(J.pdl_early != 0);
    tl_begin(J.tl, PHASE == 1 ? kTlScan1 : kTlScan3);

    // after the wait the bulk copies go out first, and the job's active flag
    // is read together with the loads of the region table (one round trip);
    // a stopped job's block leaves once its copies have landed.
    // stage: every label row of the band, one bulk copy each
    if (PHASE == 1 && from_labels && tid == 0)
        for (int q = 0; q < H; ++q)
            tma_load_1d(ring + q * N, J.labels + (size_t)(j0 + q) * N, 2u * N, bars + q);
    if (PHASE == 3 && tid == 0) {
        // the carry rows of this band: S at band, E1 at nb + band, E2 at 2 nb + band
        const T* carry = reinterpret_cast<const T*>(J.carry);
        constexpr unsigned row_bytes = (unsigned)(N * sizeof(T));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bars + H)),
                     "r"(3u * row_bytes) : "memory");
        for (int k = 0; k < 3; ++k)
            tma_copy_1d(csm + k * N, carry + (size_t)(k * nb + band) * N, row_bytes, bars + H);
    }
    const int act = J.st->active;
    const float* table = J.dens;
    int fix_bits;
    if (PHASE == 1 && from_labels && J.fuse_table) {
        // this iteration's density table, built here (every band block the
        // same; band 0 of an active job publishes it with the job state)
        fix_bits = region_table(J, dens, band == 0 && act).fix_bits;
        table = dens;
    } else {
        if (from_labels && J.n_regions + 1 <= kPbDens) {
            for (int v = tid; v <= J.n_regions; v += kPbThreads) dens[v] = J.dens[v];
            table = dens;
        }
        fix_bits = J.st->fix_bits;
    }
    const float qscale = ldexpf(1.0f, fix_bits);   // fixed-point unit (FIX64 only)

    const int i0 = tid * CB;
    __syncthreads();                                      // region table in shared memory
    if (!act) {
        if (tid == 0) {
            if (from_labels)
                for (int q = 0; q < H; ++q) mbar_wait(bars + q, 0u);
            if (PHASE == 3) mbar_wait(bars + H, 0u);
        }
        tl_end(J.tl, PHASE == 1 ? kTlScan1 : kTlScan3);
        return;
    }

    if constexpr (PHASE == 1) {
        // The band's aggregates at its last row with zero carries need no row
        // prefixes: with d the band's densities (local rows r = 0 .. H-1),
        //   S(x)  = sum_{x' <= x} c(x'),            c(x')  = sum_r d(x', r)
        //   E1(x) = sum_{t <= x + H - 1} D1(t),     D1(t)  = sum_{x' + r = t} d(x', r)
        //   E2(x) = sum_{t <= x} D2(t),             D2(t)  = sum_{x' - r + H - 1 = t} d(x', r)
        // (the sets of pixels that the rays of the recurrences cover).  Each
        // thread bins its CB columns over the H rows (the diagonal bins in a
        // window of CB + H - 1), the partial bins are added across threads in
        // thread order, and three block scans give the prefixes.
        constexpr int NBW = CB + H - 1;                  // a thread's diagonal bins
        constexpr int M = N + H - 1;                     // diagonal bins of the band
        constexpr int BPT = (M + kPbThreads - 1) / kPbThreads;
        T cs[CB], b1[NBW], b2[NBW];
#pragma unroll
        for (int k = 0; k < CB; ++k) cs[k] = Acc::zero();
#pragma unroll
        for (int q = 0; q < NBW; ++q) { b1[q] = Acc::zero(); b2[q] = Acc::zero(); }
        bool ok1 = true;
#pragma unroll
        for (int r = 0; r < H; ++r) {
            float d[CB];
            if (from_labels) {
                ok1 = ok1 && mbar_wait(bars + r, 0u);
                labels_to_density<CB>(smem_labels<CB>(ring + r * N, i0), table, d);
            } else {
#pragma unroll
                for (int k = 0; k < CB; ++k) d[k] = dtex[(size_t)(j0 + r) * N + i0 + k];
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                const T v = Acc::from(d[k], qscale);
                cs[k] = Acc::add(cs[k], v);
                b1[k + r] = Acc::add(b1[k + r], v);
                b2[k + H - 1 - r] = Acc::add(b2[k + H - 1 - r], v);
            }
        }
        if (__syncthreads_or(!ok1)) {
            if (tid == 0) {
                atomicExch(&J.st->error, INIM_E_TIMEOUT);
                for (int q = 0; q < H; ++q) mbar_wait(bars + q, 0u);
            }
            return;
        }
        T* P1 = Rs;                                      // [kPbThreads][NBW] partial D1 bins
        T* P2 = Rs + kPbThreads * NBW;                   // [kPbThreads][NBW] partial D2 bins
#pragma unroll
        for (int q = 0; q < NBW; ++q) { P1[tid * NBW + q] = b1[q]; P2[tid * NBW + q] = b2[q]; }
        __syncthreads();
        // this thread's bins g = tid * BPT + u: the partials of the threads
        // whose windows hold g, in thread order; then the local prefixes
        T f1[BPT], f2[BPT];
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
            const int g = tid * BPT + u;
            T a = Acc::zero(), b = Acc::zero();
            if (g < M) {
                // at most NTB threads hold bin g: t_hi - NTB + 1 .. t_hi, in order
                constexpr int NTB = (NBW + CB - 1) / CB;
                const int t_lo = g >= NBW ? (g - NBW) / CB + 1 : 0;
                const int t_hi = min(kPbThreads - 1, g / CB);
#pragma unroll
                for (int v = 0; v < NTB; ++v) {
                    const int t = t_hi - (NTB - 1) + v;
                    if (t >= t_lo) {
                        a = Acc::add(a, P1[t * NBW + g - t * CB]);
                        b = Acc::add(b, P2[t * NBW + g - t * CB]);
                    }
                }
            }
            f1[u] = u ? Acc::add(f1[u - 1], a) : a;
            f2[u] = u ? Acc::add(f2[u - 1], b) : b;
        }
#pragma unroll
        for (int k = 1; k < CB; ++k) cs[k] = Acc::add(cs[k - 1], cs[k]);
        // block exclusive offsets of the three local totals
        __shared__ T wt[3][kPbThreads / 32];
        T x1 = f1[BPT - 1], x2 = f2[BPT - 1], x3 = cs[CB - 1];
        T i1 = x1, i2 = x2, i3 = x3;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y1 = Acc::shfl_up(i1, o), y2 = Acc::shfl_up(i2, o), y3 = Acc::shfl_up(i3, o);
            if (lane >= o) { i1 = Acc::add(i1, y1); i2 = Acc::add(i2, y2); i3 = Acc::add(i3, y3); }
        }
        if (lane == 31) { wt[0][warp] = i1; wt[1][warp] = i2; wt[2][warp] = i3; }
        __syncthreads();
        // exclusive within the warp (the previous lane's inclusive value),
        // then the earlier warps' totals in order
        T o1 = Acc::shfl_up(i1, 1), o2 = Acc::shfl_up(i2, 1), o3 = Acc::shfl_up(i3, 1);
        if (lane == 0) { o1 = Acc::zero(); o2 = Acc::zero(); o3 = Acc::zero(); }
        for (int w = 0; w < warp; ++w) {
            o1 = Acc::add(wt[0][w], o1); o2 = Acc::add(wt[1][w], o2); o3 = Acc::add(wt[2][w], o3);
        }
        // the prefixes: D1 and D2 to shared memory (read at shifted columns),
        // the column sums' prefix in registers (this thread's own columns)
        T* F1 = Rs;                                      // [M] (the partial bins are read)
        T* F2 = Rs + M;
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
            const int g = tid * BPT + u;
            if (g < M) { F1[g] = Acc::add(o1, f1[u]); F2[g] = Acc::add(o2, f2[u]); }
        }
        T Sagg[CB], a1[CB], a2[CB];
#pragma unroll
        for (int k = 0; k < CB; ++k) Sagg[k] = Acc::add(o3, cs[k]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            a1[k] = F1[i0 + k + H - 1];                  // E1(x) = P1(x + H - 1)
            a2[k] = F2[i0 + k];                          // E2(x) = P2(x)
        }
        tl_end(J.tl, kTlScan1);
        pdl_release();
        T* agg = reinterpret_cast<T*>(J.agg);
        store_row<Acc, CB>(agg + (size_t)band * N + i0, Sagg);
        store_row<Acc, CB>(agg + (size_t)(nb + band) * N + i0, a1);
        store_row<Acc, CB>(agg + (size_t)(2 * nb + band) * N + i0, a2);
        return;
    }

    // A: row prefixes, one warp per row, in segments of 32 x CWS columns
    // (a lane owns CWS contiguous columns of each segment; the segment's
    // offset is the row's running total, so at most CWS prefixes are live)
    constexpr int NSEG = CW > 16 ? CW / 16 : 1;
    constexpr int CWS = CW / NSEG;
    bool ok = true;
    for (int r = warp; r < H; r += kPbThreads / 32) {
        if (from_labels) ok = ok && mbar_wait(bars + r, 0u);
        T seg_off = Acc::zero();
#pragma unroll
        for (int sg = 0; sg < NSEG; ++sg) {
            const int c0 = sg * 32 * CWS + lane * CWS;
            float d[CWS];
            if (from_labels) {
                labels_to_density<CWS>(smem_labels<CWS>(ring + r * N, c0), table, d);
            } else {
                const float* src = dtex + (size_t)(j0 + r) * N + c0;
#pragma unroll
                for (int k = 0; k < CWS; k += 4) {
                    const float4 v = *reinterpret_cast<const float4*>(src + k);
                    d[k] = v.x; d[k + 1] = v.y; d[k + 2] = v.z; d[k + 3] = v.w;
                }
            }
            T run = Acc::zero();
            T p[CWS];
#pragma unroll
            for (int k = 0; k < CWS; ++k) { run = Acc::add(run, Acc::from(d[k], qscale)); p[k] = run; }
            T incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T t = Acc::shfl_up(incl, o);
                if (lane >= o) incl = Acc::add(incl, t);
            }
            const T off = Acc::add(seg_off, Acc::sub(incl, run));
            T* row = Rs + r * L::kRowStride + L::at(c0);
#pragma unroll
            for (int k = 0; k < CWS; ++k) row[k] = Acc::add(off, p[k]);
            seg_off = Acc::add(seg_off, Acc::shfl(incl, 31));
        }
        if (lane == 31) rowtot[r] = seg_off;
    }
    if (PHASE == 3) ok = ok && mbar_wait(bars + H, 0u);   // the carry rows
    if (__syncthreads_or(!ok)) {
        // a staged row never arrived: record it, drain the copies (bounded)
        if (tid == 0) {
            atomicExch(&J.st->error, INIM_E_TIMEOUT);
            for (int q = 0; q < H; ++q) mbar_wait(bars + q, 0u);
            if (PHASE == 3) mbar_wait(bars + H, 0u);
        }
        return;
    }

    // B: this thread's columns over the band's rows
    auto Rp = [&](int x, int r) -> T {                   // R'(x, r)
        if (x >= N) return rowtot[r];
        if (x < 0) return Acc::zero();
        return Rs[r * L::kRowStride + L::at(x)];
    };
    // phase 3: the full rays at the band's rows, each thread its CB columns.
    // They start from the carries (the rays at row j0 - 1) and advance one
    // row at a time; the one value a row needs from beyond a thread's own
    // columns (E1 right of its last column, E2 left of its first) comes from
    // the neighbouring lane by a shuffle, or, at a warp's edge, from the
    // neighbouring warp through shared memory (one barrier per row).  Past
    // the texture's right edge E1 is the row sum so far, past its left edge
    // E2 is 0.
    constexpr int NW = kPbThreads / 32;
    __shared__ T edge1[2][NW], edge2[2][NW];
    T e1[CB], e2[CB], Sacc[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        Sacc[k] = csm[i0 + k];
        e1[k] = csm[N + i0 + k];
        e2[k] = csm[2 * N + i0 + k];
    }
    T rcum = csm[N - 1];                                 // E1 past the right edge at row j0 - 1
    if (lane == 0) edge1[0][warp] = e1[0];
    if (lane == 31) edge2[0][warp] = e2[CB - 1];
    __syncthreads();
    T* STout = reinterpret_cast<T*>(J.ST);
    T* Sout = reinterpret_cast<T*>(J.S);
    T* Tout = reinterpret_cast<T*>(J.T);
    T* Aout = reinterpret_cast<T*>(J.A);
    T* Bout = reinterpret_cast<T*>(J.B);
    T* RCout = reinterpret_cast<T*>(J.rowcum);
#pragma unroll
    for (int r = 0; r < H; ++r) {
        const int j = j0 + r, buf = r & 1;
        // E1(i0 + CB, j - 1) and E2(i0 - 1, j - 1)
        T n1 = Acc::shfl_down(e1[0], 1);
        T n2 = Acc::shfl_up(e2[CB - 1], 1);
        if (lane == 31) n1 = warp + 1 < NW ? edge1[buf][warp + 1] : rcum;
        if (lane == 0) n2 = warp > 0 ? edge2[buf][warp - 1] : Acc::zero();
        // T(i, j) = E1(i + 1, j - 1) - E2(i - 1, j - 1)
        T Tv[CB], Rv[CB];
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            Tv[k] = Acc::sub(k + 1 < CB ? e1[k + 1] : n1, k > 0 ? e2[k - 1] : n2);
            Rv[k] = Rp(i0 + k, r);
            Sacc[k] = Acc::add(Sacc[k], Rv[k]);
        }
        const size_t rowbase = (size_t)j * N + i0;
        if (STout) store_row_pairs<Acc, CB>(STout + 2 * rowbase, Sacc, Tv);
        else {
            store_row<Acc, CB>(Sout + rowbase, Sacc);
            store_row<Acc, CB>(Tout + rowbase, Tv);
        }
        // the rays at row j (ascending for E1, descending for E2: old values)
#pragma unroll
        for (int k = 0; k < CB; ++k) e1[k] = Acc::add(Rv[k], k + 1 < CB ? e1[k + 1] : n1);
#pragma unroll
        for (int k = CB - 1; k >= 0; --k) e2[k] = Acc::add(Rv[k], k > 0 ? e2[k - 1] : n2);
        rcum = Acc::add(rcum, rowtot[r]);
        if (tid == 0) Aout[j] = e1[0];                                           // A(j) = E1(0, j)
        if (tid == kPbThreads - 1) {
            RCout[j] = Sacc[CB - 1];                                             // S(N-1, j)
            if (j < N - 1) Bout[2 * N - 2 - j] = Acc::sub(Sacc[CB - 1], e2[CB - 1]);   // w = N-1-j > 0
        }
        if (j == N - 1) {
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                Aout[i0 + k + N - 1] = e1[k];                                    // A(x+N-1) = E1(x, N-1)
                Bout[i0 + k] = e2[k];                                            // B(x-N+1) = E2(x, N-1)
            }
        }
        if (r + 1 < H) {
            if (lane == 0) edge1[buf ^ 1][warp] = e1[0];
            if (lane == 31) edge2[buf ^ 1][warp] = e2[CB - 1];
            __syncthreads();
        }
    }
    tl_end(J.tl, kTlScan3);
    pdl_release();
}

template <class Acc, int N, int H>
cudaError_t launch_scan_pb(const Job* d_jobs, const BlockMap& band, const BlockMap& carry, const float* dtex,
                           int phase, cudaStream_t s) {
    using L = PbLayout<Acc, N, H>;
    static bool attr_set = false;
    cudaError_t e = cudaSuccess;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_scan_band_pb<Acc, N, H, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_scan_band_pb<Acc, N, H, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)L::kBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int2* bm = band.d_map;
    const int2* cm = carry.d_map;
    if (phase == 0 || phase == 1) e = launch_pdl(k_scan_band_pb<Acc, N, H, 1>, band.n_blocks, kPbThreads, L::kBytes, s,
                                                 d_jobs, bm, dtex);
    if (e == cudaSuccess && (phase == 0 || phase == 2)) e = launch_carry<Acc>(d_jobs, carry, s);
    if (e == cudaSuccess && (phase == 0 || phase == 3))
        e = launch_pdl(k_scan_band_pb<Acc, N, H, 3>, band.n_blocks, kPbThreads, L::kBytes, s, d_jobs, bm, dtex);
    return e;
}

}  // namespace inim
