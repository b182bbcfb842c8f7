// Parallel-rows form of the band scan (phases 1 and 3 of scan_impl.cuh) for
// short bands: the same outputs, computed without a block barrier per row.
//
//   stage  all H label rows of the band arrive by bulk copies at once;
//   A      each warp takes whole rows: a lane owns N/32 contiguous columns,
//          so a row's prefix R(x, r) is a lane-serial scan plus one warp
//          scan (shuffles only); R and the row totals go to shared memory;
//   B      after one barrier each thread owns N/256 columns and walks the H
//          rows: S accumulates R down its columns; the diagonal rays
//            E1(x, r) = R'(x, r) + E1(x + 1, r - 1)   (R'(x >= N) = row total)
//            E2(x, r) = R'(x, r) + E2(x - 1, r - 1)   (R'(x < 0) = 0)
//          are carried in registers over a halo of H columns to the right
//          (E1) and left (E2), so no thread needs a neighbour's results;
//          T = E1(i + 1, r - 1) - E2(i - 1, r - 1) plus the band's carries.
// Phase 1 stores the band's aggregates, phase 3 S, T and the 1-D arrays,
// exactly as the row-serial form does (same carries, same layout).  Phase 3
// stages the band's three carry rows into shared memory by bulk copies next
// to the label rows and reads each thread's windows of them only for stage
// B, so that no carry occupies registers during stage A (at three blocks per
// SM the register budget is 80 a thread).
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
    static constexpr size_t kR = (size_t)H * kRowStride * sizeof(T);
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
    constexpr int W = CB + H;                          // stage-B register window (halo included)
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
    pdl_start(J.pdl_early != 0);
    if (!J.st->active) return;
    tl_begin(J.tl, PHASE == 1 ? kTlScan1 : kTlScan3);
    const int band = m.y, nb = J.nb, j0 = band * H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool from_labels = (dtex == nullptr);

    // stage: every label row of the band, one bulk copy each
    if (tid == 0) {
        for (int q = 0; q <= H; ++q) mbar_init(bars + q, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (from_labels && tid == 0)
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
    const float* table = J.dens;
    int fix_bits;
    if (PHASE == 1 && from_labels && J.fuse_table) {
        // this iteration's density table, built here (every band block the
        // same; band 0 publishes it with the job state)
        fix_bits = region_table(J, dens, band == 0).fix_bits;
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

    // phase-3 carries of this thread's columns and diagonals, read from the
    // staged rows as sliding windows: at row r, c1w[k] = E1 carry at
    // i0 + 1 + k + r and c2w[k] = E2 carry at i0 + k - r - 1 (E1 past the right
    // edge is the row sum above the band, E2 past the left edge is 0); each
    // row shifts both windows by one and reads one new entry of each
    const T* cS = csm;
    T rc_above = Acc::zero();
    T Sacc[CB], c1w[CB], c2w[CB];
    auto C1 = [&](int q) -> T {
        const int x1 = i0 + 1 + q;
        return x1 < N ? csm[N + x1] : rc_above;
    };
    auto C2 = [&](int q) -> T {
        const int x2 = i0 - H + q;
        return x2 >= 0 ? csm[2 * N + x2] : Acc::zero();
    };
    if constexpr (PHASE == 3) {
        rc_above = cS[N - 1];
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            Sacc[k] = cS[i0 + k];
            c1w[k] = C1(k);
            c2w[k] = C2(k + H - 1);
        }
    } else {
#pragma unroll
        for (int k = 0; k < CB; ++k) Sacc[k] = Acc::zero();
    }

    // B: this thread's columns over the band's rows
    auto Rp = [&](int x, int r) -> T {                   // R'(x, r)
        if (x >= N) return rowtot[r];
        if (x < 0) return Acc::zero();
        return Rs[r * L::kRowStride + L::at(x)];
    };
    if constexpr (PHASE == 1) {
        // the band's aggregates at its last row with zero carries, as direct
        // sums over the rows in the order and operand order of the ray
        // recurrences below (so the same values):
        //   S(x) = sum_r R(x, r),  E1(x) = sum_r R'(x + H-1-r, r),  E2(x) = sum_r R'(x - (H-1-r), r)
        T a1[CB], a2[CB];
#pragma unroll
        for (int k = 0; k < CB; ++k) { a1[k] = Acc::zero(); a2[k] = Acc::zero(); }
#pragma unroll
        for (int r = 0; r < H; ++r) {
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                Sacc[k] = Acc::add(Sacc[k], Rp(i0 + k, r));
                a1[k] = Acc::add(Rp(i0 + k + H - 1 - r, r), a1[k]);
                a2[k] = Acc::add(Rp(i0 + k - (H - 1 - r), r), a2[k]);
            }
        }
        tl_end(J.tl, kTlScan1);
        pdl_release();
        T* agg = reinterpret_cast<T*>(J.agg);
        store_row<Acc, CB>(agg + (size_t)band * N + i0, Sacc);
        store_row<Acc, CB>(agg + (size_t)(nb + band) * N + i0, a1);
        store_row<Acc, CB>(agg + (size_t)(2 * nb + band) * N + i0, a2);
        return;
    }
    T e1[W], e2[W];                                      // e1[q] ~ x = i0 + q; e2[q] ~ x = i0 - H + q
#pragma unroll
    for (int q = 0; q < W; ++q) { e1[q] = Acc::zero(); e2[q] = Acc::zero(); }
    T* STout = reinterpret_cast<T*>(J.ST);
    T* Sout = reinterpret_cast<T*>(J.S);
    T* Tout = reinterpret_cast<T*>(J.T);
    T* Aout = reinterpret_cast<T*>(J.A);
    T* Bout = reinterpret_cast<T*>(J.B);
    T* RCout = reinterpret_cast<T*>(J.rowcum);
#pragma unroll
    for (int r = 0; r < H; ++r) {
        const int j = j0 + r;
        if constexpr (PHASE == 3) {
            // T from the previous row's local rays plus the carries
            T Tv[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                const T a = Acc::add(e1[k + 1], c1w[k]);                  // E1(i + 1, j - 1)
                const T b = Acc::add(e2[H + k - 1], c2w[k]);              // E2(i - 1, j - 1)
                Tv[k] = Acc::sub(a, b);
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) Sacc[k] = Acc::add(Sacc[k], Rp(i0 + k, r));
            const size_t rowbase = (size_t)j * N + i0;
            if (STout) store_row_pairs<Acc, CB>(STout + 2 * rowbase, Sacc, Tv);
            else {
                store_row<Acc, CB>(Sout + rowbase, Sacc);
                store_row<Acc, CB>(Tout + rowbase, Tv);
            }
        }
        // advance the rays to row r (old values of row r - 1 shift by one column)
#pragma unroll
        for (int q = 0; q < W; ++q) e1[q] = Acc::add(Rp(i0 + q, r), q + 1 < W ? e1[q + 1] : Acc::zero());
#pragma unroll
        for (int q = W - 1; q >= 0; --q) e2[q] = Acc::add(Rp(i0 - H + q, r), q > 0 ? e2[q - 1] : Acc::zero());
        if constexpr (PHASE == 3) {
            if (tid == 0) Aout[j] = Acc::add(e1[0], c1w[0]);                         // A(j) = E1(0, j)
            if (tid == kPbThreads - 1) {
                RCout[j] = Sacc[CB - 1];                                             // S(N-1, j)
                if (j < N - 1)                                                       // w = N-1-j > 0
                    Bout[2 * N - 2 - j] = Acc::sub(Sacc[CB - 1], Acc::add(e2[H + CB - 1], c2w[CB - 1]));
            }
            if (j == N - 1) {
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    Aout[i0 + k + N - 1] = Acc::add(e1[k], c1w[k]);                 // A(x+N-1) = E1(x, N-1)
                    Bout[i0 + k] = Acc::add(e2[H + k], c2w[k]);                      // B(x-N+1) = E2(x, N-1)
                }
            }
            if (r + 1 < H) {                                 // the windows of row r + 1
#pragma unroll
                for (int k = 0; k < CB - 1; ++k) c1w[k] = c1w[k + 1];
                c1w[CB - 1] = C1(CB + r);
#pragma unroll
                for (int k = CB - 1; k > 0; --k) c2w[k] = c2w[k - 1];
                c2w[0] = C2(H - 2 - r);
            }
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
