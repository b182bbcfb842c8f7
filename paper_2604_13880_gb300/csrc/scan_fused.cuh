// Single-pass form of the band scan (scan_impl.cuh) for large batches: one
// kernel per iteration instead of phase 1 + carries + phase 3.
//
// Every block takes a ticket (an atomic counter, so tickets follow the order
// in which blocks start) and works on band `ticket mod grid` of the block
// table, which lists each job's bands in order.  A block
//   1. runs phase 1 on its band (band-local aggregates S, E1, E2 of the
//      band's last row, the density table built on the way) and publishes
//      the aggregates (status A);
//   2. looks back over the earlier bands of its job: the carries into band b
//      are sums over the bands b' < b (scan_impl.cuh, phase 2)
//        Sc_b(x)  = sum aggS_b'(x)
//        E1c_b(x) = sum f1(b', x + (b - b' - 1) H)     f1 = aggE1, or aggS(N-1) past the right edge
//        E2c_b(x) = sum f2(b', x - (b - b' - 1) H)     f2 = aggE2, or 0 past the left edge
//      A band whose own carries are known publishes its inclusive prefix
//      (the carries into the next band, status P); the look-back adds the
//      aggregates of the bands after the nearest P and that P's prefix.
//      Warp 0 reads the flags of 32 earlier bands at once, and the block
//      adds their terms together;
//   3. publishes its inclusive prefix (P) and runs phase 3 on its band with
//      the carries (the band's labels come again through the bulk-copy ring,
//      from L2: they were read a moment ago).
// A block only waits on bands with smaller tickets, which have started
// already, so the waits cannot deadlock however few blocks are resident.
//
// The look-back sums in 64-bit fixed point (units 2^-f, f the fixed-point
// bits of the iteration's density table, so that no partial sum overflows):
// integer sums do not depend on the order in which the bands are combined,
// so the carries, and every InIm, are the same whichever P a band finds
// (deterministic), and the carries are the exactly rounded sums of the band
// aggregates.  Flags hold (launch epoch << 2 | status); the epoch comes from
// the ticket, so flags need no reset between launches.  Every wait is
// bounded: a band that gives up records INIM_E_TIMEOUT and publishes a
// failure status that ends its successors' waits at once.
#pragma once

// included at the end of scan_impl.cuh (uses its helpers)

namespace inim {

constexpr unsigned kFlagA = 1u, kFlagP = 2u, kFlagFail = 3u;
constexpr long long kLookbackCap = 1LL << 22;    // polls of one look-back wait (~1 s with back-off)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// fixed-point form (units 2^-f) of the accumulator values and back
template <class Acc> struct FixConv;
template <> struct FixConv<AccF32> {
    static __device__ __forceinline__ long long to(float v, float sc, double) { return __float2ll_rn(v * sc); }
    static __device__ __forceinline__ float from(long long c, float isc, double) { return __ll2float_rn(c) * isc; }
};
template <> struct FixConv<AccFix> {    // already integers in units 2^-f
    static __device__ __forceinline__ long long to(long long v, float, double) { return v; }
    static __device__ __forceinline__ long long from(long long c, float, double) { return c; }
};
template <> struct FixConv<AccKahan> {
    static __device__ __forceinline__ long long to(float2 v, float, double sc) {
        return __double2ll_rn((double)v.x * sc) + __double2ll_rn((double)v.y * sc);
    }
    static __device__ __forceinline__ float2 from(long long c, float, double isc) {
        const double d = (double)c * isc;
        const float hi = __double2float_rn(d);
        return make_float2(hi, __double2float_rn(d - (double)hi));
    }
};

struct LookbackShared {
    int n_terms;          // bands of the current window whose terms are added
    int p_band;           // the band whose inclusive prefix closes the look-back, -1 if none yet
    int status;           // 0 continue, 1 done, 2 failed
};

// Carries into `band` (fixed point) for the CPT columns of this thread, by
// look-back over the earlier bands' flags.  Returns false if a wait gave up or
// an earlier band failed.
template <class Acc, int CPT>
__device__ inline bool lookback_carries(const Job& J, int band, unsigned epoch, float sc, double scd,
                                        LookbackShared& lb, long long (&cs)[CPT], long long (&c1)[CPT],
                                        long long (&c2)[CPT]) {
    using T = typename Acc::T;
    const int n = J.n, H = J.H, nb = J.nb;
    const int tid = threadIdx.x, lane = tid & 31;
    const int i0 = tid * CPT;
    const T* agg = reinterpret_cast<const T*>(J.agg);
    const long long* inc = J.binc;
#pragma unroll
    for (int k = 0; k < CPT; ++k) { cs[k] = 0; c1[k] = 0; c2[k] = 0; }
    int base = band - 1;                  // newest band not yet added
    while (base >= 0) {
        if (tid < 32) {
            // warp 0: the flags of bands base, base - 1, ..., base - 31
            long long spins = 0;
            unsigned ns = 32;
            int status = 0;
            for (;;) {
                const int bp = base - lane;
                unsigned st = kFlagP;          // below band 0: acts as an (empty) prefix
                if (bp >= 0) {
                    const unsigned f = ld_acquire_u32(J.bflags + bp);
                    st = ((f >> 2) == epoch) ? (f & 3u) : 0u;
                }
                const unsigned m_p = __ballot_sync(0xffffffffu, st == kFlagP);
                const unsigned m_wait = __ballot_sync(0xffffffffu, st == 0u);
                const unsigned m_fail = __ballot_sync(0xffffffffu, st == kFlagFail);
                const int first_p = m_p ? __ffs(m_p) - 1 : 32;
                const unsigned before = first_p >= 32 ? 0xffffffffu : ((1u << first_p) - 1u) | (1u << first_p);
                if (m_fail & before) { status = 2; break; }
                if (!(m_wait & before)) {
                    // lanes before the first P hold aggregates: take them (and the P)
                    if (lane == 0) {
                        const int bp_p = base - first_p;
                        lb.n_terms = first_p < 32 ? first_p : 32;
                        lb.p_band = (first_p < 32 && bp_p >= 0) ? bp_p : -1;
                        lb.status = first_p < 32 ? 1 : 0;
                    }
                    break;
                }
                if (++spins > kLookbackCap) { status = 2; break; }
                __nanosleep(ns);
                if (ns < 512) ns <<= 1;
            }
            if (status == 2 && lane == 0) lb.status = 2;
        }
        __syncthreads();
        const int nt = lb.n_terms, pb = lb.p_band, done = lb.status;
        if (done == 2) return false;
        // aggregates of bands base .. base - nt + 1 (distance k = band - b' - 1),
        // two bands at a time (their loads are issued together)
#pragma unroll 1
        for (int q = 0; q < nt; q += 2) {
            T s[2][CPT], e1[2][CPT], e2[2][CPT];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const bool on = q + u < nt;
                const int bp = on ? base - q - u : base;
                const int kk = band - bp - 1;
                const T* aS = agg + (size_t)bp * n;
                const T* a1 = agg + (size_t)(nb + bp) * n;
                const T* a2 = agg + (size_t)(2 * nb + bp) * n;
                const T rt = on ? __ldcg(aS + n - 1) : Acc::zero();
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int x = i0 + c;
                    const int x1 = x + kk * H, x2 = x - kk * H;
                    s[u][c] = on ? __ldcg(aS + x) : Acc::zero();
                    e1[u][c] = !on ? Acc::zero() : (x1 < n ? __ldcg(a1 + x1) : rt);
                    e2[u][c] = (on && x2 >= 0) ? __ldcg(a2 + x2) : Acc::zero();
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    cs[c] += FixConv<Acc>::to(s[u][c], sc, scd);
                    c1[c] += FixConv<Acc>::to(e1[u][c], sc, scd);
                    c2[c] += FixConv<Acc>::to(e2[u][c], sc, scd);
                }
            }
        }
        if (pb >= 0) {
            // the inclusive prefix of band pb: the carries into band pb + 1
            const int kk = band - pb - 1;
            const long long rc = __ldcg(inc + (size_t)pb * n + n - 1);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int x = i0 + c;
                const int x1 = x + kk * H, x2 = x - kk * H;
                cs[c] += __ldcg(inc + (size_t)pb * n + x);
                c1[c] += x1 < n ? __ldcg(inc + (size_t)(nb + pb) * n + x1) : rc;
                c2[c] += x2 >= 0 ? __ldcg(inc + (size_t)(2 * nb + pb) * n + x2) : 0LL;
            }
        }
        __syncthreads();                  // lb is rewritten by the next window
        if (done == 1) break;
        base -= 32;
    }
    return true;
}

// resident blocks per SM the register budget aims at: 4 x 256 threads for
// FP32 tiles of up to 4 columns a thread, 2 x 256 otherwise (the phase-3 body
// of the wider tiles and of the 64-bit accumulators needs ~100-160 registers)
template <class Acc, int CPT, int NT>
constexpr int fused_min_blocks() {
    return (sizeof(typename Acc::T) == 4 && CPT <= 4) ? (NT >= 256 ? 1024 / NT : 4) : (NT >= 256 ? (NT >= 512 ? 1 : 2) : 4);
}

template <class Acc, int CPT, int NT>
__global__ void __launch_bounds__(NT, (fused_min_blocks<Acc, CPT, NT>())) k_scan_fused(const Job* __restrict__ jobs, const int2* __restrict__ bmap,
                                                   unsigned long long* __restrict__ ticket) {
    using T = typename Acc::T;
    __shared__ ScanShared<Acc, NT> sh;
    __shared__ uint64_t bars1[kLabelDepth], bars3[kLabelDepth];
    __shared__ unsigned long long s_ticket;
    __shared__ LookbackShared lb;
    extern __shared__ __align__(128) unsigned char scan_ring[];     // [kLabelDepth][CPT * NT] u16
    const int tid = threadIdx.x;
    if (tid == 0) s_ticket = atomicAdd(ticket, 1ull);            // tickets follow the start order
    __syncthreads();
    const unsigned long long tk = s_ticket;
    const int item = (int)(tk % gridDim.x);
    const unsigned epoch = (unsigned)((tk / gridDim.x + 1ull) & 0x3fffffffull);
    const int2 m = bmap[item];
    const Job J = jobs[m.x];                  // fixed over a run: read before the wait
    pdl_start(J.pdl_early != 0);
    if (!J.st->active) return;
    tl_begin(J.tl, kTlScan1);
    const int band = m.y, n = J.n, nb = J.nb, H = J.H;
    uint16_t* ring_rows = reinterpret_cast<uint16_t*>(scan_ring);
    unsigned* my_flag = J.bflags + band;

    // 1. band-local aggregates (and the density table), then status A
    int fix_bits = 0;
    bool ok = scan_band_body<Acc, CPT, NT, 1, kLabelDepth>(J, band, nullptr, sh, LabelRing<kLabelDepth>{ring_rows, bars1},
                                                           J.fuse_table != 0, -1, &fix_bits);
    ok = !__syncthreads_or(!ok);
    if (tid == 0) {
        __threadfence();
        st_release_u32(my_flag, (epoch << 2) | (ok ? kFlagA : kFlagFail));
    }
    if (!ok) return;

    // 2. carries by look-back
    const float sc = ldexpf(1.0f, fix_bits), isc = ldexpf(1.0f, -fix_bits);
    const double scd = ldexp(1.0, fix_bits), iscd = ldexp(1.0, -fix_bits);
    long long cs[CPT], c1[CPT], c2[CPT];
    ok = lookback_carries<Acc, CPT>(J, band, epoch, sc, scd, lb, cs, c1, c2);
    if (!ok) {
        if (tid == 0) {
            atomicExch(&J.st->error, INIM_E_TIMEOUT);
            st_release_u32(my_flag, (epoch << 2) | kFlagFail);
        }
        return;
    }
    // the carries for phase 3 (accumulator type) and, in the prefix buffer,
    // their fixed-point form, which the inclusive prefix needs at shifted columns
    T* carry = reinterpret_cast<T*>(J.carry);
    long long* inc = J.binc;
    const int i0 = tid * CPT;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int x = i0 + c;
        carry[(size_t)band * n + x] = FixConv<Acc>::from(cs[c], isc, iscd);
        carry[(size_t)(nb + band) * n + x] = FixConv<Acc>::from(c1[c], isc, iscd);
        carry[(size_t)(2 * nb + band) * n + x] = FixConv<Acc>::from(c2[c], isc, iscd);
        inc[(size_t)band * n + x] = cs[c];
        inc[(size_t)(nb + band) * n + x] = c1[c];
        inc[(size_t)(2 * nb + band) * n + x] = c2[c];
    }
    __syncthreads();
    // inclusive prefix = carries into band + 1:
    //   S: Sc + aggS;  E1: aggE1(x) + E1c(x + H) (past the edge: Sc(N-1));  E2: aggE2(x) + E2c(x - H)
    const T* agg = reinterpret_cast<const T*>(J.agg);
    long long p0[CPT], p1[CPT], p2[CPT];
    {
        const long long sc_last = __ldcg(inc + (size_t)band * n + n - 1);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int x = i0 + c;
            p0[c] = cs[c] + FixConv<Acc>::to(__ldcg(agg + (size_t)band * n + x), sc, scd);
            const long long r1 = x + H < n ? __ldcg(inc + (size_t)(nb + band) * n + x + H) : sc_last;
            p1[c] = FixConv<Acc>::to(__ldcg(agg + (size_t)(nb + band) * n + x), sc, scd) + r1;
            const long long r2 = x - H >= 0 ? __ldcg(inc + (size_t)(2 * nb + band) * n + x - H) : 0LL;
            p2[c] = FixConv<Acc>::to(__ldcg(agg + (size_t)(2 * nb + band) * n + x), sc, scd) + r2;
        }
    }
    __syncthreads();                      // every shifted read done before the overwrite
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int x = i0 + c;
        inc[(size_t)band * n + x] = p0[c];
        inc[(size_t)(nb + band) * n + x] = p1[c];
        inc[(size_t)(2 * nb + band) * n + x] = p2[c];
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        st_release_u32(my_flag, (epoch << 2) | kFlagP);
        fence_proxy_async_smem();         // the ring's rows were read by the generic proxy
    }
    __syncthreads();

    // 3. the band with its carries (this block's own carry stores are visible
    //    to it after the block barrier)
    scan_band_body<Acc, CPT, NT, 3, kLabelDepth>(J, band, nullptr, sh, LabelRing<kLabelDepth>{ring_rows, bars3}, false,
                                                 fix_bits, nullptr);
    tl_end(J.tl, kTlScan1);
    pdl_release();
}

template <class Acc, int CPT, int NT>
cudaError_t launch_scan_fused_tile(const Job* d_jobs, const BlockMap& band, cudaStream_t s) {
    constexpr size_t ring_bytes = (size_t)kLabelDepth * CPT * NT * 2;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(k_scan_fused<Acc, CPT, NT>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (!band.ticket) return cudaErrorInvalidValue;
    return launch_pdl(k_scan_fused<Acc, CPT, NT>, band.n_blocks, NT, ring_bytes, s, d_jobs, (const int2*)band.d_map,
                      band.ticket);
}

}  // namespace inim
