// Persistent form of the iteration for small batches: one cooperative launch
// runs every phase of every iteration of every job (and, for cumulative time
// series, every time step, Sec. 4.2), separated by grid-wide barriers, so the
// per-iteration cost is a few barriers instead of eight kernel launches.
//
// Phases per iteration (the same device bodies as the per-step kernels):
//   crossing keys | rows | big rows + density table | scan 1 | carries |
//   scan 3 | gather + move | areas, errors, stop rule
// The barrier is a generation counter with a bounded spin: a wait that
// exceeds its cap records INIM_E_TIMEOUT and the kernel returns (a cooperative
// launch makes every block resident, so the cap is only a safety net).
// FP32 only; N <= 2048 (the band scan runs with the launch's 256 threads, so
// N / 256 columns per thread).
#include "area_impl.cuh"
#include "gather_impl.cuh"
#include "raster_impl.cuh"

namespace inim {

namespace {

constexpr int kPersistThreads = 256;
constexpr long long kSpinCap = 1LL << 24;   // default: ~1-2 s of polling with back-off
long long g_spin_cap = kSpinCap;            // set by inim_set_wait_cap

struct PersistPlan {
    Job* jobs;
    int n_jobs;
    const int2* edge_items;   int n_edge_items;     // (job, item of kEdgesPerItem edges)
    const int2* row_items;    int n_row_items;      // (job, first of 8 rows)
    const int2* band_items;   int n_band_items;     // (job, band)
    const int2* carry_items;  int n_carry_items;    // (job, block of 256 q)
    const int2* vert_items;   int n_vert_items;     // (job, block of 256 vertices)
    const int2* region_items; int n_region_items;   // (job, block of 8 regions)
    int iters;                // iterations per round (jobs stop earlier by their rule)
    int rounds;               // time steps of the longest cumulative series (1 = one solve)
    const int* job_rounds;              // [n_jobs] time steps of each job
    const float* const* round_values;   // [n_jobs] -> [rounds][R] values (rounds > 1)
    float2* const* round_out;           // [n_jobs] -> [rounds][V] results (rounds > 1)
    JobState* round_init;               // [n_jobs] state each round starts from
    JobState* const* round_stats;       // [n_jobs] -> [rounds] final state of every round
    unsigned* bar;            // [2] arrivals, generation
    int* err;
    long long spin_cap;       // polls of a barrier wait before it gives up
    unsigned long long* phase_ns;       // NULL, or [kPhases] time spent up to each barrier (block 0)
};

constexpr int kPhases = 8;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// phase timing: block 0 accumulates the time from the previous barrier to the
// end of this one (work + wait) into phase_ns[phase]
__device__ __forceinline__ void phase_mark(const PersistPlan& P, int phase, unsigned long long& t_prev) {
    if (P.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long t = global_ns();
        P.phase_ns[phase] += t - t_prev;
        t_prev = t;
    }
}

__device__ __forceinline__ bool grid_barrier(const PersistPlan& P) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = P.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(P.bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(P.bar, 0u);
            __threadfence();
            atomicAdd(P.bar + 1, 1u);
        } else {
            long long spins = 0;
            unsigned ns = 32;
            while (*gen == g) {
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
                if (++spins > P.spin_cap) {
                    atomicExch(P.err, INIM_E_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)P.err == 0;
}

__device__ __forceinline__ bool active(const Job& J) { return __ldcg(&J.st->active) != 0; }

template <int PHASE>
__device__ void scan_phase(const PersistPlan& P, unsigned char* smem) {
    auto& sh = *reinterpret_cast<ScanShared<AccF32, kPersistThreads>*>(smem);
    for (int it = blockIdx.x; it < P.n_band_items; it += gridDim.x) {
        const int2 m = P.band_items[it];
        const Job& J = P.jobs[m.x];
        if (!active(J)) continue;
        switch (J.n) {
            case 256: scan_band_body<AccF32, 1, kPersistThreads, PHASE>(J, m.y, nullptr, sh); break;
            case 512: scan_band_body<AccF32, 2, kPersistThreads, PHASE>(J, m.y, nullptr, sh); break;
            case 1024: scan_band_body<AccF32, 4, kPersistThreads, PHASE>(J, m.y, nullptr, sh); break;
            default: scan_band_body<AccF32, 8, kPersistThreads, PHASE>(J, m.y, nullptr, sh); break;
        }
        __syncthreads();
    }
}

__device__ bool one_iteration(const PersistPlan& P, unsigned char* smem) {
    const int tid = threadIdx.x;
    unsigned long long t_prev = (P.phase_ns && blockIdx.x == 0 && tid == 0) ? global_ns() : 0ull;
    // crossing keys into the row buckets; pixel counts cleared
    for (int it = blockIdx.x; it < P.n_edge_items; it += gridDim.x) {
        const int2 m = P.edge_items[it];
        const Job& J = P.jobs[m.x];
        if (active(J)) emit_crossings_item(J, m.y);
    }
    for (int j = blockIdx.x; j < P.n_jobs; j += gridDim.x) {
        const Job& J = P.jobs[j];
        if (active(J)) reset_raster_block(J);
    }
    if (!grid_barrier(P)) return false;
    phase_mark(P, 0, t_prev);
    // rows (one warp per row)
    for (int it = blockIdx.x; it < P.n_row_items; it += gridDim.x) {
        const int2 m = P.row_items[it];
        const Job& J = P.jobs[m.x];
        if (active(J)) raster_rows_item(J, m.y, reinterpret_cast<unsigned*>(smem));
        __syncthreads();
    }
    if (!grid_barrier(P)) return false;
    phase_mark(P, 1, t_prev);
    // big rows + density table (a block per job)
    for (int j = blockIdx.x; j < P.n_jobs; j += gridDim.x) {
        const Job& J = P.jobs[j];
        if (!active(J)) continue;
        RowShared& rsh = *reinterpret_cast<RowShared*>(smem);
        density_table_body(J, rsh);
        __syncthreads();
    }
    if (!grid_barrier(P)) return false;
    phase_mark(P, 2, t_prev);
    scan_phase<1>(P, smem);
    if (!grid_barrier(P)) return false;
    phase_mark(P, 3, t_prev);
    for (int it = blockIdx.x; it < P.n_carry_items; it += gridDim.x) {
        const int2 m = P.carry_items[it];
        const Job& J = P.jobs[m.x];
        if (active(J)) scan_carry_body<AccF32>(J, m.y * kPersistThreads + tid);
    }
    if (!grid_barrier(P)) return false;
    phase_mark(P, 4, t_prev);
    scan_phase<3>(P, smem);
    if (!grid_barrier(P)) return false;
    phase_mark(P, 5, t_prev);
    for (int it = blockIdx.x; it < P.n_vert_items; it += gridDim.x) {
        const int2 m = P.vert_items[it];
        const Job& J = P.jobs[m.x];
        if (active(J)) gather_vertex<AccF32>(J, m.y * kPersistThreads + tid);
    }
    if (!grid_barrier(P)) return false;
    phase_mark(P, 6, t_prev);
    for (int it = blockIdx.x; it < P.n_region_items; it += gridDim.x) {
        const int2 m = P.region_items[it];
        const Job& J = P.jobs[m.x];
        if (active(J)) areas_item(J, m.y, 1);
        __syncthreads();
    }
    const bool ok = grid_barrier(P);
    phase_mark(P, 7, t_prev);
    return ok;
}

__global__ void __launch_bounds__(kPersistThreads, 2) k_persistent(PersistPlan P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    for (int round = 0; round < P.rounds; ++round) {
        for (int k = 0; k < P.iters; ++k) {
            bool any = false;
            for (int j = 0; j < P.n_jobs; ++j) any |= active(P.jobs[j]);
            if (!any) break;
            if (!one_iteration(P, smem)) return;
        }
        // end of a time step: statistics and results out, next values in,
        // state reset (cumulative series keep their vertices)
        for (int j = blockIdx.x; j < P.n_jobs; j += gridDim.x)
            if (tid == 0 && round < P.job_rounds[j]) P.round_stats[j][round] = *P.jobs[j].st;
        if (P.rounds == 1) break;
        for (int it = blockIdx.x; it < P.n_vert_items; it += gridDim.x) {
            const int2 m = P.vert_items[it];
            const Job& J = P.jobs[m.x];
            const int v = m.y * kPersistThreads + tid;
            if (round < P.job_rounds[m.x] && v < J.n_verts)
                P.round_out[m.x][(size_t)round * J.n_verts + v] = J.xy[v];
        }
        for (int j = blockIdx.x; j < P.n_jobs; j += gridDim.x) {
            if (round + 1 >= P.job_rounds[j]) continue;
            const Job& J = P.jobs[j];
            float* vals = const_cast<float*>(J.values);
            const float* src = P.round_values[j] + (size_t)(round + 1) * J.n_regions;
            for (int r = tid; r < J.n_regions; r += kPersistThreads) vals[r] = src[r];
            if (tid == 0) {
                JobState s = P.round_init[j];
                s.foldover = J.st->foldover;         // flags accumulate over the series
                s.overlap = J.st->overlap;
                *J.st = s;
            }
        }
        if (!grid_barrier(P)) return;
    }
}

}  // namespace

void set_wait_cap(long long spins) { g_spin_cap = spins > 0 ? spins : kSpinCap; }

int persistent_smem_bytes(int max_n) {
    size_t a = kRowSharedPadded;
    size_t b = sizeof(ScanShared<AccF32, kPersistThreads>);
    size_t c = kWarpsPerBlock * row_warp_bytes(max_n);
    size_t m = a > b ? a : b;
    return (int)(m > c ? m : c);
}

// Occupancy-sized cooperative launch.  Returns cudaErrorNotSupported when the
// device cannot run cooperative launches.
cudaError_t launch_persistent(Job* d_jobs, int n_jobs, const BlockMap& edge, const BlockMap& row,
                              const BlockMap& band, const BlockMap& carry, const BlockMap& vert,
                              const BlockMap& region, int iters, int rounds, const int* job_rounds,
                              const float* const* round_values, float2* const* round_out,
                              JobState* round_init, JobState* const* round_stats, unsigned* bar, int* err,
                              int max_n, int max_blocks, unsigned long long* phase_ns, cudaStream_t s) {
    int dev = 0, coop = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (!coop) return cudaErrorNotSupported;
    const int smem = persistent_smem_bytes(max_n);
    e = cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent, kPersistThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * sms;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    PersistPlan P;
    P.jobs = d_jobs;
    P.n_jobs = n_jobs;
    P.edge_items = edge.d_map;     P.n_edge_items = edge.n_blocks;
    P.row_items = row.d_map;       P.n_row_items = row.n_blocks;
    P.band_items = band.d_map;     P.n_band_items = band.n_blocks;
    P.carry_items = carry.d_map;   P.n_carry_items = carry.n_blocks;
    P.vert_items = vert.d_map;     P.n_vert_items = vert.n_blocks;
    P.region_items = region.d_map; P.n_region_items = region.n_blocks;
    P.iters = iters;
    P.rounds = rounds;
    P.job_rounds = job_rounds;
    P.round_values = round_values;
    P.round_out = round_out;
    P.round_init = round_init;
    P.round_stats = round_stats;
    P.bar = bar;
    P.err = err;
    P.spin_cap = g_spin_cap;
    P.phase_ns = phase_ns;
    void* args[] = {&P};
    e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void*)k_persistent, grid, kPersistThreads, args, smem, s);
    return e;
}

}  // namespace inim
