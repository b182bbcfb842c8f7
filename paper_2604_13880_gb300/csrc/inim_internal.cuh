// Internal declarations shared by the CUDA translation units of the InIm
// cartogram library: the device-resident job descriptor, per-job state, and
// small device helpers (fixed-point snap, Eq. (2), uniform-density counts).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/inim.h"

namespace inim {

constexpr int kSubBits = 8;          // sub-pixel bits of the fixed-point raster
constexpr int kMaxLog2 = 12;         // N <= 4096
constexpr int kFusedTableMax = 2048; // density table built in the scan when n_regions + 1 <= this
constexpr int kEdgesPerLane = 2;     // edges per lane of the crossing emission
constexpr int kEdgesPerItem = 256 * kEdgesPerLane;   // edges per crossing block (256 lanes)
constexpr int kMinLog2 = 8;          // N >= 256
constexpr int kKeyStride = 2048;     // crossing keys one texture row can hold (fixed-stride buckets)

// Per-solve state living in device memory: the stop rule (Sec. 4.1 defaults)
// and the statistics of the last iteration.
struct JobState {
    int   active;        // 1 while iterating; kernels skip inactive jobs
    int   iters;         // iterations done
    int   max_iters;
    int   stall_window;
    float xi_stop;
    float eps_stop;
    double best_xi;      // best max error so far (stall rule)
    int   since;         // iterations since best_xi improved
    int   pad0;
    double eps, xi;      // errors after the last iteration
    int   foldover;      // a region changed the sign of its area
    int   overlap;       // a pixel lay inside two regions
    int   error;         // INIM_E_* raised on the device (capacity, ...)
    int   fix_bits;      // fraction bits of the fixed-point InIms
    double d0;           // area-weighted mean density of the regions
    double mass;         // total mass in the texture (w(v) = s(v) / mass)
    double mass_it[2];   // the same by iteration parity: the area kernel of an
                         // iteration may run next to the next iteration's density
    int   raster_it;     // density tables built in this run (selects mass_it)
    int   area_it;       // error reductions done in this run (selects mass_it)
    double bdv_abs;      // background density in value units
    int   stop_on_rule;  // 0: run exactly max_iters (no early stop)
    int   blocks_done;   // area blocks finished in this iteration (last one reduces)
    int   n_big;         // rows of this iteration with more crossings than a warp holds
};

// Everything a kernel needs to work on one job.  Lives in device memory; one
// entry per job of a batch.  Texture element (i, j) is at j*n + i.
struct Job {
    // texture
    int n, log2n;
    // map topology (shared by all jobs of one map)
    int n_verts, n_regions, n_edges, n_rings;
    const int2* edges;         // [n_edges] vertex ids, grouped by region
    const int*  edge_region;   // [n_edges]
    const int*  reg_edge_off;  // [n_regions+1] edges of region v: [off[v], off[v+1])
    const int*  reg_ring_off;  // [n_regions+1] into reg_rings
    const int*  reg_rings;     // ring ids grouped by region
    const int*  ring_off;      // [n_rings+1]
    const int*  ring_idx;
    const float* sign0;        // [n_regions] sign of the initial area (0 = none)
    // solve
    float2*      xy;           // [n_verts] vertices, moved in place
    const float* values;       // [n_regions] s(v)
    float lam;                 // blend weight = 1 - shape
    float bdv_scale;
    float bdv_value;           // > 0: background value in value units (Eq. (Mb)), else bdv_scale * d0
    int   precision;           // INIM_FP32 / INIM_FIX64 / INIM_KAHAN
    int   fuse_table;          // 1: the scan's first phase builds the density table (no density kernel)
    int   pdl_early;           // 1: let the next kernel launch at this kernel's start (see pdl_start)
    // raster workspace
    uint16_t* labels;          // [n*n]
    int*      row_cnt;         // [n] crossing keys in each row's bucket (reset by the row rasteriser)
    int*      big_rows;        // [n] rows left to the block-per-row path
    uint32_t* keys;            // [n][kKeyStride] (region << 16 | column), row j's bucket at j * kKeyStride
    int*      counts;          // [n_regions+1] pixel areas o(v); last = background
    float*    dens;            // [n_regions+1] density relative to d0
    // integral images (element type by precision)
    void*  S;                  // [n*n] 2-D inclusive prefix (alpha)
    void*  T;                  // [n*n] top wedge (alpha_t)
    void*  ST;                 // [n*n][2] interleaved (S, T); when set, S and T are not written
    void*  A;                  // [2n-1] A(s) = sum_{i+j<=s} d
    void*  B;                  // [2n-1] w<=0: sum_{i-j<=w} d ; w>0: sum_{i-j>w} d
    void*  rowcum;             // [n] S(n-1, j)
    // band scan workspace
    int    H, nb;              // band height, number of bands
    void*  agg;                // [3][nb][n] band aggregates
    void*  carry;              // [3][nb][n] band carries
    // single-pass scan (large batches): per band a flag (launch epoch << 2 |
    // status) and the inclusive prefix, i.e. the carries into the next band,
    // in 64-bit fixed point
    unsigned*  bflags;         // [nb]
    long long* binc;           // [3][nb][n]
    // areas and errors
    double*   areas;           // [n_regions] signed shoelace areas
    JobState* st;
    unsigned long long* tl;    // kernel timeline (inim_timeline), NULL when off
};

// Warps per region (log2) of a job: about 128 edges per warp, 1..8 warps.
// A property of the map alone, so a job's areas do not depend on the batch.
__host__ __device__ inline int area_warps_log2(int n_edges, int n_regions) {
    const int per = n_regions > 0 ? n_edges / n_regions : 0;
    int lw = 0;
    while (lw < 3 && (128 << lw) < per) ++lw;
    return lw;
}

// ---------------------------------------------------------------------------
// programmatic dependent launch: the kernels of one iteration are launched so
// that the next kernel's grid is set up while the current one runs; every such
// kernel first waits for its predecessor to complete (and its writes to be
// visible).  It lets its own successor launch either at once (pdl_start, for
// jobs with pdl_early: the latency-bound small batches, whose next kernel's
// blocks then hold their SM slots before a concurrent large batch's blocks
// take them) or when its own work is issued (pdl_release at the end, for the
// large batches: waiting blocks would only hold slots the small batches
// need).  Without the launch attribute all of these return at once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_release() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void pdl_start(bool early) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (early) pdl_release();
}

bool pdl_enabled();   // INIM_PDL=0 in the environment turns the attribute off

// ---------------------------------------------------------------------------
// kernel timeline (inim_timeline): per kernel of the iteration and per launch,
// the time the first block starts its work (after the programmatic-launch
// wait) and the time the last block ends, from the GPU's global timer.
// Layout of the buffer (64-bit words): start[k][i] at k * kTlSlots + i,
// end[k][i] at kTlEnd + k * kTlSlots + i, launch i modulo kTlSlots; block
// counters (32-bit) after kTlCount.  Kernel ids: kTl* below.
// ---------------------------------------------------------------------------
constexpr int kTlSlots = 128, kTlKernels = 8, kTlEnd = kTlKernels * kTlSlots, kTlCount = 2 * kTlEnd;
constexpr int kTlWords = kTlCount + kTlKernels;          // + 2 x 8 32-bit counters
enum { kTlCrossings = 0, kTlRows, kTlScan1, kTlCarry, kTlScan3, kTlGather, kTlAreas };

__device__ __forceinline__ unsigned long long tl_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// thread 0 of every block; the first block of a launch records its start
__device__ __forceinline__ void tl_begin(unsigned long long* tl, int k) {
    if (!tl || threadIdx.x != 0) return;
    const unsigned long long t = tl_now();
    unsigned* c = reinterpret_cast<unsigned*>(tl + kTlCount);
    const unsigned old = atomicAdd(c + k, 1u);
    if (old % gridDim.x == 0) tl[k * kTlSlots + (old / gridDim.x) % kTlSlots] = t;
}
// thread 0 of every block; the last block of a launch records its end
__device__ __forceinline__ void tl_end(unsigned long long* tl, int k) {
    if (!tl || threadIdx.x != 0) return;
    const unsigned long long t = tl_now();
    unsigned* c = reinterpret_cast<unsigned*>(tl + kTlCount);
    const unsigned old = atomicAdd(c + kTlKernels + k, 1u);
    if (old % gridDim.x == gridDim.x - 1) tl[kTlEnd + k * kTlSlots + (old / gridDim.x) % kTlSlots] = t;
}

// records msg as the calling thread's last error (inim_last_error) and
// returns code
int set_last_error(int code, const char* msg);

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t s, Args... args) {
    if (grid == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// integer helpers (exact rasterisation rule, Sec. 4.1 step 2 reading)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ long long floor_div(long long a, long long b) {
    // b > 0
    long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
__host__ __device__ __forceinline__ long long ceil_div(long long a, long long b) {
    return -floor_div(-a, b);
}

// X = rint(x * 2^(k+8)) with ties to even (the scale is a power of two, so the
// product is exact).
__device__ __forceinline__ long long snap_coord(float x, float scale) {
    return __float2ll_rn(x * scale);
}

// ---------------------------------------------------------------------------
// Eq. (2): t = (1/2C)(alpha q1 + beta q2 + gamma q3 + delta q4
//                     + alpha_t (x,1) + beta_t (1,y) + gamma_t (x,0) + delta_t (0,y))
// with the anchors q1..q4 of Sec. 3.2 (y downward).  Inputs are the eight
// sums at one pixel and the pixel centre (x, y).
// ---------------------------------------------------------------------------
template <class F>
__device__ __forceinline__ void eq2(F a, F b, F g, F d, F at, F bt, F gt, F dt, F C,
                                    F x, F y, F& tx, F& ty) {
    F q1x, q1y, q3x, q3y, q2x, q2y, q4x, q4y;
    if (y < x) { q1x = F(1); q1y = F(1) + y - x; q3x = x - y; q3y = F(0); }
    else       { q1x = F(1) - y + x; q1y = F(1); q3x = F(0); q3y = y - x; }
    F s = x + y;
    if (s < F(1)) { q2x = s; q2y = F(0); q4x = F(0); q4y = s; }
    else          { q2x = F(1); q2y = s - F(1); q4x = s - F(1); q4y = F(1); }
    F inv = F(1) / (F(2) * C);
    tx = (a * q1x + b * q2x + g * q3x + d * q4x + at * x + bt + gt * x) * inv;
    ty = (a * q1y + b * q2y + g * q3y + d * q4y + at + bt * y + dt * y) * inv;
}

// Pixel counts of the eight regions for a constant texture (exact integers):
// the InIms of t(.; d0) (Sec. 4.1 step 1) in closed form.
struct Counts8 { long long a, b, g, d, at, bt, gt, dt, C; };

__host__ __device__ __forceinline__ long long anti_prefix_count(long long s, long long n) {
    // #{(i', j') in [0,n)^2 : i' + j' <= s}; the complement of s' = 2n-2-s-1
    if (s < 0) return 0;
    if (s >= 2 * n - 2) return n * n;
    if (s <= n - 1) return (s + 1) * (s + 2) / 2;
    long long m = 2 * n - 3 - s;          // i'+j' > s  <=>  (n-1-i')+(n-1-j') <= m
    return n * n - (m + 1) * (m + 2) / 2;
}

__host__ __device__ __forceinline__ Counts8 uniform_counts(int i, int j, int n) {
    Counts8 c;
    long long I = i, J = j, N = n;
    c.C = N * N;
    c.a = (I + 1) * (J + 1);
    c.b = (I + 1) * (N - 1 - J);
    c.g = (N - 1 - I) * (N - 1 - J);
    c.d = (N - 1 - I) * (J + 1);
    // left wedge: row j' holds max(0, i + 1 - |j' - j|) pixels
    long long m = I + 1;
    long long k1 = I < J ? I : J;
    long long k2 = I < (N - 1 - J) ? I : (N - 1 - J);
    long long L = m + (k1 * m - k1 * (k1 + 1) / 2) + (k2 * m - k2 * (k2 + 1) / 2);
    long long A = anti_prefix_count(I + J, N);
    long long B = anti_prefix_count(I - J + N - 1, N);   // i'-j' <= w  <=>  i'+(n-1-j') <= w+n-1
    c.bt = L;
    c.at = A - L;
    c.gt = B - L;
    c.dt = c.C - c.bt - c.at - c.gt;
    return c;
}

// t(x, y; d0) at pixel (i, j) in float, from the exact counts.
__device__ __forceinline__ float2 t_uniform(int i, int j, int n) {
    Counts8 c = uniform_counts(i, j, n);
    float inv_n = 1.0f / (float)n;
    float x = ((float)i + 0.5f) * inv_n, y = ((float)j + 0.5f) * inv_n;
    float tx, ty;
    eq2<float>((float)c.a, (float)c.b, (float)c.g, (float)c.d, (float)c.at, (float)c.bt,
               (float)c.gt, (float)c.dt, (float)c.C, x, y, tx, ty);
    return make_float2(tx, ty);
}

// ---------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
struct BlockMap {            // block -> (job, first item) tables for one kernel
    int2* d_map = nullptr;   // device [n_blocks]
    int   n_blocks = 0;
    int   q_per_block = 256; // carry maps: q values per block (32 = the grouped carry kernel)
    unsigned long long* ticket = nullptr;   // band maps of single-pass scans: block tickets (device)
};

// band height, columns per thread, threads; cpt == 0 selects the
// parallel-rows band scan (256 threads), which is instantiated per texture
// side n; fused: the single-pass kernel instead of phases 1-3 (row-serial
// form, map jobs)
struct ScanTile { int H; int cpt; int nt; int n = 0; int fused = 0; };

cudaError_t raster_setup(int max_n);   // once per process
cudaError_t launch_raster_prologue(const Job* d_jobs, int n_jobs, const BlockMap& edge_blocks, cudaStream_t s);
cudaError_t launch_raster_main(const Job* d_jobs, const BlockMap& edge_blocks, const BlockMap& row_blocks,
                               int max_n, cudaStream_t s);
cudaError_t launch_raster_crossings(const Job* d_jobs, const BlockMap& edge_blocks, cudaStream_t s);
cudaError_t launch_raster_rows(const Job* d_jobs, const BlockMap& row_blocks, int max_n, cudaStream_t s);
cudaError_t launch_density_table(const Job* d_jobs, int n_jobs, cudaStream_t s);
cudaError_t launch_scan_fp32(const Job* d_jobs, const BlockMap& band, const BlockMap& carry,
                             ScanTile tile, const float* dtex, cudaStream_t s, int phase = 0);
cudaError_t launch_scan_fix64(const Job* d_jobs, const BlockMap& band, const BlockMap& carry,
                              ScanTile tile, const float* dtex, cudaStream_t s, int phase = 0);
cudaError_t launch_scan_kahan(const Job* d_jobs, const BlockMap& band, const BlockMap& carry,
                              ScanTile tile, const float* dtex, cudaStream_t s, int phase = 0);
cudaError_t launch_gather(const Job* d_jobs, const BlockMap& vert_blocks, int precision,
                          cudaStream_t s);
// update_state: 1 = errors + stop rule, 0 = errors only, -1 = areas only
cudaError_t launch_areas_errors(const Job* d_jobs, const BlockMap& region_blocks, int update_state,
                                cudaStream_t s);
cudaError_t launch_displacement(const Job* d_job, const float* xy, int n, float* delta,
                                int precision, cudaStream_t s);
cudaError_t launch_finalize_B(const Job* d_job, int precision, cudaStream_t s);

// persistent form (small FP32 batches, N <= 2048)
int persistent_smem_bytes(int max_n);
void set_wait_cap(long long spins);    // polls of a device-side barrier wait; <= 0: the default
cudaError_t launch_persistent(Job* d_jobs, int n_jobs, const BlockMap& edge, const BlockMap& row,
                              const BlockMap& band, const BlockMap& carry, const BlockMap& vert,
                              const BlockMap& region, int iters, int rounds, const int* job_rounds,
                              const float* const* round_values, float2* const* round_out,
                              JobState* round_init, JobState* const* round_stats, unsigned* bar, int* err,
                              int max_n, int max_blocks, unsigned long long* phase_ns, cudaStream_t s);

// learned warm start
constexpr int kFieldRes = 64;          // CNN input / output resolution
constexpr float kFieldScale = 10.0f;   // the CNN predicts 10 x the displacement
cudaError_t launch_density_pooled(const Job* d_job, int n, int pool, float* out, cudaStream_t s);
cudaError_t launch_apply_field(const Job* d_jobs, const BlockMap& vert_blocks, const float* const* fields, int m,
                               float inv_scale, cudaStream_t s);
int warmstart_predict(const float* x, int B, float* y, cudaStream_t s);   // x [B][r][r], r = warmstart_input_res()
bool warmstart_loaded();
int warmstart_input_res();             // input resolution of the loaded network (64, 128, 256)

// geographic quality measures (Sec. 3.3).  Bounding-box mask layout of one
// region in raster 0 (the map) and 1 (the cartogram): origin (x0, y0), size
// w x h pixels, W words a row at word offset off; W = 0 when the region is
// missing from either raster.
struct QRegion {
    int x0[2], y0[2], w[2], h[2], W[2];
    long long off[2];
};
cudaError_t launch_adjacency(const uint16_t* lab, int log2n, int R, uint32_t* bits, cudaStream_t s);
cudaError_t launch_pair_counts(const uint32_t* a, const uint32_t* b, long long nw, unsigned long long* out,
                               cudaStream_t s);
cudaError_t launch_bbox(const uint16_t* lab, int log2n, int R, int* box, cudaStream_t s);
cudaError_t launch_pack(const uint16_t* lab, int log2n, int R, const QRegion* reg, int which, uint32_t* masks,
                        cudaStream_t s);
cudaError_t launch_correlate(const int2* items, int n_items, const QRegion* reg, const uint32_t* mm,
                             const uint32_t* mc, int* omax, cudaStream_t s);
cudaError_t launch_shape_final(const int* cm, const int* cc, const int* omax, int R, double* per, double* out,
                               cudaStream_t s);
cudaError_t launch_barycentres(const int* reg_ring_off, const int* reg_rings, const int* ring_off,
                               const int* ring_idx, const float2* xy, int R, double2* bary, cudaStream_t s);
int rel_pos_blocks();
cudaError_t launch_rel_pos(const double2* bm, const double2* bc, int R, double* partial, double* out,
                           cudaStream_t s);
constexpr int kQualityChunk = 256;     // translations of one correlation block

// plain (unfused) form: extra full textures of one job
struct PlainWork {
    float*  d   = nullptr;   // [n*n] density
    float*  R   = nullptr;   // [n*n] row prefix
    float*  S   = nullptr;   // [n*n] 2-D prefix
    float*  D1  = nullptr;   // [n*n] diagonal ray sums
    float*  D2  = nullptr;   // [n*n] anti-diagonal ray sums
    float*  L   = nullptr;   // [n*n] left wedge
    float*  ad  = nullptr;   // [2n-1] anti-diagonal sums -> A
    float*  dd  = nullptr;   // [2n-1] diagonal sums -> B
    float2* t0  = nullptr;   // [n*n] t(.; d0), computed once
    float2* fld = nullptr;   // [n*n] displacement field
    int     n   = 0;
};
cudaError_t plain_alloc(PlainWork& w, int n);
void plain_free(PlainWork& w);
cudaError_t plain_iteration(const Job* d_job, const Job& h_job, PlainWork& w, cudaStream_t s);

}  // namespace inim
