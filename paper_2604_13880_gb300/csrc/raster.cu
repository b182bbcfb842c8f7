// Step 2 of the static algorithm (Sec. 4.1): rasterise the current region
// polygons into a label texture and count the pixel area o(v) of every region.
//
// Exact integer rule (shared reading with the oracle): vertices snap to
// X = rint(x 2^(k+8)); pixel (i, j) has its centre at (256 i + 128, 256 j + 128);
// an edge ordered so that Y0 < Y1 counts for a centre iff Y0 <= Yc < Y1 and
// (Xc - X0)(Y1 - Y0) >= (X1 - X0)(Yc - Y0).  For the centres of row j that is
// exactly the columns i >= c with
//   c = ceil(((X1 - X0)(Yc - Y0) + (X0 - 128)(Y1 - Y0)) / (256 (Y1 - Y0))).
// A pixel is inside region v iff v's crossing count is odd; inside several
// regions it takes the smallest id and the overlap flag is raised.
//
// Kernels (edge-parallel, then row-parallel; no per-pixel global atomics):
//   k_crossings    two edges per lane: (region << 16 | c) appended to the
//                  fixed-stride bucket of every row the edge crosses (no
//                  histogram or prefix pass: each bucket holds up to 2048 keys;
//                  the rule in 32-bit integers where the end points allow)
//   k_raster_rows  warp per row (a block's 8 rows spread over the texture):
//                  sort the row's keys in registers, pair them
//                  into spans, enter the spans into a shared-memory difference
//                  array and build every label by one striped prefix pass
//                  (pixels inside two spans resolved to the smallest region);
//                  rows with more than 256 crossings are finished by the
//                  block-per-row path of the same block
//   k_density_table the density table (table.cuh), only for maps of more than
//                  2047 regions (otherwise scan phase 1 builds it)
#include "raster_impl.cuh"

namespace inim {

namespace {

// Empty buckets and restarted iteration-parity counters (a block per job) at
// the start of a run.
__global__ void __launch_bounds__(256) k_raster_reset(const Job* __restrict__ jobs) {
    const Job& J = jobs[blockIdx.x];
    pdl_start(J.pdl_early != 0);
    if (!J.st->active) return;
    if (threadIdx.x == 0) {
        J.st->raster_it = 0;
        J.st->area_it = 0;
    }
    reset_buckets_block(J);
}

// The crossing keys of the current vertex positions, one lane per edge, the
// crossings spread over each warp; the first edge block of a job also clears
// its pixel counts and big-row list.
__global__ void __launch_bounds__(256, 5) k_crossings(const Job* __restrict__ jobs, const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];                 // (job, item of kEdgesPerItem edges)
    const Job J = jobs[m.x];
    // the job's fields and the mesh (edges, regions) are fixed over a run:
    // read them before the wait; the vertex positions and the active flag after
    bool valid[kEdgesPerLane];
    int2 ab[kEdgesPerLane];
    unsigned reg[kEdgesPerLane];
#pragma unroll
    for (int s = 0; s < kEdgesPerLane; ++s) {
        const int e = m.y * kEdgesPerItem + s * 256 + (int)threadIdx.x;
        valid[s] = e < J.n_edges;
        ab[s] = make_int2(0, 0);
        reg[s] = 0;
        if (valid[s]) {
            ab[s] = J.edges[e];
            reg[s] = (unsigned)J.edge_region[e];
        }
    }
    pdl_start(J.pdl_early != 0);
    const int act = J.st->active;
    float2 p[kEdgesPerLane], q[kEdgesPerLane];
#pragma unroll
    for (int s = 0; s < kEdgesPerLane; ++s) {
        p[s] = q[s] = make_float2(0.0f, 0.0f);
        if (valid[s]) {
            p[s] = J.xy[ab[s].x];
            q[s] = J.xy[ab[s].y];
        }
    }
    if (!act) return;
    tl_begin(J.tl, kTlCrossings);
    emit_crossings_warp<kEdgesPerLane>(J, valid, reg, p, q);
    if (m.y == 0) reset_raster_block(J);
    tl_end(J.tl, kTlCrossings);
    pdl_release();
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32, 5) k_raster_rows(const Job* __restrict__ jobs,
                                                                    const int2* __restrict__ bmap) {
    extern __shared__ __align__(16) unsigned rows_smem[];
    __shared__ int big[kWarpsPerBlock];
    const int2 m = bmap[blockIdx.x];                 // (job, 8 x row item)
    const Job J = jobs[m.x];                         // fixed over a run: read before the wait
    pdl_start(J.pdl_early != 0);
    tl_begin(J.tl, kTlRows);
    const int jb = raster_rows_item(J, m.y, rows_smem, true, true);
    if ((threadIdx.x & 31) == 0) big[threadIdx.x >> 5] = jb;
    __syncthreads();
    // rows with more crossings than a warp holds: the whole block, one at a
    // time, in the (now free) row scratch
    for (int w = 0; w < kWarpsPerBlock; ++w) {
        const int j = big[w];
        if (j >= 0) {
            raster_row_block(J, j, *reinterpret_cast<RowShared*>(rows_smem));
            __syncthreads();
        }
    }
    tl_end(J.tl, kTlRows);
    pdl_release();
}

__global__ void __launch_bounds__(kRowThreads, 1) k_density_table(const Job* __restrict__ jobs) {
    __shared__ RowShared rsh;
    const Job J = jobs[blockIdx.x];           // fixed over a run: read before the wait
    pdl_start(J.pdl_early != 0);
    if (!J.st->active) return;
    density_table_body(J, rsh);
    pdl_release();
}

}  // namespace

cudaError_t raster_setup(int max_n) {
    // the largest row buffer any batch needs (N = 4096); set once
    (void)max_n;
    static bool done = false;
    if (done) return cudaSuccess;
    const int bytes = (int)rows_smem_bytes(1 << kMaxLog2);
    cudaError_t e = cudaFuncSetAttribute(k_raster_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_raster_prologue(const Job* d_jobs, int n_jobs, const BlockMap& edge_blocks, cudaStream_t s) {
    (void)edge_blocks;
    return launch_pdl(k_raster_reset, n_jobs, 256, 0, s, d_jobs);
}

cudaError_t launch_raster_crossings(const Job* d_jobs, const BlockMap& edge_blocks, cudaStream_t s) {
    return launch_pdl(k_crossings, edge_blocks.n_blocks, 256, 0, s, d_jobs, (const int2*)edge_blocks.d_map);
}

cudaError_t launch_raster_rows(const Job* d_jobs, const BlockMap& row_blocks, int max_n, cudaStream_t s) {
    return launch_pdl(k_raster_rows, row_blocks.n_blocks, kWarpsPerBlock * 32, rows_smem_bytes(max_n), s,
                      d_jobs, (const int2*)row_blocks.d_map);
}

// crossing keys into the row buckets, then the rows (rows with more than 256
// crossings are finished by the row kernel's own block)
cudaError_t launch_raster_main(const Job* d_jobs, const BlockMap& edge_blocks, const BlockMap& row_blocks,
                               int max_n, cudaStream_t s) {
    cudaError_t e = launch_raster_crossings(d_jobs, edge_blocks, s);
    if (e == cudaSuccess) e = launch_raster_rows(d_jobs, row_blocks, max_n, s);
    return e;
}

cudaError_t launch_density_table(const Job* d_jobs, int n_jobs, cudaStream_t s) {
    return launch_pdl(k_density_table, n_jobs, 256, 0, s, d_jobs);
}

}  // namespace inim
