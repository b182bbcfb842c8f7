/*
 * inim.h -- C ABI of the GB300 integral-image (InIm) cartogram library.
 *
 * The library computes contiguous cartograms by the iterative
 * density-equalising transformation of "Fast Time-Varying Contiguous
 * Cartograms Using Integral Images" (Molchanov, Rave, Linsen):
 *   per iteration (Sec. 4.1, steps 2-7)
 *     rasterise the region polygons into a label texture and count o(v)
 *     build the density texture d = s(v)/o(v), background = bdv_scale * d0
 *     build the integral images (Sec. 3.1)
 *     evaluate t(x,y;d) - t(x,y;d0) (Eq. 2, Eq. 3) at the pixels around each
 *     vertex, interpolate bilinearly, blend with the shape parameter, move
 *     compute shoelace areas, cartographic errors (Sec. 3.3), stop rule
 *   per time step, in direct or cumulative mode (Sec. 4.2).
 *
 * Conventions shared by every entry point
 *   - Coordinates are in the unit square, x to the right, y downward
 *     (Sec. 3.2).  Vertex arrays are interleaved float pairs (x, y).
 *   - The texture is N x N with N = 2^log2_res, 8 <= log2_res <= 12
 *     (Sec. 3.1: textures of size 2^k x 2^k).  Textures are row-major:
 *     element (i, j) (column i = x, row j = y) is at offset j*N + i.
 *   - Pointers: the caller owns every pointer it passes.  Entry points whose
 *     comment says "host or device" accept either kind of memory (the kind
 *     is queried with cudaPointerGetAttributes); "device" means device memory
 *     of the current CUDA device.  The library copies what it keeps.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  A call first waits for the work already enqueued on
 *     it, runs on streams of the library (inim_quality: on `stream`) and
 *     returns once its results are complete; inim_inims_noalloc instead
 *     enqueues its kernels on `stream` and returns at once.
 *   - Return value: INIM_OK (0) on success, a negative INIM_E_* error code,
 *     or a positive INIM_W_* soft status (results are still written).
 *     Errors leave outputs unspecified; the message of the last error on the
 *     calling thread is available from inim_last_error().
 */
#ifndef INIM_H
#define INIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define INIM_OK                0
#define INIM_E_ARG            -1   /* bad size, index, resolution or pointer */
#define INIM_E_VALUE          -2   /* non-finite or negative region value */
#define INIM_E_CUDA           -3   /* a CUDA runtime call failed */
#define INIM_E_TIMEOUT        -4   /* a device-side wait hit its iteration cap */
#define INIM_E_CAPACITY       -5   /* an internal or caller buffer is too small */
#define INIM_E_STATE          -6   /* call not valid in the current state */
#define INIM_W_NOT_CONVERGED   1   /* stopped by max_iters before xi_stop */
#define INIM_W_FOLDOVER        2   /* a region changed orientation or overlapped */

/* inim_params.mode (Sec. 4.2) */
#define INIM_DIRECT            0   /* every time step starts from the original map */
#define INIM_CUMULATIVE        1   /* every time step starts from the previous result */

/* inim_params.precision of the integral images */
#define INIM_FP32              0   /* float prefix sums */
#define INIM_FIX64             1   /* 64-bit fixed-point prefix sums (exact) */
#define INIM_KAHAN             2   /* compensated (double-float) prefix sums */

/* inim_params.form */
#define INIM_FORM_FUSED        0   /* fused kernels, batched, CUDA graph, device stop */
#define INIM_FORM_PLAIN        1   /* one unfused kernel per step, host stop test */

/* inim_map_create flags */
#define INIM_MAP_DEVICE_PTRS   1   /* all input arrays are device pointers */

typedef struct inim_map inim_map;   /* opaque: device copy of a region map */

/* Parameters of one solve.  Fill with inim_params_default() first. */
typedef struct {
    int32_t log2_res;     /* k, N = 2^k (Sec. 3.1); 8..12; default 10 (Sec. 4.1) */
    float   shape;        /* shape parameter in [0, 1): vertices move by
                             (1 - shape) * displacement per iteration */
    float   bdv_scale;    /* background density = bdv_scale * d0 (Sec. 4.1); default 1 */
    int32_t max_iters;    /* iteration cap per time step; default 512 (Sec. 4.1) */
    float   xi_stop;      /* stop when max error xi < xi_stop; default 0.01; <= 0 off */
    int32_t stall_window; /* stop when xi has not improved for this many
                             iterations; default 32; 0 off */
    float   eps_stop;     /* stop when average error eps < eps_stop; default 0 (off) */
    int32_t mode;         /* INIM_DIRECT or INIM_CUMULATIVE */
    int32_t precision;    /* INIM_FP32, INIM_FIX64 or INIM_KAHAN */
    int32_t form;         /* INIM_FORM_FUSED or INIM_FORM_PLAIN */
    int32_t warm_start;   /* 1: move vertices by the learned field first (needs
                             inim_warmstart_load); default 0 */
    float   bdv_value;    /* > 0: background density in value units per pixel,
                             replacing bdv_scale * d0 (dynamic area, Sec. 4.3,
                             Eq. (Mb): one value per time step from
                             inim_background_values); default 0 (off) */
} inim_params;

/* Per time-step statistics. */
typedef struct {
    int32_t iters;        /* iterations performed */
    float   eps;          /* average cartographic error after the last iteration */
    float   xi;           /* maximum cartographic error after the last iteration */
    int32_t foldover;     /* 1 if a region changed the sign of its area */
    int32_t overlap;      /* 1 if some pixel was inside two regions */
    int32_t status;       /* INIM_OK / INIM_W_* of this step */
} inim_step_stats;

/* One independent solve for inim_run_batch. */
typedef struct {
    const inim_map* map;
    const float*    values;    /* [n_regions] s(v) >= 0; host or device */
    const float*    init_xy;   /* [n_verts*2] start vertices, NULL = the map's own; host or device */
    float*          out_xy;    /* [n_verts*2] result; host or device */
    inim_params     params;    /* mode is ignored: every job is one time step */
    inim_step_stats* stats;    /* NULL or one host struct */
} inim_job;

/* One time series for inim_run_series. */
typedef struct {
    const inim_map* map;
    const float*    values;    /* [T*n_regions] s_t(v); host or device */
    int32_t         T;         /* time steps */
    const float*    init_xy;   /* [n_verts*2] start vertices, NULL = the map's own; host or device */
    float*          out_xy;    /* [T*n_verts*2] vertices after each step; host or device */
    inim_params     params;    /* mode: INIM_DIRECT or INIM_CUMULATIVE; fused form */
    inim_step_stats* stats;    /* NULL or [T] host structs */
} inim_series;

/* Defaults of Sec. 4.1: 1024^2, stop at xi < 0.01 / 32-iteration stall / 512 iterations. */
void inim_params_default(inim_params* p);

/* Text of a status code; static storage. */
const char* inim_status_string(int status);

/* Message of the last error reported on the calling thread ("" if none). */
const char* inim_last_error(void);

/*
 * Background values of a time series whose map area follows its global
 * integral (dynamic area, Sec. 4.3, Eq. (Mb)); host memory, no GPU work.
 *   values        [T*n_regions] host s_t(v) >= 0.
 *   a_min, a_max  area fractions of the map at the smallest and the largest
 *                 global integral M(t) = sum_v s_t(v) over the selected
 *                 steps [t0, t1]; 0 < a_min < a_max < 1.
 *   t0, t1        selected steps; t1 < 0 means T - 1.
 *   bdv           [T] out: the background value of step t in value units per
 *                 pixel, M_b(t) / ((1 - A(t)) N^2) with A(t) interpolated
 *                 linearly in M(t) between a_min and a_max (clipped to them
 *                 outside [t0, t1]; a_max when M is constant) and
 *                 M_b(t) = M(t) (1 - A(t)) / A(t).  Pass bdv[t] as
 *                 inim_params.bdv_value of the solve of step t.
 *   area_fraction [T] out A(t), or NULL.
 * Errors: INIM_E_ARG for NULL pointers or sizes, fractions or steps out of
 * range; INIM_E_VALUE for a negative or non-finite value.
 */
int inim_background_values(const float* values, int32_t T, int32_t n_regions, int32_t log2_res, double a_min,
                           double a_max, int32_t t0, int32_t t1, double* bdv, double* area_fraction);

/*
 * Values of an animation with frames_per_step frames per time step (Sec. 5.5:
 * the in-between frames interpolate the statistical data linearly between
 * consecutive steps, and every frame gets a cartogram of its own, e.g. one
 * inim_run over the result); host memory, no GPU work.
 *   values [T*n_regions] host s_t(v) >= 0.
 *   out    [((T-1)*frames_per_step + 1)*n_regions] host: frame t f + q
 *          (0 <= q < f) = (1 - q/f) s_t + (q/f) s_{t+1} in double, rounded to
 *          float; the last frame is the last step.
 * Errors: INIM_E_ARG for NULL pointers, T < 1, n_regions < 1 or
 * frames_per_step < 1; INIM_E_VALUE for a negative or non-finite value.
 */
int inim_interpolate_values(const float* values, int32_t T, int32_t n_regions, int32_t frames_per_step,
                            float* out);

/*
 * Create a map (Sec. 4.1 step 0: regions described by polygons; the
 * background is the complement of the regions in the unit square).
 *   xy          [n_verts*2] unique vertex positions.
 *   ring_off    [n_rings+1] CSR offsets into ring_idx (ring_off[0] = 0).
 *   ring_idx    [ring_off[n_rings]] vertex ids; each ring closes implicitly.
 *   ring_region [n_rings] region id of each ring, 0 <= id < n_regions.
 *   n_regions   1 .. 65534.
 * Membership is even-odd over all rings of a region, so holes are rings of
 * the same region.  Shared boundaries must use the same vertex ids in both
 * regions so that they move together.  Arrays are host memory unless
 * flags has INIM_MAP_DEVICE_PTRS.  Errors: INIM_E_ARG for sizes out of
 * range or a vertex id outside [0, n_verts).
 */
int inim_map_create(const float* xy, int32_t n_verts,
                    const int32_t* ring_off, int32_t n_rings,
                    const int32_t* ring_idx, const int32_t* ring_region,
                    int32_t n_regions, int32_t flags, inim_map** out);

int inim_map_destroy(inim_map* map);

/* Sizes of a map (any pointer may be NULL). */
int inim_map_info(const inim_map* map, int32_t* n_verts, int32_t* n_regions,
                  int32_t* n_rings, int32_t* n_edges);

/*
 * Time-varying cartogram (Sec. 4.1 algorithm per step; Sec. 4.2 modes).
 *   values  [T*n_regions] s_t(v) for t = 0..T-1; host or device.
 *   init_xy [n_verts*2] start vertices or NULL (the map's own); host or device.
 *   out_xy  [T*n_verts*2] vertices after each step; host or device.
 *   stats   [T] host array or NULL.
 * Direct mode runs all T steps as one batch; cumulative mode runs them in
 * order.  Returns the worst per-step status.
 */
int inim_run(inim_map* map, const float* values, int32_t T, const inim_params* params,
             const float* init_xy, float* out_xy, inim_step_stats* stats, void* stream);

/*
 * A time series whose map area follows its global integral (dynamic area,
 * Sec. 4.3, Eq. (Mb)): the background value of every step is computed as by
 * inim_background_values(values, T, n_regions, params->log2_res, a_min,
 * a_max, t0, t1) and each step is solved with it as params.bdv_value.
 * params->mode INIM_DIRECT: one batch of T independent solves;
 * INIM_CUMULATIVE: the steps in order, each from the previous step's
 * vertices (one inim_run_batch call per step).  values are host memory;
 * the other arguments are those of inim_run.  Returns the worst per-step
 * status; the errors of inim_background_values and inim_run_batch.
 */
int inim_run_dynamic(inim_map* map, const float* values, int32_t T, const inim_params* params, double a_min,
                     double a_max, int32_t t0, int32_t t1, const float* init_xy, float* out_xy,
                     inim_step_stats* stats, void* stream);

/*
 * Many independent single-step solves of possibly different maps and
 * resolutions in one batched launch sequence captured in a CUDA graph
 * (params.form must be INIM_FORM_FUSED).  Jobs run together until each one's
 * stop rule fires.
 */
int inim_run_batch(const inim_job* jobs, int32_t n_jobs, void* stream);

/*
 * Many time series at once (Sec. 4.2 direct and cumulative modes).  Direct
 * series run as independent solves of one batch; cumulative series run
 * their steps in order, all series together.  Every batch runs as CUDA
 * graphs of the per-iteration kernels; with inim_set_persistent(1), small
 * FP32 batches (N <= 2048, fewer than 2^23 pixels in total) run instead in
 * one persistent cooperative launch that covers every iteration and, for
 * cumulative series, every time step.  All series need the fused form and
 * one precision.  inim_run is this call with one series.
 */
int inim_run_series(const inim_series* series, int32_t n_series, void* stream);

/* Geographic quality of a cartogram against its original map (Sec. 3.3). */
typedef struct {
    double  tau;          /* topology distortion 1 - |E_c & E_m| / |E_c | E_m| (0 if both empty) */
    double  shape;        /* mean shape distortion over regions with pixels in both rasters */
    double  rel_pos;      /* relative position error R in [0, 1] */
    int64_t adj_map;      /* adjacent region pairs |E_m| */
    int64_t adj_cart;     /* |E_c| */
    int64_t adj_both;     /* |E_c & E_m| */
    int32_t n_present;    /* regions with pixels in both rasters */
    int32_t pad;
} inim_quality_out;

/*
 * Quality measures of Sec. 3.3, comparing the map at xy_map (NULL: the map's
 * own vertices) with the cartogram at xy_cart ([n_verts*2], host or device),
 * both rasterised at N = 2^log2_res:
 *   tau       regions are adjacent when two of their pixels are 4-neighbours;
 *   shape     per region, |P_m sym-diff P_c| / |P_m union P_c| of its pixel
 *             sets, minimised over whole-pixel translations; a region without
 *             pixels in either raster scores 1 and is left out of the mean;
 *   rel_pos   mean over ordered region pairs of the angle between the vectors
 *             joining their barycentres (polygon area centroids) in the two
 *             maps, over pi; NaN when a region's polygon has zero area in
 *             either map (its barycentre is undefined).
 *   shape_per [n_regions] host out per-region shape distortion, or NULL.
 * Works in device memory of its own: two R x R bit adjacency tables and the
 * bounding-box masks of every region.  The shape search visits every
 * translation of a region's two masks, O(sum over regions of
 * (w_m + w_c)(h_m + h_c) h w / 32) word operations.  Errors: INIM_E_ARG for
 * NULL map/xy_cart/out or a resolution out of range; INIM_E_CAPACITY when
 * the translation work does not fit one launch.
 */
int inim_quality(const inim_map* map, const float* xy_map, const float* xy_cart, int32_t log2_res,
                 inim_quality_out* out, double* shape_per, void* stream);

/* Use (1) or skip (0, default) the persistent launch for small batches. */
int inim_set_persistent(int32_t enable);

/*
 * Single-pass scan (default 0): with 1, batches of at least 2^23 pixels per
 * texture size build their integral images (Sec. 3.1) with one kernel per
 * iteration, whose bands take their carries from the earlier bands by
 * look-back, instead of three kernels (band aggregates, carries, bands with
 * carries).  The carries are summed in 64-bit fixed point, so the result does
 * not depend on the order in which bands finish.  Off by default: the three
 * kernels measured faster on the benchmark's large batch.  Drops the cached
 * batches.
 */
int inim_set_single_pass_scan(int32_t enable);

/*
 * Overlapped area kernel (default 1): each fused iteration's area, error and
 * stop-rule kernel (Sec. 3.3, Sec. 4.1 step 7) runs beside the next
 * iteration's raster and scan, and the next move waits for it.  With a stop
 * rule the raster and scan after the stopping iteration still run on the
 * returned vertices (the move after them sees the stop and leaves the
 * vertices alone), so the returned vertices, iteration counts and errors are
 * those of the sequential order (0), and the overlap flag also covers the
 * raster of the returned vertices.  Drops no cached batch (both forms of the
 * graphs are kept per batch).
 */
int inim_set_area_overlap(int32_t enable);

/*
 * Kernel timeline (a profiling aid; no counterpart in the paper).  With
 * enable = 1 every batch built afterwards records, per launch of each kernel
 * of the iteration, when its first block starts working (after waiting for
 * the previous kernel) and when its last block ends, from the GPU's global
 * nanosecond timer; the graphs keep their programmatic launches, so the
 * durations and gaps are those of the real iteration.  Kernels: 0 crossing
 * keys, 1 rows, 2 scan phase 1 (or the single-pass scan), 3 carries, 4 scan
 * phase 3, 5 gather and move, 6 areas and errors.  Each kernel keeps its last
 * 128 launches (slot = launch index mod 128, counted from the last read).
 * inim_timeline drops the cached batches; enable = 0 frees the buffer.
 * inim_timeline_read copies start_ns[k * 128 + i] and end_ns[k * 128 + i]
 * (n >= 8 * 128 entries each, zero where nothing ran) and clears the record;
 * INIM_E_STATE when the timeline is off.
 */
int inim_timeline(int32_t enable);
int inim_timeline_read(uint64_t* start_ns, uint64_t* end_ns, int32_t n);

/*
 * Failure detection of device-side waits (no counterpart in the paper).
 * The grid barrier of the persistent launch polls at most `spins` times
 * (each poll sleeps up to 256 ns); a wait that runs out records
 * INIM_E_TIMEOUT, the kernel's blocks return without waiting further, and the
 * call returns INIM_E_TIMEOUT with the CUDA context still usable.  spins <= 0
 * restores the default of 2^24 polls (a second or two).  Process-wide; takes
 * effect at the next launch.  (The single-pass scan's look-back waits have a
 * fixed cap of 2^22 polls and end the same way.)
 */
int inim_set_wait_cap(int64_t spins);

/*
 * Phase timing of persistent launches: while enabled, block 0 of the
 * persistent kernel adds the time from one grid barrier to the next (its own
 * work plus the wait for the slowest block) to 8 counters, one per phase of
 * an iteration: crossings, rows, density, scan 1, carries, scan 3, gather,
 * areas.  The call copies the counters (ms, n <= 8 entries, may be NULL),
 * resets them and sets the switch.
 */
int inim_persistent_phase_times(int32_t enable, double* ms, int32_t n);

/* ---------------- single steps of the iteration (device memory) -------- */

/*
 * Step 2 of Sec. 4.1: rasterise the map at vertex positions xy.
 *   xy      [n_verts*2] device.
 *   labels  [N*N] device uint16: region id, or n_regions for background.
 *   counts  [n_regions+1] device int32: o(v) in pixels; counts[n_regions]
 *           is the background pixel count.
 *   overlap NULL or host int32: 1 if some pixel lay inside two regions.
 * Rule: vertices snap to X = rint(x*2^(k+8)); pixel (i,j) has centre
 * (256i+128, 256j+128); an edge with Y0 < Y1 counts for the centre iff
 * Y0 <= Yc < Y1 and the centre is on or right of the edge (exact integer
 * test); a pixel is inside a region iff its count over the region's rings is
 * odd; inside several regions -> the smallest id.
 */
int inim_raster(const inim_map* map, const float* xy, int32_t log2_res, uint16_t* labels,
                int32_t* counts, int32_t* overlap, void* stream);

/*
 * Step 4 of Sec. 4.1 on a given texture: the integral images of Sec. 3.1.
 *   density [N*N] device float, d >= 0.
 *   S       [N*N] device: alpha(i,j) = sum_{i'<=i, j'<=j} d   (2-D prefix)
 *   T       [N*N] device: alpha_t(i,j) = top-wedge sum, the pixels
 *           (i',j') with j'<j and i-(j-j') < i' <= i+(j-j')
 *   A       [2N-1] device: A(s) = sum_{i'+j'<=s} d
 *   B       [2N-1] device: B(w+N-1) = sum_{i'-j'<=w} d
 * Element type of S and T: float for INIM_FP32; int64 fixed point with
 * 2^frac_bits units for INIM_FIX64 (d is quantised to llrint(d*2^frac_bits);
 * A, B are then int64 as well); float pairs (hi, lo) for INIM_KAHAN (A, B
 * float pairs).  frac_bits is ignored unless precision is INIM_FIX64 and
 * must keep every sum below 2^62.  The other six InIms follow from these by
 * Eq. (1) (see inim_displacement).
 */
int inim_inims(const float* density, int32_t log2_res, int32_t precision, int32_t frac_bits,
               void* S, void* T, void* A, void* B, void* stream);

/*
 * Steps 5-6 of Sec. 4.1 on a given texture: Eq. (3) displacement
 * t(p;d) - t(p;d0) interpolated bilinearly at n points.
 *   density [N*N] device float; xy [n*2] device; delta [n*2] device out.
 * Samples are pixel centres; bilinear weights use f = x*N - 1/2,
 * i0 = clamp(floor f, 0, N-2), a = clamp(f - i0, 0, 1).
 */
int inim_displacement(const float* density, int32_t log2_res, int32_t precision,
                      const float* xy, int32_t n, float* delta, void* stream);

/*
 * Run n_iters full iterations in place on device vertices (Sec. 4.1 steps
 * 2-6 plus the areas and errors of Sec. 3.3).  values [n_regions] device.
 * stats: NULL or host struct, filled after the last iteration.  The stop
 * rule is NOT applied (exactly n_iters iterations).
 */
int inim_iterate(const inim_map* map, float* xy, const float* values,
                 const inim_params* params, int32_t n_iters, inim_step_stats* stats,
                 void* stream);

/*
 * Signed shoelace area per region (sum over its rings), accumulated in
 * double (Sec. 3.3).  xy [n_verts*2] device; areas [n_regions] device double.
 */
int inim_areas(const inim_map* map, const float* xy, double* areas, void* stream);

/*
 * Allocation-free FP32 integral images (the paper has no counterpart; this is
 * a service of this library).  Same inputs, outputs and meaning as
 * inim_inims with precision INIM_FP32, for callers that cannot allocate
 * device memory: code running under another framework's memory manager that
 * owns the whole device pool, or a latency-critical loop in which cudaMalloc /
 * cudaFree (which can synchronise the device) are not acceptable.
 *   density [N*N], S [N*N], T [N*N], A [2N-1], B [2N-1]: device float,
 *   all provided by the caller.  Work is enqueued on `stream`; the call does
 *   not wait for it.
 * The working memory (band aggregates, carries, job descriptor, block tables)
 * is one fixed array inside the library, about 1.6 MB, held by every GPU that
 * loads the library until the process exits.  Limit: log2_res <= 10
 * (N <= 1024); larger textures return INIM_E_CAPACITY.  Every call reuses the
 * same array, so calls whose kernels overlap on the GPU (e.g. on two
 * unordered streams) race.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current): make that
 * first call before any stream capture.  The address is kept for the life of
 * the process, so a cudaDeviceReset between calls is not supported.  No
 * cudaMalloc, cudaFree or other allocating routine is called.  Errors set the
 * message of inim_last_error() like every other entry point.
 */
int inim_inims_noalloc(const float* density, int32_t log2_res, float* S, float* T,
                       float* A, float* B, void* stream);

/* ---------------- learned warm start (not part of the paper) ------------ */

/*
 * CNN input of a map state: rasterise the map at xy (host or device, like
 * inim_raster), build the density texture of Sec. 4.1 step 3 with values
 * (host or device, [n_regions]) and average log(d / d0) over pool x pool
 * pixel blocks.  out: [(N/pool)^2] float, row-major, host or device.
 */
int inim_density_pooled(const inim_map* map, const float* xy, int32_t log2_res, const float* values,
                        int32_t pool, float* out, void* stream);

typedef struct inim_cnn inim_cnn;   /* encoder-decoder CNN, r^2 -> 64^2 x 2, r = 64, 128 or 256 */

/* Create with He-initialised weights (seeded); 1,163,234 f32 parameters;
 * input resolution 64^2. */
int inim_cnn_create(int32_t seed, inim_cnn** out);
/*
 * The same network for an input of in_res^2 (64, 128 or 256; else
 * INIM_E_ARG): the first convolution (1 -> 32 channels) runs at in_res and its
 * output is 2x2 average-pooled down to 64^2 before the second; the parameter
 * blob is the same.  inim_cnn_input_res returns in_res.
 */
int inim_cnn_create_res(int32_t seed, int32_t in_res, inim_cnn** out);
int inim_cnn_input_res(const inim_cnn* cnn);
int inim_cnn_destroy(inim_cnn* cnn);
long long inim_cnn_num_params(const inim_cnn* cnn);   /* cnn may be NULL */
/* Parameter blob (per layer: weights [cout][3][3][cin], bias [cout]) to / from host or device. */
int inim_cnn_get_params(const inim_cnn* cnn, float* out, long long n);
int inim_cnn_set_params(inim_cnn* cnn, const float* in, long long n);
/*
 * x: [B][r][r] f32 pooled log densities (r = the input resolution), y:
 * [B][64][64][2] f32 predicted displacement x 10 (unit-square units); device
 * memory.
 */
int inim_cnn_forward(inim_cnn* cnn, const float* x, int32_t B, float* y, void* stream);
/* Mean squared error against targets y and its gradient w.r.t. every parameter
 * (grads: host or device [n_params], may be NULL; loss: host, may be NULL). */
int inim_cnn_gradients(inim_cnn* cnn, const float* x, const float* y, int32_t B, float* loss, float* grads,
                       void* stream);
/*
 * One Adam step (beta 0.9 / 0.999) on the mean squared error.  x and y are
 * copied on `stream` (after its earlier work; the caller may reuse them in
 * that stream's order); the step then runs on the network's own stream.  With
 * loss != NULL (host) the call waits for the step and returns its loss; with
 * loss = NULL it returns at once, and inim_cnn_loss_mean later gives the mean
 * loss of the steps since its previous call.  Calls on one network are
 * ordered.
 */
int inim_cnn_train_step(inim_cnn* cnn, const float* x, const float* y, int32_t B, float lr, float* loss,
                        void* stream);
int inim_cnn_loss_mean(inim_cnn* cnn, double* mean);
const char* inim_cnn_last_error(void);

/*
 * Load the network used by inim_params.warm_start (the f32 parameter blob of
 * inim_cnn_get_params; bytes = 4 * inim_cnn_num_params(NULL)).  Direct steps
 * with warm_start = 1 first move every vertex by the predicted field, then
 * iterate as usual.
 */
int inim_warmstart_load(const void* weights, size_t bytes);
/* The same for a network of input resolution in_res (64, 128 or 256): the
 * solve's density texture is pooled by N / in_res (N >= in_res). */
int inim_warmstart_load_res(const void* weights, size_t bytes, int32_t in_res);

/* ---------------- scan tiles and their autotuner ------------------------- */

/*
 * Tile of the integral-image band scan for one (resolution, precision, size
 * class): band_rows rows per band (one block each), cols_per_thread columns
 * per thread, threads per block (cols_per_thread * threads == N).
 * cols_per_thread = 0 with threads = 256 selects the parallel-rows form (a
 * warp computes each row's prefix, one barrier per band; N = 512 or 1024,
 * band_rows = 8 or 16).  large = 1 for resolution groups of a batch holding
 * >= 2^23 pixels in total, 0 below.  band_rows = 0 restores the built-in
 * default.  The tile changes the FP32 summation order (not the FIX64
 * result).  Setting a tile drops the cached batches.  INIM_E_ARG if no
 * compiled kernel has this tile.
 */
int inim_set_scan_tile(int32_t log2_res, int32_t precision, int32_t large, int32_t band_rows,
                       int32_t cols_per_thread, int32_t threads);
int inim_get_scan_tile(int32_t log2_res, int32_t precision, int32_t large, int32_t* band_rows,
                       int32_t* cols_per_thread, int32_t* threads);

/*
 * Autotuner (not part of the paper): builds a batch of these jobs, rasterises
 * their start positions, times every compiled tile (band heights 4..64,
 * every (columns, threads) pair with columns * threads == N, and the
 * parallel-rows form where it is compiled) on it with CUDA
 * events over `reps` runs of the three scan phases, and sets the fastest tile
 * for each resolution group's (resolution, precision, size class).
 */
int inim_autotune_scan(const inim_job* jobs, int32_t n_jobs, int32_t reps);

/* ---------------- profiling ------------------------------------------- */

/*
 * Average device time of every kernel stage of one fused iteration of the
 * batch used most recently by inim_run / inim_run_batch / inim_iterate: each
 * stage is launched `reps` times back to back, captured into one CUDA graph
 * (with programmatic dependent launch, as in the iteration graphs), and one
 * replay is timed between two CUDA events on the library's stream
 * (ms[i] = elapsed / reps).  Stages, in iteration order:
 * crossings, raster_rows, density_table, scan_phase1, scan_carry,
 * scan_phase3, gather_move, areas_errors, scan_fused (names from
 * inim_stage_name); the two raster kernels run as pairs: the crossing kernel
 * is timed alone (its keys overflow the buckets, whose guard skips the
 * stores) and the rows get the pairs' time minus that; the buckets are
 * emptied afterwards.  For batches whose maps have at most 2047 regions the
 * density table is built by scan_phase1 (there is no density_table kernel in
 * the iteration) and ms[2] = 0.  With inim_set_single_pass_scan(1), large
 * batches (at least 2^23 pixels per resolution) scan in one pass: scan_fused
 * holds that kernel and the three scan phases read 0 (otherwise scan_fused
 * reads 0).  The
 * batch's vertices move while it runs; the next run resets them.  ms must
 * hold >= 9 floats; *n_stages receives 9.  INIM_E_STATE if no map batch ran
 * yet.
 */
int inim_profile_stages(int32_t reps, float* ms, int32_t max_stages, int32_t* n_stages);
const char* inim_stage_name(int32_t i);

/* Number of kernel launches issued by this library so far (graph replays count
 * every kernel node they run). */
long long inim_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* INIM_H */
