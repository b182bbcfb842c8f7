// C ABI of the InIm cartogram library: maps, batches of jobs, the fused and
// the plain iteration drivers, the direct / cumulative time loop (Sec. 4.2),
// and the single-step entry points.  See include/inim.h for the contract.
#include <algorithm>
#include <atomic>
#include <climits>
#include <functional>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "scan_impl.cuh"

using namespace inim;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

}  // namespace

int inim::set_last_error(int code, const char* msg) { return fail(code, msg ? msg : ""); }

namespace {

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(INIM_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// device allocations of one call, freed on every return path
struct DevScratch {
    std::vector<void*> p;
    DevScratch() = default;
    DevScratch(const DevScratch&) = delete;
    DevScratch& operator=(const DevScratch&) = delete;
    ~DevScratch() {
        for (void* q : p) cudaFree(q);
    }
    template <class T>
    cudaError_t get(T** out, size_t bytes) {
        void* q = nullptr;
        const cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) p.push_back(q);
        *out = (T*)q;
        return e;
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// map
// ---------------------------------------------------------------------------
struct inim_map {
    int n_verts = 0, n_regions = 0, n_rings = 0, n_edges = 0;
    int2* edges = nullptr;
    int* edge_region = nullptr;
    int* reg_edge_off = nullptr;
    int* reg_ring_off = nullptr;
    int* reg_rings = nullptr;
    int* ring_off = nullptr;
    int* ring_idx = nullptr;
    float* sign0 = nullptr;
    float2* xy0 = nullptr;
    std::vector<float> h_xy0;
    std::vector<int> h_edge_a, h_edge_b;   // for capacity estimates
};

namespace {

// ---------------------------------------------------------------------------
// per-job device buffers
// ---------------------------------------------------------------------------
size_t elem_size(int precision) { return precision == INIM_FP32 ? 4 : 8; }

constexpr int kRowsPerBlock = 8;     // rows of one k_raster_rows block (one warp each)

struct Buffers {
    int n = 0, precision = 0, R = 0, nb = 0, V = 0;
    uint16_t* labels = nullptr;
    int* row_cnt = nullptr;
    int* big_rows = nullptr;
    uint32_t* keys = nullptr;
    int* counts = nullptr;
    float* dens = nullptr;
    float* values = nullptr;
    void* S = nullptr;
    void* T = nullptr;
    void* A = nullptr;
    void* B = nullptr;
    void* rowcum = nullptr;
    void* agg = nullptr;
    void* carry = nullptr;
    double* areas = nullptr;
    float2* xy = nullptr;
    unsigned* flags = nullptr;          // single-pass scan: band flags
    long long* binc = nullptr;          // single-pass scan: band inclusive prefixes (fixed point)

    cudaError_t alloc(int n_, int prec, int R_, int V_, int nb_, bool interleaved) {
        n = n_; precision = prec; R = R_; V = V_; nb = nb_;
        const size_t np = (size_t)n * n, es = elem_size(prec);
        cudaError_t e = cudaSuccess;
        auto A_ = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes < 16 ? 16 : bytes); };
        A_((void**)&labels, np * 2);
        A_((void**)&row_cnt, (size_t)n * 4);
        A_((void**)&big_rows, (size_t)n * 4);
        A_((void**)&keys, (size_t)n * kKeyStride * 4);     // one fixed-stride bucket per row
        A_((void**)&counts, (size_t)(R + 1) * 4);
        A_((void**)&dens, (size_t)(R + 1) * 4);
        A_((void**)&values, (size_t)R * 4);
        // map jobs store interleaved (S, T) pairs in S; texture jobs S and T apart
        A_(&S, (interleaved ? 2 : 1) * np * es);
        A_(&T, interleaved ? 16 : np * es);
        A_(&A, (size_t)(2 * n) * es);
        A_(&B, (size_t)(2 * n) * es);
        A_(&rowcum, (size_t)n * es);
        A_(&agg, (size_t)3 * nb * n * es);
        A_(&carry, (size_t)3 * nb * n * es);
        A_((void**)&areas, (size_t)R * 8);
        A_((void**)&xy, (size_t)V * 8);
        // map jobs may run the single-pass scan (large batches)
        A_((void**)&flags, interleaved ? (size_t)nb * 4 : 16);
        A_((void**)&binc, interleaved ? (size_t)3 * nb * n * 8 : 16);
        if (e == cudaSuccess) e = cudaMemset(row_cnt, 0, (size_t)n * 4);
        if (e == cudaSuccess) e = cudaMemset(flags, 0, interleaved ? (size_t)nb * 4 : 16);
        return e;
    }
    void release() {
        dfree(labels); dfree(row_cnt); dfree(big_rows); dfree(keys); dfree(counts); dfree(dens);
        dfree(values); dfree(S); dfree(T); dfree(A); dfree(B); dfree(rowcum); dfree(agg);
        dfree(carry); dfree(areas); dfree(xy); dfree(flags); dfree(binc);
    }
};

// scan tiles per (precision, resolution): band height, columns per thread,
// threads.  Defaults below; inim_set_scan_tile / inim_autotune_scan override.
// Separate entries for small and large groups (total pixels of the group's
// jobs below / at least 2^23): small batches are latency-bound, large ones
// bandwidth-bound, and they prefer different tiles.
ScanTile g_tiles[3][2][kMaxLog2 + 1] = {};

int size_class(long long group_pixels) { return group_pixels >= (1LL << 23) ? 1 : 0; }

ScanTile default_tile(int log2n) {
    switch (log2n) {
        case 8: return {8, 2, 128};
        case 9: return {8, 4, 128};
        case 10: return {16, 8, 128};
        case 11: return {16, 8, 256};
        default: return {32, 8, 512};
    }
}

ScanTile tile_for(int log2n, int precision, int cls) {
    ScanTile t = g_tiles[precision][cls][log2n];
    if (t.H <= 0) t = default_tile(log2n);
    t.n = 1 << log2n;
    return t;
}

// (columns per thread, threads) pairs with a compiled band-scan kernel
constexpr int kTilePairs[][2] = {{2, 128}, {4, 128}, {2, 256}, {8, 128}, {4, 256}, {8, 256}, {4, 512}, {8, 512},
                                 {16, 64}, {32, 32}, {0, 256}};
constexpr int kTileHeights[] = {4, 8, 16, 32, 64};

bool tile_valid(int log2n, ScanTile t) {
    const int n = 1 << log2n;
    if (t.cpt == 0)                               // parallel-rows form: its instantiations
        return t.nt == 256 && (n == 512 || n == 1024) && (t.H == 8 || t.H == 16);
    bool pair = false;
    for (auto& q : kTilePairs) pair |= (q[0] == t.cpt && q[1] == t.nt);
    bool h = false;
    for (int x : kTileHeights) h |= (x == t.H);
    return pair && h && t.cpt * t.nt == n && t.H * 4 <= n;
}

// ---------------------------------------------------------------------------
// batch: jobs + buffers + block maps (+ a captured CUDA graph)
// ---------------------------------------------------------------------------
struct JobSpec {
    const inim_map* map;
    int log2n;
    int precision;
    bool operator==(const JobSpec& o) const {
        return map == o.map && log2n == o.log2n && precision == o.precision;
    }
};

struct Group {
    int log2n;
    ScanTile tile;
    BlockMap band, carry;     // band.ticket: the single-pass scan's ticket counter
};

// With inim_set_single_pass_scan(1), large groups of map jobs scan in one
// pass (scan_fused.cuh) with the row-serial tiles; by default every group
// uses the three kernels (phase 1, carries, phase 3), which measured faster
// on the 72-solve batch of the time-varying sweep (334 against 484 us per
// iteration with 16-row bands, 305 against 377 us with 32-row bands): the
// single-pass blocks hold their SM slots during the look-back (median 9 us)
// and their phases run slower next to blocks in other phases.
int g_single_pass = 0;

// kernel timeline buffer (inim_timeline); set in the jobs of batches built
// while it is on
unsigned long long* g_tl = nullptr;

int fused_for(const ScanTile& t, int size_cls, bool maps) {
    return (g_single_pass && maps && t.cpt > 0 && size_cls == 1) ? 1 : 0;
}

// Block order of a single-pass scan: band 0 of every job, then band 1 of
// every job, ...  A band's look-back then finds its predecessor (dispatched a
// whole round of jobs earlier) already finished, instead of adding up the
// aggregates of many bands that started at the same time.
std::vector<int2> interleave_bands(const std::vector<int2>& band) {
    std::vector<int2> out;
    out.reserve(band.size());
    int max_b = 0;
    for (const int2& x : band) max_b = std::max(max_b, x.y);
    for (int b = 0; b <= max_b; ++b)
        for (const int2& x : band)
            if (x.y == b) out.push_back(x);
    return out;
}

constexpr int kGraphSizes = 6;     // CUDA graphs of 1, 2, 4, 8, 16, 32 iterations per batch

struct Batch {
    std::vector<JobSpec> spec;
    std::vector<Job> h_jobs;
    std::vector<JobState> h_states;
    std::vector<Buffers> bufs;
    Job* d_jobs = nullptr;
    JobState* d_states = nullptr;
    BlockMap edge_blocks, job_blocks, row_blocks, vert_blocks, region_blocks;
    std::vector<Group> groups;
    int precision = INIM_FP32;
    int max_n = 0;
    bool fuse_table = false;            // the scan builds the density table (no density kernel)
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    // CUDA graphs of 1, 2, 4, ... 32 fused iterations (captured on first use),
    // plain [0] and overlapped [1]: in the overlapped form each iteration's
    // area kernel runs on a side branch, next to the next iteration's raster
    // and scan
    cudaGraphExec_t graphs[2][kGraphSizes] = {};
    cudaStream_t side = nullptr;
    cudaEvent_t ev_moved = nullptr, ev_areas = nullptr;
    std::vector<PlainWork> plain;   // per job (plain form only)
    // persistent form: all resolution groups' band / carry items, barrier words,
    // per-job round tables (time series), their device pointer arrays
    BlockMap all_band, all_carry;
    unsigned* d_bar = nullptr;
    int* d_err = nullptr;
    int round_cap = 0;                      // rounds the round buffers hold
    std::vector<float*> round_vals;         // per job [round_cap][R]
    std::vector<float2*> round_outs;        // per job [round_cap][V]
    std::vector<JobState*> round_stats;     // per job [round_cap]
    int* d_job_rounds = nullptr;
    const float** d_round_vals = nullptr;
    float2** d_round_outs = nullptr;
    JobState** d_round_stats = nullptr;
    JobState* d_round_init = nullptr;
    long long total_px = 0;
    // cumulative rounds enqueued at once: per round, the jobs and states to
    // upload and the final states read back (pinned host memory)
    int pin_rounds = 0;
    Job* pin_jobs = nullptr;
    JobState* pin_states = nullptr;
    JobState* pin_out_states = nullptr;
    // stop-rule polls: two pinned copies of the states, an event each
    JobState* pin_poll = nullptr;
    cudaEvent_t ev_poll[2] = {nullptr, nullptr};
    // learned warm start: pooled inputs, predicted fields, per-job field pointers
    float* ws_in = nullptr;
    float* ws_out = nullptr;
    int ws_res = 0;                      // input resolution ws_in was sized for
    const float** ws_ptrs = nullptr;

    void free_rounds() {
        for (auto& p : round_vals) dfree(p);
        for (auto& p : round_outs) dfree(p);
        for (auto& p : round_stats) dfree(p);
        round_vals.clear(); round_outs.clear(); round_stats.clear();
        dfree(d_job_rounds); dfree(d_round_vals); dfree(d_round_outs); dfree(d_round_stats); dfree(d_round_init);
        round_cap = 0;
    }

    void free_pinned() {
        if (pin_jobs) cudaFreeHost(pin_jobs);
        if (pin_states) cudaFreeHost(pin_states);
        if (pin_out_states) cudaFreeHost(pin_out_states);
        pin_jobs = nullptr; pin_states = nullptr; pin_out_states = nullptr;
        pin_rounds = 0;
    }

    void free_poll() {
        if (pin_poll) cudaFreeHost(pin_poll);
        pin_poll = nullptr;
        for (auto& e : ev_poll)
            if (e) cudaEventDestroy(e);
        ev_poll[0] = ev_poll[1] = nullptr;
    }

    ~Batch() {
        if (stream) cudaStreamSynchronize(stream);     // no copy from the pinned buffers is still queued
        free_pinned();
        free_poll();
        free_rounds();
        dfree(ws_in); dfree(ws_out); dfree(ws_ptrs);
        dfree(d_bar); dfree(d_err); dfree(all_band.d_map); dfree(all_carry.d_map);
        for (auto& row : graphs)
            for (auto& g : row)
                if (g) cudaGraphExecDestroy(g);
        for (auto& b : bufs) b.release();
        for (auto& p : plain) plain_free(p);
        dfree(d_jobs); dfree(d_states);
        BlockMap* maps[] = {&edge_blocks, &job_blocks, &row_blocks, &vert_blocks, &region_blocks};
        for (BlockMap* m : maps) dfree(m->d_map);
        for (auto& g : groups) { dfree(g.band.d_map); dfree(g.carry.d_map); dfree(g.band.ticket); }
        if (ev_moved) cudaEventDestroy(ev_moved);
        if (ev_areas) cudaEventDestroy(ev_areas);
        if (side) cudaStreamDestroy(side);
        if (ev) cudaEventDestroy(ev);
        if (stream) cudaStreamDestroy(stream);
    }
};

cudaError_t make_map(BlockMap& bm, const std::vector<int2>& entries) {
    bm.n_blocks = (int)entries.size();
    if (entries.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(&bm.d_map, entries.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(bm.d_map, entries.data(), entries.size() * sizeof(int2), cudaMemcpyHostToDevice);
    return e;
}

int build_batch(Batch& B, const std::vector<JobSpec>& spec,
                int min_H = 0) {
    B.spec = spec;
    const int nj = (int)spec.size();
    B.precision = spec[0].precision;
    // Small batches are latency-bound chains of short kernels (a cumulative
    // series advances one iteration at a time); they get the highest stream
    // priority so that, next to a large batch on another stream, their blocks
    // are scheduled first and the large batch fills the remaining SMs.
    long long total_px = 0;
    for (auto& sp : spec) total_px += 1LL << (2 * sp.log2n);
    int prio_least = 0, prio_greatest = 0;
    CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    CUDA_TRY(cudaStreamCreateWithPriority(&B.stream, cudaStreamNonBlocking,
                                          size_class(total_px) == 0 ? prio_greatest : prio_least));
    CUDA_TRY(cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming));
    CUDA_TRY(cudaMalloc(&B.d_jobs, nj * sizeof(Job)));
    CUDA_TRY(cudaMalloc(&B.d_states, nj * sizeof(JobState)));
    B.h_jobs.resize(nj);
    B.h_states.assign(nj, JobState{});
    B.bufs.resize(nj);
    long long group_px[kMaxLog2 + 1] = {};
    for (auto& sp : spec) group_px[sp.log2n] += 1LL << (2 * sp.log2n);
    std::vector<int2> eb, jb, rb, vb, gb;
    for (int k = 0; k < nj; ++k) {
        const JobSpec& s = spec[k];
        const inim_map* m = s.map;
        const int n = 1 << s.log2n;
        const ScanTile tile = tile_for(s.log2n, s.precision, size_class(group_px[s.log2n]));
        const int nb = (n + tile.H - 1) / tile.H;
        const int nb_alloc = min_H > 0 ? (n + min_H - 1) / min_H : nb;
        Buffers& b = B.bufs[k];
        CUDA_TRY(b.alloc(n, s.precision, m ? m->n_regions : 1, m ? m->n_verts : 1, nb_alloc, m != nullptr));
        Job J{};
        J.n = n; J.log2n = s.log2n;
        if (m) {
            J.n_verts = m->n_verts; J.n_regions = m->n_regions; J.n_edges = m->n_edges; J.n_rings = m->n_rings;
            J.edges = m->edges; J.edge_region = m->edge_region; J.reg_edge_off = m->reg_edge_off;
            J.reg_ring_off = m->reg_ring_off;
            J.reg_rings = m->reg_rings; J.ring_off = m->ring_off; J.ring_idx = m->ring_idx; J.sign0 = m->sign0;
        }
        J.xy = b.xy; J.values = b.values; J.lam = 1.0f; J.bdv_scale = 1.0f; J.precision = s.precision;
        J.labels = b.labels; J.row_cnt = b.row_cnt; J.big_rows = b.big_rows;
        J.keys = b.keys;
        J.counts = b.counts; J.dens = b.dens;
        J.pdl_early = size_class(total_px) == 0 ? 1 : 0;
        J.S = b.S; J.T = b.T; J.A = b.A; J.B = b.B; J.rowcum = b.rowcum;
        // map jobs: one interleaved (S, T) table (S's buffer holds both halves)
        J.ST = m ? b.S : nullptr;
        J.H = tile.H; J.nb = nb; J.agg = b.agg; J.carry = b.carry;
        J.bflags = b.flags; J.binc = b.binc;
        J.areas = b.areas; J.st = B.d_states + k;
        J.tl = g_tl;
        B.h_jobs[k] = J;
        if (m) {
            for (int q = 0; q < (m->n_edges + kEdgesPerItem - 1) / kEdgesPerItem; ++q) eb.push_back(make_int2(k, q));
            for (int q = 0; q < (m->n_verts + 255) / 256; ++q) vb.push_back(make_int2(k, q));
            const int rpb = 8 >> area_warps_log2(m->n_edges, m->n_regions);   // regions per area block
            for (int q = 0; q < (m->n_regions + rpb - 1) / rpb; ++q) gb.push_back(make_int2(k, q));
        }
        jb.push_back(make_int2(k, 0));
        for (int j = 0; j < n; j += kRowsPerBlock) rb.push_back(make_int2(k, j));
        B.max_n = std::max(B.max_n, n);
    }
    CUDA_TRY(raster_setup(B.max_n));
    CUDA_TRY(make_map(B.edge_blocks, eb));
    CUDA_TRY(make_map(B.job_blocks, jb));
    CUDA_TRY(make_map(B.row_blocks, rb));
    CUDA_TRY(make_map(B.vert_blocks, vb));
    CUDA_TRY(make_map(B.region_blocks, gb));
    // scan groups by resolution (and, for the persistent form, all of them)
    std::vector<int2> all_band, all_carry;
    for (int k = 0; k < nj; ++k) {
        const Job& J = B.h_jobs[k];
        B.total_px += (long long)J.n * J.n;
        for (int b = 0; b < J.nb; ++b) all_band.push_back(make_int2(k, b));
        const int len = carry_qspace(J.n, J.nb, J.H);
        for (int q = 0; q < (len + 255) / 256; ++q) all_carry.push_back(make_int2(k, q));
    }
    CUDA_TRY(make_map(B.all_band, all_band));
    CUDA_TRY(make_map(B.all_carry, all_carry));
    CUDA_TRY(cudaMalloc(&B.d_bar, 2 * sizeof(unsigned)));
    CUDA_TRY(cudaMalloc(&B.d_err, sizeof(int)));
    for (int l = kMinLog2; l <= kMaxLog2; ++l) {
        std::vector<int2> band, carry;
        for (int k = 0; k < nj; ++k) {
            if (spec[k].log2n != l) continue;
            const Job& J = B.h_jobs[k];
            for (int b = 0; b < J.nb; ++b) band.push_back(make_int2(k, b));
            const int len = carry_qspace(J.n, J.nb, J.H);
            const int qpb = carry_q_per_block(J.nb, size_class(group_px[l]));
            for (int q = 0; q < (len + qpb - 1) / qpb; ++q) carry.push_back(make_int2(k, q));
        }
        if (band.empty()) continue;
        bool maps = true;
        for (int k = 0; k < nj; ++k) if (spec[k].log2n == l && !spec[k].map) maps = false;
        Group g;
        g.log2n = l;
        g.tile = tile_for(l, B.precision, size_class(group_px[l]));
        g.tile.fused = fused_for(g.tile, size_class(group_px[l]), maps);
        if (g.tile.fused) band = interleave_bands(band);
        CUDA_TRY(make_map(g.band, band));
        CUDA_TRY(make_map(g.carry, carry));
        CUDA_TRY(cudaMalloc(&g.band.ticket, sizeof(unsigned long long)));
        CUDA_TRY(cudaMemset(g.band.ticket, 0, sizeof(unsigned long long)));
        g.carry.q_per_block = carry_q_per_block(((1 << l) + g.tile.H - 1) / g.tile.H, size_class(group_px[l]));
        B.groups.push_back(g);
    }
    // map jobs with small region tables: the scan's first phase builds the
    // density table (and the iteration state), the density kernel is left out
    B.fuse_table = true;
    for (int k = 0; k < nj; ++k)
        if (!spec[k].map || B.h_jobs[k].n_regions + 1 > kFusedTableMax) B.fuse_table = false;
    for (auto& J : B.h_jobs) J.fuse_table = B.fuse_table ? 1 : 0;
    CUDA_TRY(cudaMemcpy(B.d_jobs, B.h_jobs.data(), nj * sizeof(Job), cudaMemcpyHostToDevice));
    return INIM_OK;
}

// batch cache (same job specs -> same buffers, block maps and graph)
std::mutex g_cache_mu;
std::list<std::unique_ptr<Batch>> g_cache;
constexpr size_t kCacheMax = 6;

Batch* get_batch(const std::vector<JobSpec>& spec, int* status) {
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
        if ((*it)->spec == spec) {
            g_cache.splice(g_cache.begin(), g_cache, it);
            *status = INIM_OK;
            return g_cache.front().get();
        }
    }
    auto b = std::make_unique<Batch>();
    *status = build_batch(*b, spec);
    if (*status != INIM_OK) return nullptr;
    g_cache.push_front(std::move(b));
    while (g_cache.size() > kCacheMax) g_cache.pop_back();
    return g_cache.front().get();
}

void purge_all() {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache.clear();
}

// retile one resolution group of a batch in place (buffers sized for min_H)
long long group_pixels(const Batch& B, int log2n) {
    long long px = 0;
    for (auto& sp : B.spec) if (sp.log2n == log2n) px += 1LL << (2 * sp.log2n);
    return px;
}

int retile_group(Batch& B, Group& g, ScanTile t) {
    std::vector<int2> band, carry;
    bool maps = true;
    for (int k = 0; k < (int)B.spec.size(); ++k) {
        if (B.spec[k].log2n != g.log2n) continue;
        maps = maps && B.spec[k].map != nullptr;
        Job& J = B.h_jobs[k];
        J.H = t.H;
        J.nb = (J.n + t.H - 1) / t.H;
        // a new grid: the single-pass scan's flags start over (with its tickets)
        CUDA_TRY(cudaMemsetAsync(B.bufs[k].flags, 0, B.spec[k].map ? (size_t)B.bufs[k].nb * 4 : 16, B.stream));
        for (int b = 0; b < J.nb; ++b) band.push_back(make_int2(k, b));
        const int len = carry_qspace(J.n, J.nb, J.H);
        const int qpb = carry_q_per_block(J.nb, size_class(group_pixels(B, g.log2n)));
        for (int q = 0; q < (len + qpb - 1) / qpb; ++q) carry.push_back(make_int2(k, q));
    }
    const int fused = fused_for(t, size_class(group_pixels(B, g.log2n)), maps);
    if (fused) band = interleave_bands(band);
    dfree(g.band.d_map);
    dfree(g.carry.d_map);
    unsigned long long* ticket = g.band.ticket;
    g.band = BlockMap{};
    g.carry = BlockMap{};
    g.band.ticket = ticket;
    CUDA_TRY(make_map(g.band, band));
    CUDA_TRY(make_map(g.carry, carry));
    CUDA_TRY(cudaMemsetAsync(g.band.ticket, 0, sizeof(unsigned long long), B.stream));
    g.carry.q_per_block = carry_q_per_block((1 << g.log2n) / t.H, size_class(group_pixels(B, g.log2n)));
    g.tile = t;
    g.tile.fused = fused;
    CUDA_TRY(cudaMemcpyAsync(B.d_jobs, B.h_jobs.data(), B.h_jobs.size() * sizeof(Job), cudaMemcpyHostToDevice,
                             B.stream));
    return INIM_OK;
}

void purge_map(const inim_map* m) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        bool uses = false;
        for (auto& s : (*it)->spec) uses |= (s.map == m);
        if (uses) it = g_cache.erase(it);
        else ++it;
    }
}

// ---------------------------------------------------------------------------
// iteration drivers
// ---------------------------------------------------------------------------
// the first iteration of a run needs the row histogram of the start positions
cudaError_t enqueue_prologue(Batch& B, cudaStream_t s) {
    return launch_raster_prologue(B.d_jobs, (int)B.spec.size(), B.edge_blocks, s);
}

// One fused iteration.  overlap: the area kernel goes to the side stream once
// the vertices have moved, and the next iteration's move waits for it (the
// raster of the next iteration only reads the vertices, the move rewrites
// them); `first` marks the first iteration of a captured sequence (the
// previous area kernel finished with the previous graph launch).  With a stop
// rule the next iteration's raster and scan may start before the area kernel
// has stopped the job: they work on the vertices the run returns and change
// nothing the run reports but the raster flags (the overlap flag then covers
// the returned vertices too); the move, which waits for the area kernel, sees
// the stop and leaves the vertices alone, and every later kernel of the job
// returns at once.
cudaError_t enqueue_fused_iteration(Batch& B, cudaStream_t s, bool overlap = false, bool first = true) {
    cudaError_t e = launch_raster_main(B.d_jobs, B.edge_blocks, B.row_blocks, B.max_n, s);
    if (e == cudaSuccess && !B.fuse_table) e = launch_density_table(B.d_jobs, (int)B.spec.size(), s);
    for (auto& g : B.groups) {
        if (e != cudaSuccess) break;
        if (B.precision == INIM_FIX64) e = launch_scan_fix64(B.d_jobs, g.band, g.carry, g.tile, nullptr, s);
        else if (B.precision == INIM_KAHAN) e = launch_scan_kahan(B.d_jobs, g.band, g.carry, g.tile, nullptr, s);
        else e = launch_scan_fp32(B.d_jobs, g.band, g.carry, g.tile, nullptr, s);
    }
    if (overlap && !first && e == cudaSuccess) e = cudaStreamWaitEvent(s, B.ev_areas, 0);
    if (e == cudaSuccess) e = launch_gather(B.d_jobs, B.vert_blocks, B.precision, s);
    if (!overlap) {
        if (e == cudaSuccess) e = launch_areas_errors(B.d_jobs, B.region_blocks, 1, s);
        return e;
    }
    if (e == cudaSuccess) e = cudaEventRecord(B.ev_moved, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B.side, B.ev_moved, 0);
    if (e == cudaSuccess) e = launch_areas_errors(B.d_jobs, B.region_blocks, 1, B.side);
    if (e == cudaSuccess) e = cudaEventRecord(B.ev_areas, B.side);
    return e;
}

constexpr int kPollIters = 8;   // iterations between host polls of the stop rule

// the overlapped graphs (inim_set_area_overlap; see enqueue_fused_iteration)
std::atomic<int> g_area_overlap{1};

std::atomic<long long> g_launches{0};

}  // namespace

bool inim::pdl_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("INIM_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

namespace {

int kernels_per_fused_iteration(const Batch& B) {
    int k = 1 + (B.edge_blocks.n_blocks ? 1 : 0);          // crossing keys, rows
    k += B.fuse_table ? 0 : 1;                               // density table (else built by the scan)
    for (auto& g : B.groups) k += g.tile.fused ? 1 : 3;      // single-pass scan, or phases 1-3
    k += B.vert_blocks.n_blocks ? 1 : 0;                     // gather / move
    k += B.region_blocks.n_blocks ? 1 : 0;                   // areas + errors + stop rule
    return k;
}
constexpr int kKernelsPerPlainIteration = 15;

cudaError_t capture_iterations(Batch& B, int iters, cudaGraphExec_t* out, bool overlap) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < iters && e == cudaSuccess; ++k) e = enqueue_fused_iteration(B, B.stream, overlap, k == 0);
    if (overlap && e == cudaSuccess) e = cudaStreamWaitEvent(B.stream, B.ev_areas, 0);     // join the side branch
    const cudaError_t e2 = cudaStreamEndCapture(B.stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) *out = nullptr;
    return e;
}

int ensure_graph(Batch& B, bool overlap = false) {
    if (overlap && !B.side) {
        int prio = 0;
        CUDA_TRY(cudaStreamGetPriority(B.stream, &prio));
        CUDA_TRY(cudaStreamCreateWithPriority(&B.side, cudaStreamNonBlocking, prio));
        CUDA_TRY(cudaEventCreateWithFlags(&B.ev_moved, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&B.ev_areas, cudaEventDisableTiming));
    }
    for (int q = 0; q < kGraphSizes; ++q) {
        if (B.graphs[overlap][q]) continue;
        const cudaError_t e = capture_iterations(B, 1 << q, &B.graphs[overlap][q], overlap);
        if (e != cudaSuccess) return fail(INIM_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    return INIM_OK;
}

// launch the graphs for `iters` more iterations, largest first (the binary
// digits of iters: 50 = 32 + 16 + 2, three graph launches)
cudaError_t launch_iterations(Batch& B, int iters, bool overlap = false) {
    const int per = kernels_per_fused_iteration(B);
    for (int q = kGraphSizes - 1; q >= 0 && iters > 0; --q) {
        while (iters >= (1 << q)) {
            cudaError_t e = cudaGraphLaunch(B.graphs[overlap][q], B.stream);
            if (e != cudaSuccess) return e;
            g_launches += (long long)per << q;
            iters -= 1 << q;
        }
    }
    return cudaSuccess;
}

JobState initial_state(const inim_params& p, int stop_on_rule, int max_iters) {
    JobState st{};
    st.active = 1;
    st.iters = 0;
    st.max_iters = max_iters;
    st.stall_window = p.stall_window;
    st.xi_stop = p.xi_stop;
    st.eps_stop = p.eps_stop;
    st.best_xi = 1e300;
    st.since = 0;
    st.stop_on_rule = stop_on_rule;
    return st;
}

// persistent form: small FP32 batches of textures up to 2048^2
int g_persistent = 0;                         // off by default: see inim_set_persistent
int g_phase_profile = 0;                      // record per-phase time of persistent runs
unsigned long long* g_phase_ns = nullptr;     // device [8]

bool persistent_ok(const Batch& B) {
    return g_persistent && B.precision == INIM_FP32 && B.max_n <= 2048 && B.total_px < (1LL << 23) &&
           B.spec[0].map != nullptr;
}

int ensure_rounds(Batch& B, int rounds) {
    if (B.round_cap >= rounds && (int)B.round_vals.size() == (int)B.spec.size()) return INIM_OK;
    B.free_rounds();
    const int nj = (int)B.spec.size();
    B.round_vals.assign(nj, nullptr);
    B.round_outs.assign(nj, nullptr);
    B.round_stats.assign(nj, nullptr);
    for (int k = 0; k < nj; ++k) {
        const Job& J = B.h_jobs[k];
        CUDA_TRY(cudaMalloc(&B.round_vals[k], (size_t)rounds * J.n_regions * sizeof(float)));
        CUDA_TRY(cudaMalloc(&B.round_outs[k], (size_t)rounds * J.n_verts * sizeof(float2)));
        CUDA_TRY(cudaMalloc(&B.round_stats[k], (size_t)rounds * sizeof(JobState)));
    }
    CUDA_TRY(cudaMalloc(&B.d_job_rounds, nj * sizeof(int)));
    CUDA_TRY(cudaMalloc(&B.d_round_vals, nj * sizeof(float*)));
    CUDA_TRY(cudaMalloc(&B.d_round_outs, nj * sizeof(float2*)));
    CUDA_TRY(cudaMalloc(&B.d_round_stats, nj * sizeof(JobState*)));
    CUDA_TRY(cudaMalloc(&B.d_round_init, nj * sizeof(JobState)));
    CUDA_TRY(cudaMemcpy(B.d_round_vals, B.round_vals.data(), nj * sizeof(float*), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(B.d_round_outs, B.round_outs.data(), nj * sizeof(float2*), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(B.d_round_stats, B.round_stats.data(), nj * sizeof(JobState*), cudaMemcpyHostToDevice));
    B.round_cap = rounds;
    return INIM_OK;
}

// One cooperative launch for every iteration (and every time step when
// rounds > 1) of the batch.  Values of round 0 must be in the jobs' value
// buffers, later rounds in round_vals; states (round 0) must be uploaded;
// h_states gets the final state of each job.
int run_persistent(Batch& B, int iters, int rounds, const std::vector<int>& job_rounds) {
    const int nj = (int)B.spec.size();
    int st = ensure_rounds(B, rounds);
    if (st != INIM_OK) return st;
    CUDA_TRY(enqueue_prologue(B, B.stream));              // empty buckets, restarted parity counters
    g_launches += 1;
    CUDA_TRY(cudaMemcpyAsync(B.d_job_rounds, job_rounds.data(), nj * sizeof(int), cudaMemcpyHostToDevice, B.stream));
    CUDA_TRY(cudaMemcpyAsync(B.d_round_init, B.h_states.data(), nj * sizeof(JobState), cudaMemcpyHostToDevice,
                             B.stream));
    CUDA_TRY(launch_persistent(B.d_jobs, nj, B.edge_blocks, B.row_blocks, B.all_band, B.all_carry, B.vert_blocks,
                               B.region_blocks, iters, rounds, B.d_job_rounds, B.d_round_vals,
                               reinterpret_cast<float2* const*>(B.d_round_outs), B.d_round_init,
                               B.d_round_stats, B.d_bar, B.d_err, B.max_n, 0,
                               g_phase_profile ? g_phase_ns : nullptr, B.stream));
    g_launches += 1;
    int err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, B.d_err, sizeof(int), cudaMemcpyDeviceToHost, B.stream));
    CUDA_TRY(cudaMemcpyAsync(B.h_states.data(), B.d_states, nj * sizeof(JobState), cudaMemcpyDeviceToHost, B.stream));
    CUDA_TRY(cudaStreamSynchronize(B.stream));
    if (err) return fail(err, "persistent kernel: a grid barrier wait hit its cap");
    return INIM_OK;
}

// enqueue a fixed-iteration run of the batch (graph replays) without waiting
int enqueue_fused_async(Batch& B, int max_iters) {
    const bool ov = g_area_overlap.load() != 0;
    int st = ensure_graph(B, ov);
    if (st != INIM_OK) return st;
    CUDA_TRY(enqueue_prologue(B, B.stream));
    g_launches += 1;                                       // bucket reset
    CUDA_TRY(launch_iterations(B, max_iters, ov));
    return INIM_OK;
}

// pinned per-round staging for `rounds` rounds of the batch's jobs
int ensure_pinned_rounds(Batch& B, int rounds) {
    if (B.pin_rounds >= rounds) return INIM_OK;
    CUDA_TRY(cudaStreamSynchronize(B.stream));          // the old buffers may still be read by queued copies
    B.free_pinned();
    const size_t nj = B.spec.size();
    CUDA_TRY(cudaMallocHost(&B.pin_jobs, (size_t)rounds * nj * sizeof(Job)));
    CUDA_TRY(cudaMallocHost(&B.pin_states, (size_t)rounds * nj * sizeof(JobState)));
    CUDA_TRY(cudaMallocHost(&B.pin_out_states, (size_t)rounds * nj * sizeof(JobState)));
    B.pin_rounds = rounds;
    return INIM_OK;
}

bool needs_poll(const inim_params& p) {
    return p.xi_stop > 0.0f || p.eps_stop > 0.0f || p.stall_window > 0;
}

// run the fused form until every job stopped; states must be uploaded
int run_fused(Batch& B, int max_iters, bool poll) {
    const int nj = (int)B.spec.size();
    if (persistent_ok(B)) return run_persistent(B, max_iters, 1, std::vector<int>(nj, 1));
    const bool ov = g_area_overlap.load() != 0;
    int st = ensure_graph(B, ov);
    if (st != INIM_OK) return st;
    CUDA_TRY(enqueue_prologue(B, B.stream));
    g_launches += 1;                                       // bucket reset
    if (!poll) {
        CUDA_TRY(launch_iterations(B, max_iters, ov));
    } else {
        // stop rule: graphs of kPollIters iterations; the states after each
        // are copied to pinned memory behind an event, and the next graph is
        // queued before the host waits for that event, so the GPU does not
        // idle during a poll.  Graphs queued past the stop find every job
        // inactive: their kernels return at once and change nothing.
        if (!B.pin_poll) {
            CUDA_TRY(cudaMallocHost(&B.pin_poll, 2 * (size_t)nj * sizeof(JobState)));
            for (auto& e : B.ev_poll) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        int done = 0, slot = 0, pending = -1;
        while (done < max_iters) {
            const int step = std::min(kPollIters, max_iters - done);
            CUDA_TRY(launch_iterations(B, step, ov));
            done += step;
            if (pending >= 0) {                            // the previous graph's states
                CUDA_TRY(cudaEventSynchronize(B.ev_poll[pending]));
                bool any = false;
                for (int k = 0; k < nj; ++k) any |= (B.pin_poll[(size_t)pending * nj + k].active != 0);
                if (!any) break;
            }
            if (done < max_iters) {
                CUDA_TRY(cudaMemcpyAsync(B.pin_poll + (size_t)slot * nj, B.d_states, nj * sizeof(JobState),
                                         cudaMemcpyDeviceToHost, B.stream));
                CUDA_TRY(cudaEventRecord(B.ev_poll[slot], B.stream));
                pending = slot;
                slot ^= 1;
            }
        }
    }
    CUDA_TRY(cudaMemcpyAsync(B.h_states.data(), B.d_states, nj * sizeof(JobState), cudaMemcpyDeviceToHost, B.stream));
    CUDA_TRY(cudaStreamSynchronize(B.stream));
    return INIM_OK;
}

// the plain form: one job at a time, host stop test after every iteration
int run_plain(Batch& B, int max_iters) {
    const int nj = (int)B.spec.size();
    if ((int)B.plain.size() != nj) {
        B.plain.resize(nj);
        for (int k = 0; k < nj; ++k) CUDA_TRY(plain_alloc(B.plain[k], B.h_jobs[k].n));
    }
    if (nj != 1) return fail(INIM_E_ARG, "the plain form runs one job at a time");
    for (int k = 0; k < nj; ++k) {
        const Job* dj = B.d_jobs + k;
        for (int it = 0; it < max_iters; ++it) {
            CUDA_TRY(launch_raster_prologue(B.d_jobs, (int)B.spec.size(), B.edge_blocks, B.stream));
            CUDA_TRY(launch_raster_main(B.d_jobs, B.edge_blocks, B.row_blocks, B.max_n, B.stream));
            CUDA_TRY(launch_density_table(dj, 1, B.stream));
            CUDA_TRY(plain_iteration(dj, B.h_jobs[k], B.plain[k], B.stream));
            CUDA_TRY(launch_areas_errors(B.d_jobs, B.region_blocks, 1, B.stream));
            g_launches += kKernelsPerPlainIteration;
            CUDA_TRY(cudaMemcpyAsync(&B.h_states[k], B.d_states + k, sizeof(JobState), cudaMemcpyDeviceToHost, B.stream));
            CUDA_TRY(cudaStreamSynchronize(B.stream));
            if (!B.h_states[k].active) break;
        }
    }
    return INIM_OK;
}

int check_params(const inim_params* p) {
    if (!p) return fail(INIM_E_ARG, "params is NULL");
    if (p->log2_res < kMinLog2 || p->log2_res > kMaxLog2) return fail(INIM_E_ARG, "log2_res must be in [8, 12]");
    if (!(p->shape >= 0.0f && p->shape < 1.0f)) return fail(INIM_E_ARG, "shape must be in [0, 1)");
    if (!(p->bdv_scale > 0.0f) || !std::isfinite(p->bdv_scale)) return fail(INIM_E_ARG, "bdv_scale must be > 0");
    if (!(p->bdv_value >= 0.0f) || !std::isfinite(p->bdv_value)) return fail(INIM_E_ARG, "bdv_value must be finite and >= 0");
    if (p->max_iters < 1) return fail(INIM_E_ARG, "max_iters must be >= 1");
    if (p->precision < INIM_FP32 || p->precision > INIM_KAHAN) return fail(INIM_E_ARG, "bad precision");
    if (p->form != INIM_FORM_FUSED && p->form != INIM_FORM_PLAIN) return fail(INIM_E_ARG, "bad form");
    if (p->mode != INIM_DIRECT && p->mode != INIM_CUMULATIVE) return fail(INIM_E_ARG, "bad mode");
    if (p->warm_start && !warmstart_loaded()) return fail(INIM_E_STATE, "no warm-start network loaded");
    if (p->warm_start && p->mode != INIM_DIRECT) return fail(INIM_E_ARG, "the warm start applies to direct steps");
    return INIM_OK;
}

int check_values(const float* v, size_t n) {
    for (size_t k = 0; k < n; ++k)
        if (!(v[k] >= 0.0f) || !std::isfinite(v[k])) return fail(INIM_E_VALUE, "region values must be finite and >= 0");
    return INIM_OK;
}

std::vector<float> to_host(const float* p, size_t n) {
    std::vector<float> h(n);
    if (is_device_ptr(p)) cudaMemcpy(h.data(), p, n * sizeof(float), cudaMemcpyDeviceToHost);
    else std::memcpy(h.data(), p, n * sizeof(float));
    return h;
}

int fill_stats(const JobState& s, inim_step_stats* out) {
    int status = INIM_OK;
    if (s.error) status = s.error;
    else if (s.foldover || s.overlap) status = INIM_W_FOLDOVER;
    else if (s.stop_on_rule && s.xi_stop > 0.0f && s.iters >= s.max_iters && !(s.xi < s.xi_stop))
        status = INIM_W_NOT_CONVERGED;
    if (out) {
        out->iters = s.iters;
        out->eps = (float)s.eps;
        out->xi = (float)s.xi;
        out->foldover = s.foldover;
        out->overlap = s.overlap;
        out->status = status;
    }
    return status;
}

int worst(int a, int b) {
    if (a < 0 || b < 0) return std::min(a, b);
    return std::max(a, b);
}

// Learned warm start of the jobs flagged in warm[]: rasterise their start
// positions, pool log(d/d0) to 64^2, predict the displacement field with the
// loaded network and move every vertex by it (bilinear).  States and values
// must be uploaded.
int apply_warm_start(Batch& B, const std::vector<char>& warm) {
    const int nj = (int)B.spec.size();
    std::vector<int> idx;
    for (int k = 0; k < nj; ++k) if (warm[k]) idx.push_back(k);
    if (idx.empty()) return INIM_OK;
    const size_t cell = (size_t)kFieldRes * kFieldRes;
    const int in_res = warmstart_input_res();          // the network's input: N / in_res pooling
    const size_t in_cell = (size_t)in_res * in_res;
    if (!B.ws_in || B.ws_res != in_res) {
        dfree(B.ws_in); dfree(B.ws_out); dfree(B.ws_ptrs);
        CUDA_TRY(cudaMalloc(&B.ws_in, nj * in_cell * sizeof(float)));
        CUDA_TRY(cudaMalloc(&B.ws_out, nj * cell * 2 * sizeof(float)));
        CUDA_TRY(cudaMalloc(&B.ws_ptrs, nj * sizeof(float*)));
        B.ws_res = in_res;
    }
    CUDA_TRY(enqueue_prologue(B, B.stream));
    CUDA_TRY(launch_raster_main(B.d_jobs, B.edge_blocks, B.row_blocks, B.max_n, B.stream));
    CUDA_TRY(launch_density_table(B.d_jobs, nj, B.stream));
    for (int q = 0; q < (int)idx.size(); ++q) {
        const Job& J = B.h_jobs[idx[q]];
        if (J.n < in_res || J.n % in_res) return fail(INIM_E_ARG, "warm start needs N >= the network's input resolution");
        CUDA_TRY(launch_density_pooled(B.d_jobs + idx[q], J.n, J.n / in_res, B.ws_in + q * in_cell, B.stream));
    }
    const int st = warmstart_predict(B.ws_in, (int)idx.size(), B.ws_out, B.stream);
    if (st != INIM_OK) return fail(st, "warm-start prediction failed");
    std::vector<const float*> ptrs(nj, nullptr);
    for (int q = 0; q < (int)idx.size(); ++q) ptrs[idx[q]] = B.ws_out + q * cell * 2;
    CUDA_TRY(cudaMemcpyAsync(B.ws_ptrs, ptrs.data(), nj * sizeof(float*), cudaMemcpyHostToDevice, B.stream));
    CUDA_TRY(launch_apply_field(B.d_jobs, B.vert_blocks, B.ws_ptrs, kFieldRes, 1.0f / kFieldScale, B.stream));
    CUDA_TRY(cudaStreamSynchronize(B.stream));
    return INIM_OK;
}

// Many time series at once (the fused form).  Direct series become T
// independent jobs of one batch; cumulative series become one job each with T
// rounds, run in one persistent launch when the batch is small enough, else
// round by round.
int run_series_impl(const inim_series* S, int n) {
    int result = INIM_OK;
    struct Ref { int series, t; };
    std::vector<JobSpec> dspec, cspec;
    std::vector<Ref> dref, cref;
    for (int i = 0; i < n; ++i) {
        const inim_series& x = S[i];
        const JobSpec sp{x.map, x.params.log2_res, x.params.precision};
        if (x.params.mode == INIM_DIRECT) {
            for (int t = 0; t < x.T; ++t) {
                dspec.push_back(sp); dref.push_back({i, t});
            }
        } else {
            cspec.push_back(sp); cref.push_back({i, 0});
        }
    }
    int st = INIM_OK;
    auto setup_job = [&](Batch& B, int k, const inim_series& x, int t, bool reset_xy) -> int {
        Job& J = B.h_jobs[k];
        J.lam = 1.0f - x.params.shape;
        J.bdv_scale = x.params.bdv_scale;
        J.bdv_value = x.params.bdv_value;
        const int R = x.map->n_regions, V = x.map->n_verts;
        CUDA_TRY(cudaMemcpyAsync(B.bufs[k].values, x.values + (size_t)t * R, (size_t)R * 4, cudaMemcpyDefault, B.stream));
        if (reset_xy)
            CUDA_TRY(cudaMemcpyAsync(B.bufs[k].xy, x.init_xy ? x.init_xy : (const float*)x.map->xy0, (size_t)V * 8,
                                     cudaMemcpyDefault, B.stream));
        B.h_states[k] = initial_state(x.params, 1, x.params.max_iters);
        return INIM_OK;
    };
    // The direct batch (bandwidth-bound) and the cumulative chain (latency-
    // bound) are independent: when the direct batch needs no host polling it
    // is enqueued on its own stream and runs while the cumulative rounds
    // proceed on theirs.
    Batch* D = nullptr;
    bool d_async = false;
    if (!dspec.empty()) {
        D = get_batch(dspec, &st);
        if (!D) return st;
        int max_it = 1;
        bool poll = false;
        for (int k = 0; k < (int)dspec.size(); ++k) {
            const inim_series& x = S[dref[k].series];
            st = setup_job(*D, k, x, dref[k].t, true);
            if (st != INIM_OK) return st;
            max_it = std::max(max_it, x.params.max_iters);
            poll |= needs_poll(x.params);
        }
        CUDA_TRY(cudaMemcpyAsync(D->d_jobs, D->h_jobs.data(), dspec.size() * sizeof(Job), cudaMemcpyHostToDevice, D->stream));
        CUDA_TRY(cudaMemcpyAsync(D->d_states, D->h_states.data(), dspec.size() * sizeof(JobState),
                                 cudaMemcpyHostToDevice, D->stream));
        std::vector<char> warm(dspec.size(), 0);
        bool any_warm = false;
        for (int k = 0; k < (int)dspec.size(); ++k) any_warm |= (warm[k] = S[dref[k].series].params.warm_start != 0);
        if (any_warm) {
            st = apply_warm_start(*D, warm);
            if (st != INIM_OK) return st;
        }
        d_async = !poll && !cspec.empty() && !persistent_ok(*D);
        if (d_async) st = enqueue_fused_async(*D, max_it);
        else st = run_fused(*D, max_it, poll);
        if (st != INIM_OK) return st;
    }
    auto collect_direct = [&]() -> int {
        if (!D) return INIM_OK;
        if (d_async) {
            CUDA_TRY(cudaMemcpyAsync(D->h_states.data(), D->d_states, dspec.size() * sizeof(JobState),
                                     cudaMemcpyDeviceToHost, D->stream));
        }
        for (int k = 0; k < (int)dspec.size(); ++k) {
            const inim_series& x = S[dref[k].series];
            const int V = x.map->n_verts, t = dref[k].t;
            CUDA_TRY(cudaMemcpyAsync(x.out_xy + (size_t)t * V * 2, D->bufs[k].xy, (size_t)V * 8, cudaMemcpyDefault,
                                     D->stream));
        }
        CUDA_TRY(cudaStreamSynchronize(D->stream));
        for (int k = 0; k < (int)dspec.size(); ++k) {
            const inim_series& x = S[dref[k].series];
            result = worst(result, fill_stats(D->h_states[k], x.stats ? x.stats + dref[k].t : nullptr));
        }
        return INIM_OK;
    };
    if (!d_async) {
        st = collect_direct();
        if (st != INIM_OK) return st;
    }
    if (!cspec.empty()) {
        Batch* B = get_batch(cspec, &st);
        if (!B) return st;
        const int nc = (int)cspec.size();
        int rounds = 1, max_it = 1;
        bool poll = false;
        std::vector<int> job_rounds(nc);
        for (int k = 0; k < nc; ++k) {
            const inim_series& x = S[cref[k].series];
            job_rounds[k] = x.T;
            rounds = std::max(rounds, x.T);
            max_it = std::max(max_it, x.params.max_iters);
            poll |= needs_poll(x.params);
            st = setup_job(*B, k, x, 0, true);
            if (st != INIM_OK) return st;
        }
        if (persistent_ok(*B)) {
            st = ensure_rounds(*B, rounds);
            if (st != INIM_OK) return st;
            for (int k = 0; k < nc; ++k) {
                const inim_series& x = S[cref[k].series];
                CUDA_TRY(cudaMemcpyAsync(B->round_vals[k], x.values, (size_t)x.T * x.map->n_regions * 4,
                                         cudaMemcpyDefault, B->stream));
            }
            CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), nc * sizeof(Job), cudaMemcpyHostToDevice, B->stream));
            CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), nc * sizeof(JobState), cudaMemcpyHostToDevice,
                                     B->stream));
            st = run_persistent(*B, max_it, rounds, job_rounds);
            if (st != INIM_OK) return st;
            std::vector<JobState> rs(rounds);
            for (int k = 0; k < nc; ++k) {
                const inim_series& x = S[cref[k].series];
                const int V = x.map->n_verts;
                CUDA_TRY(cudaMemcpyAsync(x.out_xy, B->round_outs[k], (size_t)x.T * V * 8, cudaMemcpyDefault, B->stream));
                CUDA_TRY(cudaMemcpyAsync(rs.data(), B->round_stats[k], (size_t)x.T * sizeof(JobState),
                                         cudaMemcpyDeviceToHost, B->stream));
                CUDA_TRY(cudaStreamSynchronize(B->stream));
                for (int t = 0; t < x.T; ++t) result = worst(result, fill_stats(rs[t], x.stats ? x.stats + t : nullptr));
            }
        } else if (!poll) {
            // no stop rule: every round is enqueued at once (its jobs and
            // states staged through pinned memory, its final states copied
            // back to pinned memory), with one host wait at the end
            st = ensure_pinned_rounds(*B, rounds);
            if (st != INIM_OK) return st;
            for (int t = 0; t < rounds; ++t) {
                for (int k = 0; k < nc; ++k) {
                    const inim_series& x = S[cref[k].series];
                    if (t > 0 && t < x.T) {
                        st = setup_job(*B, k, x, t, false);
                        if (st != INIM_OK) return st;
                    } else if (t >= x.T) {
                        B->h_states[k].active = 0;
                    }
                }
                Job* pj = B->pin_jobs + (size_t)t * nc;
                JobState* ps = B->pin_states + (size_t)t * nc;
                std::copy(B->h_jobs.begin(), B->h_jobs.end(), pj);
                std::copy(B->h_states.begin(), B->h_states.end(), ps);
                CUDA_TRY(cudaMemcpyAsync(B->d_jobs, pj, nc * sizeof(Job), cudaMemcpyHostToDevice, B->stream));
                CUDA_TRY(cudaMemcpyAsync(B->d_states, ps, nc * sizeof(JobState), cudaMemcpyHostToDevice, B->stream));
                st = enqueue_fused_async(*B, max_it);
                if (st != INIM_OK) return st;
                CUDA_TRY(cudaMemcpyAsync(B->pin_out_states + (size_t)t * nc, B->d_states, nc * sizeof(JobState),
                                         cudaMemcpyDeviceToHost, B->stream));
                for (int k = 0; k < nc; ++k) {
                    const inim_series& x = S[cref[k].series];
                    if (t >= x.T) continue;
                    const int V = x.map->n_verts;
                    CUDA_TRY(cudaMemcpyAsync(x.out_xy + (size_t)t * V * 2, B->bufs[k].xy, (size_t)V * 8,
                                             cudaMemcpyDefault, B->stream));
                }
            }
            CUDA_TRY(cudaStreamSynchronize(B->stream));
            for (int t = 0; t < rounds; ++t)
                for (int k = 0; k < nc; ++k) {
                    const inim_series& x = S[cref[k].series];
                    if (t >= x.T) continue;
                    const JobState& rs = B->pin_out_states[(size_t)t * nc + k];
                    result = worst(result, fill_stats(rs, x.stats ? x.stats + t : nullptr));
                }
            std::copy(B->pin_out_states + (size_t)(rounds - 1) * nc, B->pin_out_states + (size_t)rounds * nc,
                      B->h_states.begin());
        } else {
            for (int t = 0; t < rounds; ++t) {
                for (int k = 0; k < nc; ++k) {
                    const inim_series& x = S[cref[k].series];
                    if (t > 0 && t < x.T) {
                        st = setup_job(*B, k, x, t, false);
                        if (st != INIM_OK) return st;
                    } else if (t >= x.T) {
                        B->h_states[k].active = 0;
                    }
                }
                CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), nc * sizeof(Job), cudaMemcpyHostToDevice, B->stream));
                CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), nc * sizeof(JobState), cudaMemcpyHostToDevice,
                                         B->stream));
                st = run_fused(*B, max_it, poll);
                if (st != INIM_OK) return st;
                for (int k = 0; k < nc; ++k) {
                    const inim_series& x = S[cref[k].series];
                    if (t >= x.T) continue;
                    const int V = x.map->n_verts;
                    CUDA_TRY(cudaMemcpyAsync(x.out_xy + (size_t)t * V * 2, B->bufs[k].xy, (size_t)V * 8,
                                             cudaMemcpyDefault, B->stream));
                    result = worst(result, fill_stats(B->h_states[k], x.stats ? x.stats + t : nullptr));
                }
                CUDA_TRY(cudaStreamSynchronize(B->stream));
            }
        }
    }
    if (d_async) {
        st = collect_direct();
        if (st != INIM_OK) return st;
    }
    return result;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void inim_params_default(inim_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->log2_res = 10;
    p->shape = 0.0f;
    p->bdv_scale = 1.0f;
    p->max_iters = 512;
    p->xi_stop = 0.01f;
    p->stall_window = 32;
    p->eps_stop = 0.0f;
    p->mode = INIM_DIRECT;
    p->precision = INIM_FP32;
    p->form = INIM_FORM_FUSED;
    p->warm_start = 0;
}

const char* inim_status_string(int s) {
    switch (s) {
        case INIM_OK: return "ok";
        case INIM_E_ARG: return "invalid argument";
        case INIM_E_VALUE: return "invalid region value";
        case INIM_E_CUDA: return "CUDA error";
        case INIM_E_TIMEOUT: return "device wait timed out";
        case INIM_E_CAPACITY: return "buffer capacity exceeded";
        case INIM_E_STATE: return "invalid state";
        case INIM_W_NOT_CONVERGED: return "not converged";
        case INIM_W_FOLDOVER: return "fold-over detected";
        default: return "unknown status";
    }
}

const char* inim_last_error(void) { return g_last_error.c_str(); }

// Frames of Sec. 5.5: linear interpolation of the values between consecutive
// time steps, in double, rounded to float.
int inim_interpolate_values(const float* values, int32_t T, int32_t n_regions, int32_t frames_per_step,
                            float* out) {
    if (!values || !out || T < 1 || n_regions < 1 || frames_per_step < 1)
        return fail(INIM_E_ARG, "bad arguments to inim_interpolate_values");
    if (int st = check_values(values, (size_t)T * n_regions)) return st;
    const int f = frames_per_step;
    size_t row = 0;
    for (int t = 0; t + 1 < T; ++t) {
        const float* a = values + (size_t)t * n_regions;
        const float* b = a + n_regions;
        for (int q = 0; q < f; ++q, ++row) {
            const double w = (double)q / (double)f;
            for (int v = 0; v < n_regions; ++v)
                out[row * n_regions + v] = (float)((1.0 - w) * (double)a[v] + w * (double)b[v]);
        }
    }
    std::memcpy(out + row * n_regions, values + (size_t)(T - 1) * n_regions, (size_t)n_regions * 4);
    return INIM_OK;
}

// Eq. (Mb) of Sec. 4.3, host arithmetic in double: the global integral of
// each step, its extremes over the selected steps, the interpolated area
// fraction, the background mass and its spread over the background pixels.
int inim_background_values(const float* values, int32_t T, int32_t n_regions, int32_t log2_res, double a_min,
                           double a_max, int32_t t0, int32_t t1, double* bdv, double* area_fraction) {
    if (!values || !bdv || T < 1 || n_regions < 1) return fail(INIM_E_ARG, "bad arguments to inim_background_values");
    if (log2_res < kMinLog2 || log2_res > kMaxLog2) return fail(INIM_E_ARG, "log2_res must be in [8, 12]");
    if (!(a_min > 0.0 && a_min < a_max && a_max < 1.0)) return fail(INIM_E_ARG, "need 0 < a_min < a_max < 1");
    if (t1 < 0) t1 = T - 1;
    if (t0 < 0 || t0 > t1 || t1 >= T) return fail(INIM_E_ARG, "need 0 <= t0 <= t1 < T");
    if (int st = check_values(values, (size_t)T * n_regions)) return st;
    std::vector<double> mi((size_t)T, 0.0);
    for (int t = 0; t < T; ++t)
        for (int v = 0; v < n_regions; ++v) mi[t] += (double)values[(size_t)t * n_regions + v];
    double m_min = mi[t0], m_max = mi[t0];
    for (int t = t0; t <= t1; ++t) { m_min = std::min(m_min, mi[t]); m_max = std::max(m_max, mi[t]); }
    const double npx = (double)(1 << log2_res) * (double)(1 << log2_res);
    for (int t = 0; t < T; ++t) {
        // weight of a_max; steps outside [t0, t1] are clipped to the ends
        double w = 1.0;
        if (m_max > m_min) w = std::min(1.0, std::max(0.0, (mi[t] - m_min) / (m_max - m_min)));
        const double a = (1.0 - w) * a_min + w * a_max;
        const double m_b = mi[t] * (1.0 - a) / a;           // background mass
        bdv[t] = m_b / ((1.0 - a) * npx);                   // per background pixel of the target
        if (area_fraction) area_fraction[t] = a;
    }
    return INIM_OK;
}

int inim_map_create(const float* xy, int32_t n_verts, const int32_t* ring_off, int32_t n_rings,
                    const int32_t* ring_idx, const int32_t* ring_region, int32_t n_regions, int32_t flags,
                    inim_map** out) {
    if (!out) return fail(INIM_E_ARG, "out is NULL");
    *out = nullptr;
    if (!xy || !ring_off || !ring_idx || !ring_region) return fail(INIM_E_ARG, "NULL input array");
    if (n_verts < 1 || n_rings < 1) return fail(INIM_E_ARG, "n_verts and n_rings must be >= 1");
    if (n_regions < 1 || n_regions > 65534) return fail(INIM_E_ARG, "n_regions must be in [1, 65534]");
    const bool dev = (flags & INIM_MAP_DEVICE_PTRS) != 0;
    auto fetch = [&](const void* src, void* dst, size_t bytes) {
        if (dev) return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
        std::memcpy(dst, src, bytes);
        return cudaSuccess;
    };
    std::vector<float> hxy((size_t)n_verts * 2);
    std::vector<int> hoff(n_rings + 1), hreg(n_rings);
    CUDA_TRY(fetch(xy, hxy.data(), hxy.size() * 4));
    CUDA_TRY(fetch(ring_off, hoff.data(), hoff.size() * 4));
    CUDA_TRY(fetch(ring_region, hreg.data(), hreg.size() * 4));
    if (hoff[0] != 0) return fail(INIM_E_ARG, "ring_off[0] must be 0");
    for (int r = 0; r < n_rings; ++r) {
        if (hoff[r + 1] < hoff[r]) return fail(INIM_E_ARG, "ring_off must be non-decreasing");
        if (hreg[r] < 0 || hreg[r] >= n_regions) return fail(INIM_E_ARG, "ring_region out of range");
    }
    const int total = hoff[n_rings];
    std::vector<int> hidx(std::max(total, 1));
    if (total > 0) CUDA_TRY(fetch(ring_idx, hidx.data(), (size_t)total * 4));
    for (int k = 0; k < total; ++k)
        if (hidx[k] < 0 || hidx[k] >= n_verts) return fail(INIM_E_ARG, "ring_idx out of range");
    for (float v : hxy)
        if (!std::isfinite(v) || v < -1.0f || v > 2.0f) return fail(INIM_E_ARG, "vertex coordinates must lie in [-1, 2]");

    auto m = std::make_unique<inim_map>();
    m->n_verts = n_verts; m->n_regions = n_regions; m->n_rings = n_rings;
    // rings grouped by region, edges grouped by region (ring order kept)
    std::vector<int> reg_ring_off(n_regions + 1, 0), reg_rings(n_rings);
    for (int r = 0; r < n_rings; ++r) reg_ring_off[hreg[r] + 1]++;
    for (int v = 0; v < n_regions; ++v) reg_ring_off[v + 1] += reg_ring_off[v];
    {
        std::vector<int> fill(reg_ring_off.begin(), reg_ring_off.end() - 1);
        for (int r = 0; r < n_rings; ++r) reg_rings[fill[hreg[r]]++] = r;
    }
    std::vector<int2> edges;
    std::vector<int> edge_region;
    std::vector<int> reg_edge_off(n_regions + 1, 0);
    std::vector<float> sign0(n_regions, 0.0f);
    edges.reserve(total);
    for (int v = 0; v < n_regions; ++v) {
        reg_edge_off[v] = (int)edges.size();
        double area2 = 0.0;
        for (int q = reg_ring_off[v]; q < reg_ring_off[v + 1]; ++q) {
            const int r = reg_rings[q];
            const int b = hoff[r], e = hoff[r + 1];
            for (int k = b; k < e; ++k) {
                const int a = hidx[k], c = hidx[k + 1 == e ? b : k + 1];
                edges.push_back(make_int2(a, c));
                edge_region.push_back(v);
                m->h_edge_a.push_back(a);
                m->h_edge_b.push_back(c);
                area2 += (double)hxy[2 * a] * hxy[2 * c + 1] - (double)hxy[2 * c] * hxy[2 * a + 1];
            }
        }
        sign0[v] = area2 > 0.0 ? 1.0f : (area2 < 0.0 ? -1.0f : 0.0f);
    }
    m->n_edges = (int)edges.size();
    reg_edge_off[n_regions] = m->n_edges;
    m->h_xy0 = hxy;
    auto up = [&](void** dst, const void* src, size_t bytes) {
        cudaError_t e = cudaMalloc(dst, bytes < 16 ? 16 : bytes);
        if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = up((void**)&m->edges, edges.data(), edges.size() * sizeof(int2));
    if (e == cudaSuccess) e = up((void**)&m->edge_region, edge_region.data(), edge_region.size() * 4);
    if (e == cudaSuccess) e = up((void**)&m->reg_edge_off, reg_edge_off.data(), reg_edge_off.size() * 4);
    if (e == cudaSuccess) e = up((void**)&m->reg_ring_off, reg_ring_off.data(), reg_ring_off.size() * 4);
    if (e == cudaSuccess) e = up((void**)&m->reg_rings, reg_rings.data(), reg_rings.size() * 4);
    if (e == cudaSuccess) e = up((void**)&m->ring_off, hoff.data(), hoff.size() * 4);
    if (e == cudaSuccess) e = up((void**)&m->ring_idx, hidx.data(), (size_t)total * 4);
    if (e == cudaSuccess) e = up((void**)&m->sign0, sign0.data(), sign0.size() * 4);
    if (e == cudaSuccess) e = up((void**)&m->xy0, hxy.data(), hxy.size() * 4);
    if (e != cudaSuccess) {
        inim_map_destroy(m.release());
        return fail(INIM_E_CUDA, std::string("map upload: ") + cudaGetErrorString(e));
    }
    *out = m.release();
    return INIM_OK;
}

int inim_map_destroy(inim_map* m) {
    if (!m) return INIM_OK;
    purge_map(m);
    dfree(m->edges); dfree(m->edge_region); dfree(m->reg_edge_off); dfree(m->reg_ring_off); dfree(m->reg_rings);
    dfree(m->ring_off); dfree(m->ring_idx); dfree(m->sign0); dfree(m->xy0);
    delete m;
    return INIM_OK;
}

int inim_map_info(const inim_map* m, int32_t* nv, int32_t* nr, int32_t* nrings, int32_t* ne) {
    if (!m) return fail(INIM_E_ARG, "map is NULL");
    if (nv) *nv = m->n_verts;
    if (nr) *nr = m->n_regions;
    if (nrings) *nrings = m->n_rings;
    if (ne) *ne = m->n_edges;
    return INIM_OK;
}

int inim_run_batch(const inim_job* jobs, int32_t n_jobs, void* stream);

int inim_run(inim_map* map, const float* values, int32_t T, const inim_params* params, const float* init_xy,
             float* out_xy, inim_step_stats* stats, void* stream) {
    if (!map || !values || !out_xy || T < 1) return fail(INIM_E_ARG, "bad arguments to inim_run");
    int st = check_params(params);
    if (st != INIM_OK) return st;
    const int R = map->n_regions, V = map->n_verts;
    // host values are checked here, device values where the density table is built
    const bool val_dev = is_device_ptr(values);
    if (!val_dev) {
        st = check_values(values, (size_t)T * R);
        if (st != INIM_OK) return st;
    }
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    const bool out_dev = is_device_ptr(out_xy);
    const float* start = init_xy ? init_xy : map->h_xy0.data();   // host or device

    std::lock_guard<std::mutex> lk(g_cache_mu);
    const bool direct = params->mode == INIM_DIRECT;
    const bool plain = params->form == INIM_FORM_PLAIN;
    if (!plain) {       // the fused form: one series
        inim_series x{map, values, T, init_xy, out_xy, *params, stats};
        return run_series_impl(&x, 1);
    }
    const int nj = (direct && !plain) ? T : 1;
    std::vector<JobSpec> spec(nj, JobSpec{map, params->log2_res, params->precision});
    Batch* B = get_batch(spec, &st);
    if (!B) return st;
    int result = INIM_OK;
    const int rounds = (nj == T) ? 1 : T;
    for (int t = 0; t < rounds; ++t) {
        // values, vertices and state of the jobs of this round
        for (int k = 0; k < nj; ++k) {
            const int step = (nj == T) ? k : t;
            Job& J = B->h_jobs[k];
            J.lam = 1.0f - params->shape;
            J.bdv_scale = params->bdv_scale;
            J.bdv_value = params->bdv_value;
            CUDA_TRY(cudaMemcpyAsync(B->bufs[k].values, values + (size_t)step * R, R * 4, cudaMemcpyDefault, B->stream));
            const bool reset = direct || t == 0;
            if (reset) CUDA_TRY(cudaMemcpyAsync(B->bufs[k].xy, start, (size_t)V * 8, cudaMemcpyDefault, B->stream));
            B->h_states[k] = initial_state(*params, 1, params->max_iters);
        }
        CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), nj * sizeof(Job), cudaMemcpyHostToDevice, B->stream));
        CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), nj * sizeof(JobState), cudaMemcpyHostToDevice, B->stream));
        st = plain ? run_plain(*B, params->max_iters) : run_fused(*B, params->max_iters, needs_poll(*params));
        if (st != INIM_OK) return st;
        for (int k = 0; k < nj; ++k) {
            const int step = (nj == T) ? k : t;
            float* dst = out_xy + (size_t)step * V * 2;
            CUDA_TRY(cudaMemcpyAsync(dst, B->bufs[k].xy, (size_t)V * 8,
                                     out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, B->stream));
            result = worst(result, fill_stats(B->h_states[k], stats ? stats + step : nullptr));
        }
        CUDA_TRY(cudaStreamSynchronize(B->stream));
    }
    return result;
}

int inim_run_series(const inim_series* S, int32_t n, void* stream) {
    if (!S || n < 1) return fail(INIM_E_ARG, "no series");
    for (int i = 0; i < n; ++i) {
        const inim_series& x = S[i];
        if (!x.map || !x.values || !x.out_xy || x.T < 1) return fail(INIM_E_ARG, "series with NULL map/values/out or T < 1");
        int st = check_params(&x.params);
        if (st != INIM_OK) return st;
        if (x.params.form != INIM_FORM_FUSED) return fail(INIM_E_ARG, "inim_run_series needs the fused form");
        if (x.params.precision != S[0].params.precision) return fail(INIM_E_ARG, "all series need one precision");
        if (!is_device_ptr(x.values)) {
            st = check_values(x.values, (size_t)x.T * x.map->n_regions);
            if (st != INIM_OK) return st;
        }
    }
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    std::lock_guard<std::mutex> lk(g_cache_mu);
    return run_series_impl(S, n);
}

int inim_set_persistent(int32_t enable) {
    g_persistent = enable ? 1 : 0;
    return INIM_OK;
}

int inim_set_area_overlap(int32_t enable) {
    g_area_overlap = enable ? 1 : 0;
    return INIM_OK;
}

int inim_set_single_pass_scan(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_single_pass = enable ? 1 : 0;
    g_cache.clear();                  // cached batches keep the form they were built with
    return INIM_OK;
}

int inim_timeline(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    CUDA_TRY(cudaDeviceSynchronize());
    g_cache.clear();                  // cached batches carry the buffer pointer (or none)
    if (enable && !g_tl) {
        CUDA_TRY(cudaMalloc(&g_tl, kTlWords * sizeof(unsigned long long)));
        CUDA_TRY(cudaMemset(g_tl, 0, kTlWords * sizeof(unsigned long long)));
    } else if (!enable && g_tl) {
        dfree(g_tl);
    }
    return INIM_OK;
}

int inim_timeline_read(uint64_t* start_ns, uint64_t* end_ns, int32_t n) {
    if (!start_ns || !end_ns || n < kTlKernels * kTlSlots) return fail(INIM_E_ARG, "timeline buffers too small");
    if (!g_tl) return fail(INIM_E_STATE, "the timeline is off");
    std::vector<unsigned long long> h(kTlWords);
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(h.data(), g_tl, kTlWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(g_tl, 0, kTlWords * sizeof(unsigned long long)));
    for (int i = 0; i < kTlKernels * kTlSlots; ++i) {
        start_ns[i] = h[i];
        end_ns[i] = h[kTlEnd + i];
    }
    return INIM_OK;
}

int inim_set_wait_cap(int64_t spins) {
    set_wait_cap((long long)spins);
    return INIM_OK;
}

int inim_persistent_phase_times(int32_t enable, double* ms, int32_t n) {
    if (enable && !g_phase_ns) CUDA_TRY(cudaMalloc(&g_phase_ns, 8 * sizeof(unsigned long long)));
    if (g_phase_ns && ms && n > 0) {
        unsigned long long h[8];
        CUDA_TRY(cudaMemcpy(h, g_phase_ns, sizeof(h), cudaMemcpyDeviceToHost));
        for (int k = 0; k < n && k < 8; ++k) ms[k] = (double)h[k] * 1e-6;
    }
    if (g_phase_ns) CUDA_TRY(cudaMemset(g_phase_ns, 0, 8 * sizeof(unsigned long long)));
    g_phase_profile = enable ? 1 : 0;
    return INIM_OK;
}

int inim_run_batch(const inim_job* jobs, int32_t n_jobs, void* stream) {
    if (!jobs || n_jobs < 1) return fail(INIM_E_ARG, "no jobs");
    std::vector<JobSpec> spec(n_jobs);
    std::vector<const float*> start_ptr(n_jobs);
    bool poll = false;
    for (int k = 0; k < n_jobs; ++k) {
        const inim_job& j = jobs[k];
        if (!j.map || !j.values || !j.out_xy) return fail(INIM_E_ARG, "job with NULL map, values or out_xy");
        int st = check_params(&j.params);
        if (st != INIM_OK) return st;
        if (j.params.form != INIM_FORM_FUSED) return fail(INIM_E_ARG, "inim_run_batch needs the fused form");
        if (j.params.precision != jobs[0].params.precision) return fail(INIM_E_ARG, "all jobs need one precision");
        if (!is_device_ptr(j.values)) {     // device values are checked where the density table is built
            st = check_values(j.values, j.map->n_regions);
            if (st != INIM_OK) return st;
        }
        start_ptr[k] = j.init_xy ? j.init_xy : (const float*)j.map->xy0;   // the map's device copy
        spec[k] = JobSpec{j.map, j.params.log2_res, j.params.precision};
        poll |= needs_poll(j.params);
    }
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    std::lock_guard<std::mutex> lk(g_cache_mu);
    int st = INIM_OK;
    Batch* B = get_batch(spec, &st);
    if (!B) return st;
    int max_it = 1;
    for (int k = 0; k < n_jobs; ++k) {
        const inim_job& j = jobs[k];
        Job& J = B->h_jobs[k];
        J.lam = 1.0f - j.params.shape;
        J.bdv_scale = j.params.bdv_scale;
        J.bdv_value = j.params.bdv_value;
        CUDA_TRY(cudaMemcpyAsync(B->bufs[k].values, j.values, (size_t)j.map->n_regions * 4, cudaMemcpyDefault, B->stream));
        CUDA_TRY(cudaMemcpyAsync(B->bufs[k].xy, start_ptr[k], (size_t)j.map->n_verts * 8, cudaMemcpyDefault, B->stream));
        B->h_states[k] = initial_state(j.params, 1, j.params.max_iters);
        max_it = std::max(max_it, j.params.max_iters);
    }
    CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), n_jobs * sizeof(Job), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), n_jobs * sizeof(JobState), cudaMemcpyHostToDevice, B->stream));
    st = run_fused(*B, max_it, poll);
    if (st != INIM_OK) return st;
    int result = INIM_OK;
    for (int k = 0; k < n_jobs; ++k) {
        const inim_job& j = jobs[k];
        CUDA_TRY(cudaMemcpyAsync(j.out_xy, B->bufs[k].xy, (size_t)j.map->n_verts * 8, cudaMemcpyDefault, B->stream));
        result = worst(result, fill_stats(B->h_states[k], j.stats));
    }
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    return result;
}

// Dynamic area (Eq. (Mb), Sec. 4.3) over a series: the per-step background
// values on the host, then the steps as single-step jobs carrying them
// (direct: one batch; cumulative: one call per step, each from the previous
// step's vertices).
int inim_run_dynamic(inim_map* map, const float* values, int32_t T, const inim_params* params, double a_min,
                     double a_max, int32_t t0, int32_t t1, const float* init_xy, float* out_xy,
                     inim_step_stats* stats, void* stream) {
    if (!map || !values || !params || !out_xy || T < 1) return fail(INIM_E_ARG, "bad arguments to inim_run_dynamic");
    if (is_device_ptr(values)) return fail(INIM_E_ARG, "inim_run_dynamic takes host values");
    if (params->mode != INIM_DIRECT && params->mode != INIM_CUMULATIVE) return fail(INIM_E_ARG, "bad mode");
    std::vector<double> bdv((size_t)T);
    int st = inim_background_values(values, T, map->n_regions, params->log2_res, a_min, a_max, t0, t1, bdv.data(),
                                    nullptr);
    if (st != INIM_OK) return st;
    const size_t R = (size_t)map->n_regions, V2 = (size_t)map->n_verts * 2;
    std::vector<inim_job> jobs((size_t)T);
    for (int t = 0; t < T; ++t) {
        inim_job& j = jobs[t];
        j.map = map;
        j.values = values + (size_t)t * R;
        j.init_xy = init_xy;
        j.out_xy = out_xy + (size_t)t * V2;
        j.params = *params;
        j.params.mode = INIM_DIRECT;                  // every job is one time step
        j.params.bdv_value = (float)bdv[t];
        j.stats = stats ? stats + t : nullptr;
    }
    if (params->mode == INIM_DIRECT) return inim_run_batch(jobs.data(), T, stream);
    int result = INIM_OK;
    for (int t = 0; t < T; ++t) {
        if (t > 0) jobs[t].init_xy = out_xy + (size_t)(t - 1) * V2;
        st = inim_run_batch(&jobs[t], 1, stream);
        if (st < 0) return st;
        result = worst(result, st);
    }
    return result;
}

int inim_raster(const inim_map* map, const float* xy, int32_t log2_res, uint16_t* labels, int32_t* counts,
                int32_t* overlap, void* stream) {
    if (!map || !xy || !labels || !counts) return fail(INIM_E_ARG, "NULL argument");
    if (log2_res < kMinLog2 || log2_res > kMaxLog2) return fail(INIM_E_ARG, "log2_res must be in [8, 12]");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    std::lock_guard<std::mutex> lk(g_cache_mu);
    int st = INIM_OK;
    std::vector<JobSpec> spec{JobSpec{map, log2_res, INIM_FP32}};
    Batch* B = get_batch(spec, &st);
    if (!B) return st;
    inim_params p;
    inim_params_default(&p);
    B->h_states[0] = initial_state(p, 0, 1);
    B->h_jobs[0].lam = 1.0f;
    B->h_jobs[0].bdv_scale = 1.0f;
    B->h_jobs[0].bdv_value = 0.0f;
    const int R = map->n_regions;
    const int n = 1 << log2_res;
    std::vector<float> ones(R, 1.0f);
    CUDA_TRY(cudaMemcpyAsync(B->bufs[0].values, ones.data(), R * 4, cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->bufs[0].xy, xy, (size_t)map->n_verts * 8, cudaMemcpyDefault, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), sizeof(Job), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), sizeof(JobState), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(launch_raster_prologue(B->d_jobs, (int)B->spec.size(), B->edge_blocks, B->stream));
    CUDA_TRY(launch_raster_main(B->d_jobs, B->edge_blocks, B->row_blocks, B->max_n, B->stream));
    CUDA_TRY(launch_density_table(B->d_jobs, 1, B->stream));
    CUDA_TRY(cudaMemcpyAsync(labels, B->bufs[0].labels, (size_t)n * n * 2, cudaMemcpyDeviceToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(counts, B->bufs[0].counts, (size_t)(R + 1) * 4, cudaMemcpyDeviceToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->h_states.data(), B->d_states, sizeof(JobState), cudaMemcpyDeviceToHost, B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    if (overlap) *overlap = B->h_states[0].overlap;
    if (B->h_states[0].error) return fail(B->h_states[0].error, "raster capacity exceeded");
    return INIM_OK;
}

int inim_density_pooled(const inim_map* map, const float* xy, int32_t log2_res, const float* values, int32_t pool,
                        float* out, void* stream) {
    if (!map || !xy || !values || !out || pool < 1) return fail(INIM_E_ARG, "NULL argument");
    if (log2_res < kMinLog2 || log2_res > kMaxLog2) return fail(INIM_E_ARG, "log2_res must be in [8, 12]");
    if (((1 << log2_res) % pool) != 0) return fail(INIM_E_ARG, "pool must divide N");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    std::lock_guard<std::mutex> lk(g_cache_mu);
    int st = INIM_OK;
    std::vector<JobSpec> spec{JobSpec{map, log2_res, INIM_FP32}};
    Batch* B = get_batch(spec, &st);
    if (!B) return st;
    inim_params p;
    inim_params_default(&p);
    B->h_states[0] = initial_state(p, 0, 1);
    B->h_jobs[0].bdv_scale = 1.0f;
    B->h_jobs[0].bdv_value = 0.0f;
    CUDA_TRY(cudaMemcpyAsync(B->bufs[0].values, values, (size_t)map->n_regions * 4, cudaMemcpyDefault, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->bufs[0].xy, xy, (size_t)map->n_verts * 8, cudaMemcpyDefault, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), sizeof(Job), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), sizeof(JobState), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(launch_raster_prologue(B->d_jobs, (int)B->spec.size(), B->edge_blocks, B->stream));
    CUDA_TRY(launch_raster_main(B->d_jobs, B->edge_blocks, B->row_blocks, B->max_n, B->stream));
    CUDA_TRY(launch_density_table(B->d_jobs, 1, B->stream));
    const int m = (1 << log2_res) / pool;
    float* tmp = nullptr;
    const bool dev = is_device_ptr(out);
    if (!dev) CUDA_TRY(cudaMalloc(&tmp, (size_t)m * m * 4));
    CUDA_TRY(launch_density_pooled(B->d_jobs, 1 << log2_res, pool, dev ? out : tmp, B->stream));
    if (!dev) CUDA_TRY(cudaMemcpyAsync(out, tmp, (size_t)m * m * 4, cudaMemcpyDeviceToHost, B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    if (tmp) cudaFree(tmp);
    return INIM_OK;
}

static int texture_batch(int log2_res, int precision, int frac_bits, const float* density, Batch** out) {
    int st = INIM_OK;
    std::vector<JobSpec> spec{JobSpec{nullptr, log2_res, precision}};
    Batch* B = get_batch(spec, &st);
    if (!B) return st;
    inim_params p;
    inim_params_default(&p);
    B->h_states[0] = initial_state(p, 0, 1);
    B->h_states[0].fix_bits = frac_bits;
    CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), sizeof(Job), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), sizeof(JobState), cudaMemcpyHostToDevice, B->stream));
    const Group& g = B->groups[0];
    if (precision == INIM_FIX64) CUDA_TRY(launch_scan_fix64(B->d_jobs, g.band, g.carry, g.tile, density, B->stream));
    else if (precision == INIM_KAHAN) CUDA_TRY(launch_scan_kahan(B->d_jobs, g.band, g.carry, g.tile, density, B->stream));
    else CUDA_TRY(launch_scan_fp32(B->d_jobs, g.band, g.carry, g.tile, density, B->stream));
    *out = B;
    return INIM_OK;
}

int inim_inims(const float* density, int32_t log2_res, int32_t precision, int32_t frac_bits, void* S, void* T,
               void* A, void* Bv, void* stream) {
    if (!density || !S || !T || !A || !Bv) return fail(INIM_E_ARG, "NULL argument");
    if (log2_res < kMinLog2 || log2_res > kMaxLog2) return fail(INIM_E_ARG, "log2_res must be in [8, 12]");
    if (precision < INIM_FP32 || precision > INIM_KAHAN) return fail(INIM_E_ARG, "bad precision");
    if (precision == INIM_FIX64 && (frac_bits < 0 || frac_bits > 62)) return fail(INIM_E_ARG, "bad frac_bits");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    std::lock_guard<std::mutex> lk(g_cache_mu);
    Batch* B = nullptr;
    int st = texture_batch(log2_res, precision, frac_bits, density, &B);
    if (st != INIM_OK) return st;
    CUDA_TRY(launch_finalize_B(B->d_jobs, precision, B->stream));
    const size_t n = (size_t)1 << log2_res, es = elem_size(precision);
    CUDA_TRY(cudaMemcpyAsync(S, B->bufs[0].S, n * n * es, cudaMemcpyDeviceToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(T, B->bufs[0].T, n * n * es, cudaMemcpyDeviceToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(A, B->bufs[0].A, (2 * n - 1) * es, cudaMemcpyDeviceToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(Bv, B->bufs[0].B, (2 * n - 1) * es, cudaMemcpyDeviceToDevice, B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    return INIM_OK;
}

int inim_displacement(const float* density, int32_t log2_res, int32_t precision, const float* xy, int32_t n,
                      float* delta, void* stream) {
    if (!density || !xy || !delta || n < 0) return fail(INIM_E_ARG, "bad arguments");
    if (log2_res < kMinLog2 || log2_res > kMaxLog2) return fail(INIM_E_ARG, "log2_res must be in [8, 12]");
    if (precision < INIM_FP32 || precision > INIM_KAHAN) return fail(INIM_E_ARG, "bad precision");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    std::lock_guard<std::mutex> lk(g_cache_mu);
    // fixed point: 2^30 units per unit density keeps 4096^2 textures of
    // densities up to 2^6 below 2^62
    Batch* B = nullptr;
    int st = texture_batch(log2_res, precision, 30, density, &B);
    if (st != INIM_OK) return st;
    CUDA_TRY(launch_displacement(B->d_jobs, xy, n, delta, precision, B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    return INIM_OK;
}

int inim_iterate(const inim_map* map, float* xy, const float* values, const inim_params* params, int32_t n_iters,
                 inim_step_stats* stats, void* stream) {
    if (!map || !xy || !values || n_iters < 0) return fail(INIM_E_ARG, "bad arguments");
    int st = check_params(params);
    if (st != INIM_OK) return st;
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    std::vector<float> hv = to_host(values, map->n_regions);
    st = check_values(hv.data(), hv.size());
    if (st != INIM_OK) return st;
    std::vector<float> hxy = to_host(xy, (size_t)map->n_verts * 2);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    std::vector<JobSpec> spec{JobSpec{map, params->log2_res, params->precision}};
    Batch* B = get_batch(spec, &st);
    if (!B) return st;
    Job& J = B->h_jobs[0];
    J.lam = 1.0f - params->shape;
    J.bdv_scale = params->bdv_scale;
    J.bdv_value = params->bdv_value;
    B->h_states[0] = initial_state(*params, 0, std::max(n_iters, 1));
    CUDA_TRY(cudaMemcpyAsync(B->bufs[0].values, hv.data(), hv.size() * 4, cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->bufs[0].xy, hxy.data(), hxy.size() * 4, cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), sizeof(Job), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), sizeof(JobState), cudaMemcpyHostToDevice, B->stream));
    if (n_iters > 0) {
        if (params->form == INIM_FORM_PLAIN) st = run_plain(*B, n_iters);
        else {
            CUDA_TRY(enqueue_prologue(*B, B->stream));
            for (int k = 0; k < n_iters; ++k) CUDA_TRY(enqueue_fused_iteration(*B, B->stream));
            g_launches += 1 + (long long)n_iters * kernels_per_fused_iteration(*B);
            CUDA_TRY(cudaMemcpyAsync(B->h_states.data(), B->d_states, sizeof(JobState), cudaMemcpyDeviceToHost, B->stream));
            CUDA_TRY(cudaStreamSynchronize(B->stream));
        }
        if (st != INIM_OK) return st;
    }
    CUDA_TRY(cudaMemcpyAsync(xy, B->bufs[0].xy, (size_t)map->n_verts * 8, cudaMemcpyDefault, B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    return fill_stats(B->h_states[0], stats);
}

int inim_areas(const inim_map* map, const float* xy, double* areas, void* stream) {
    if (!map || !xy || !areas) return fail(INIM_E_ARG, "NULL argument");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    std::vector<float> hxy = to_host(xy, (size_t)map->n_verts * 2);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    int st = INIM_OK;
    std::vector<JobSpec> spec{JobSpec{map, kMinLog2, INIM_FP32}};
    Batch* B = get_batch(spec, &st);
    if (!B) return st;
    inim_params p;
    inim_params_default(&p);
    B->h_states[0] = initial_state(p, 0, 1);
    CUDA_TRY(cudaMemcpyAsync(B->bufs[0].xy, hxy.data(), hxy.size() * 4, cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs.data(), sizeof(Job), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_states, B->h_states.data(), sizeof(JobState), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(launch_areas_errors(B->d_jobs, B->region_blocks, -1, B->stream));
    CUDA_TRY(cudaMemcpyAsync(areas, B->bufs[0].areas, (size_t)map->n_regions * 8, cudaMemcpyDefault, B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    return INIM_OK;
}

// Quality measures of Sec. 3.3: both rasters through inim_raster, then the
// kernels of quality.cu on the caller's stream; the bounding boxes come back
// to the host once to lay out the shape masks and the translation work.
int inim_quality(const inim_map* map, const float* xy_map, const float* xy_cart, int32_t log2_res,
                 inim_quality_out* out, double* shape_per, void* stream) {
    if (!map || !xy_cart || !out) return fail(INIM_E_ARG, "NULL map, xy_cart or out");
    if (log2_res < kMinLog2 || log2_res > kMaxLog2) return fail(INIM_E_ARG, "log2_res must be in [8, 12]");
    const int R = map->n_regions, V = map->n_verts, n = 1 << log2_res;
    const size_t np = (size_t)n * n;
    const cudaStream_t s = (cudaStream_t)stream;
    DevScratch w;
    uint16_t* lab[2];
    int* cnt[2];
    const float* xy[2] = {xy_map ? xy_map : (const float*)map->xy0, xy_cart};
    for (int r = 0; r < 2; ++r) {
        CUDA_TRY(w.get(&lab[r], np * 2));
        CUDA_TRY(w.get(&cnt[r], (size_t)(R + 1) * 4));
        const int st = inim_raster(map, xy[r], log2_res, lab[r], cnt[r], nullptr, stream);
        if (st < 0) return st;
    }
    // topology: one adjacency bitmap per raster, then the four pair counts
    const long long nw = ((long long)R * R + 31) / 32;
    uint32_t* bits[2];
    unsigned long long* pc;
    for (int r = 0; r < 2; ++r) {
        CUDA_TRY(w.get(&bits[r], (size_t)nw * 4));
        CUDA_TRY(cudaMemsetAsync(bits[r], 0, (size_t)nw * 4, s));
        CUDA_TRY(launch_adjacency(lab[r], log2_res, R, bits[r], s));
    }
    CUDA_TRY(w.get(&pc, 4 * sizeof(unsigned long long)));
    CUDA_TRY(cudaMemsetAsync(pc, 0, 4 * sizeof(unsigned long long), s));
    CUDA_TRY(launch_pair_counts(bits[0], bits[1], nw, pc, s));
    // shape: bounding boxes, mask layout and translation chunks
    int* box[2];
    std::vector<int> hb[2];
    for (int r = 0; r < 2; ++r) {
        CUDA_TRY(w.get(&box[r], (size_t)R * 16));
        CUDA_TRY(launch_bbox(lab[r], log2_res, R, box[r], s));
        hb[r].resize((size_t)R * 4);
        CUDA_TRY(cudaMemcpyAsync(hb[r].data(), box[r], (size_t)R * 16, cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<QRegion> reg((size_t)R);
    std::vector<int2> items;
    long long words[2] = {0, 0};
    for (int v = 0; v < R; ++v) {
        QRegion& g = reg[v];
        g = QRegion{};
        if (hb[0][4 * v + 1] < 0 || hb[1][4 * v + 1] < 0) continue;      // missing from a raster
        for (int r = 0; r < 2; ++r) {
            g.x0[r] = hb[r][4 * v + 0];
            g.y0[r] = hb[r][4 * v + 2];
            g.w[r] = hb[r][4 * v + 1] - g.x0[r] + 1;
            g.h[r] = hb[r][4 * v + 3] - g.y0[r] + 1;
            g.W[r] = (g.w[r] + 31) / 32;
            g.off[r] = words[r];
            words[r] += (long long)g.W[r] * g.h[r];
        }
        const long long ntr = (long long)(g.w[0] + g.w[1] - 1) * (g.h[0] + g.h[1] - 1);
        const long long chunks = (ntr + kQualityChunk - 1) / kQualityChunk;
        if ((long long)items.size() + chunks > (long long)INT_MAX)
            return fail(INIM_E_CAPACITY, "shape distortion: too many translations for one launch");
        for (long long c = 0; c < chunks; ++c) items.push_back(make_int2(v, (int)c));
    }
    QRegion* d_reg;
    int2* d_items;
    uint32_t* masks[2];
    int* omax;
    double *per, *shp;
    CUDA_TRY(w.get(&d_reg, (size_t)R * sizeof(QRegion)));
    CUDA_TRY(cudaMemcpyAsync(d_reg, reg.data(), (size_t)R * sizeof(QRegion), cudaMemcpyHostToDevice, s));
    CUDA_TRY(w.get(&d_items, items.size() * sizeof(int2)));
    if (!items.empty())
        CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    for (int r = 0; r < 2; ++r) {
        CUDA_TRY(w.get(&masks[r], (size_t)words[r] * 4));
        CUDA_TRY(cudaMemsetAsync(masks[r], 0, (size_t)words[r] * 4, s));
        CUDA_TRY(launch_pack(lab[r], log2_res, R, d_reg, r, masks[r], s));
    }
    CUDA_TRY(w.get(&omax, (size_t)R * 4));
    CUDA_TRY(cudaMemsetAsync(omax, 0, (size_t)R * 4, s));
    CUDA_TRY(launch_correlate(d_items, (int)items.size(), d_reg, masks[0], masks[1], omax, s));
    CUDA_TRY(w.get(&per, (size_t)R * 8));
    CUDA_TRY(w.get(&shp, 2 * sizeof(double)));
    CUDA_TRY(launch_shape_final(cnt[0], cnt[1], omax, R, per, shp, s));
    // relative positions: barycentres of both vertex sets
    float2* dxy[2];
    double2* bary[2];
    for (int r = 0; r < 2; ++r) {
        if (r == 0 && !xy_map) {
            dxy[0] = map->xy0;
        } else {
            CUDA_TRY(w.get(&dxy[r], (size_t)V * 8));
            CUDA_TRY(cudaMemcpyAsync(dxy[r], xy[r], (size_t)V * 8, cudaMemcpyDefault, s));
        }
        CUDA_TRY(w.get(&bary[r], (size_t)R * sizeof(double2)));
        CUDA_TRY(launch_barycentres(map->reg_ring_off, map->reg_rings, map->ring_off, map->ring_idx, dxy[r], R,
                                    bary[r], s));
    }
    double *partial, *rp;
    CUDA_TRY(w.get(&partial, (size_t)rel_pos_blocks() * 8));
    CUDA_TRY(w.get(&rp, 8));
    CUDA_TRY(launch_rel_pos(bary[0], bary[1], R, partial, rp, s));
    unsigned long long hc[4];
    double hs[2], hr;
    CUDA_TRY(cudaMemcpyAsync(hc, pc, sizeof(hc), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(hs, shp, sizeof(hs), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&hr, rp, sizeof(hr), cudaMemcpyDeviceToHost, s));
    if (shape_per) CUDA_TRY(cudaMemcpyAsync(shape_per, per, (size_t)R * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    out->adj_map = (int64_t)hc[0];
    out->adj_cart = (int64_t)hc[1];
    out->adj_both = (int64_t)hc[2];
    out->tau = hc[3] == 0 ? 0.0 : 1.0 - (double)hc[2] / (double)hc[3];
    out->n_present = (int32_t)hs[1];
    out->shape = hs[1] > 0.0 ? hs[0] / hs[1] : 0.0;
    out->rel_pos = hr;
    out->pad = 0;
    return INIM_OK;
}

int inim_set_scan_tile(int32_t log2_res, int32_t precision, int32_t large, int32_t band_rows,
                       int32_t cols_per_thread, int32_t threads) {
    if (log2_res < kMinLog2 || log2_res > kMaxLog2 || precision < INIM_FP32 || precision > INIM_KAHAN)
        return fail(INIM_E_ARG, "bad resolution or precision");
    ScanTile t{band_rows, cols_per_thread, threads};
    if (band_rows == 0) t = ScanTile{0, 0, 0};              // back to the default
    else if (!tile_valid(log2_res, t)) return fail(INIM_E_ARG, "no compiled scan kernel for this tile");
    purge_all();
    g_tiles[precision][large ? 1 : 0][log2_res] = t;
    return INIM_OK;
}

int inim_get_scan_tile(int32_t log2_res, int32_t precision, int32_t large, int32_t* band_rows,
                       int32_t* cols_per_thread, int32_t* threads) {
    if (log2_res < kMinLog2 || log2_res > kMaxLog2 || precision < INIM_FP32 || precision > INIM_KAHAN)
        return fail(INIM_E_ARG, "bad resolution or precision");
    const ScanTile t = tile_for(log2_res, precision, large ? 1 : 0);
    if (band_rows) *band_rows = t.H;
    if (cols_per_thread) *cols_per_thread = t.cpt;
    if (threads) *threads = t.nt;
    return INIM_OK;
}

int inim_autotune_scan(const inim_job* jobs, int32_t n_jobs, int32_t reps) {
    if (!jobs || n_jobs < 1 || reps < 1) return fail(INIM_E_ARG, "bad arguments");
    std::vector<JobSpec> spec(n_jobs);
    for (int k = 0; k < n_jobs; ++k) {
        const inim_job& j = jobs[k];
        if (!j.map || !j.values) return fail(INIM_E_ARG, "job with NULL map or values");
        int st = check_params(&j.params);
        if (st != INIM_OK) return st;
        if (j.params.precision != jobs[0].params.precision) return fail(INIM_E_ARG, "all jobs need one precision");
        spec[k] = JobSpec{j.map, j.params.log2_res, j.params.precision};
    }
    Batch B;
    int st = build_batch(B, spec, kTileHeights[0]);
    if (st != INIM_OK) return st;
    for (int k = 0; k < n_jobs; ++k) {
        const inim_job& j = jobs[k];
        B.h_jobs[k].lam = 1.0f - j.params.shape;
        B.h_jobs[k].bdv_scale = j.params.bdv_scale;
        B.h_jobs[k].bdv_value = j.params.bdv_value;
        CUDA_TRY(cudaMemcpyAsync(B.bufs[k].values, j.values, (size_t)j.map->n_regions * 4, cudaMemcpyDefault, B.stream));
        CUDA_TRY(cudaMemcpyAsync(B.bufs[k].xy, j.init_xy ? j.init_xy : j.map->h_xy0.data(),
                                 (size_t)j.map->n_verts * 8, cudaMemcpyDefault, B.stream));
        B.h_states[k] = initial_state(j.params, 0, INT_MAX);
    }
    CUDA_TRY(cudaMemcpyAsync(B.d_jobs, B.h_jobs.data(), n_jobs * sizeof(Job), cudaMemcpyHostToDevice, B.stream));
    CUDA_TRY(cudaMemcpyAsync(B.d_states, B.h_states.data(), n_jobs * sizeof(JobState), cudaMemcpyHostToDevice, B.stream));
    // labels and densities of the start positions
    CUDA_TRY(launch_raster_prologue(B.d_jobs, (int)B.spec.size(), B.edge_blocks, B.stream));
    CUDA_TRY(launch_raster_main(B.d_jobs, B.edge_blocks, B.row_blocks, B.max_n, B.stream));
    CUDA_TRY(launch_density_table(B.d_jobs, n_jobs, B.stream));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    std::vector<std::pair<int, ScanTile>> chosen;
    for (auto& g : B.groups) {
        float best = 1e30f;
        ScanTile best_t = g.tile;
        for (auto& q : kTilePairs) {
            for (int H : kTileHeights) {
                ScanTile t{H, q[0], q[1], 1 << g.log2n};
                if (!tile_valid(g.log2n, t)) continue;
                st = retile_group(B, g, t);
                if (st != INIM_OK) return st;
                auto scan = [&]() {
                    if (B.precision == INIM_FIX64) return launch_scan_fix64(B.d_jobs, g.band, g.carry, t, nullptr, B.stream);
                    if (B.precision == INIM_KAHAN) return launch_scan_kahan(B.d_jobs, g.band, g.carry, t, nullptr, B.stream);
                    return launch_scan_fp32(B.d_jobs, g.band, g.carry, t, nullptr, B.stream);
                };
                CUDA_TRY(scan());                                  // warm
                CUDA_TRY(cudaEventRecord(e0, B.stream));
                for (int r = 0; r < reps; ++r) CUDA_TRY(scan());
                CUDA_TRY(cudaEventRecord(e1, B.stream));
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.0f;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; best_t = t; }
            }
        }
        long long px = 0;
        for (auto& sp : spec) if (sp.log2n == g.log2n) px += 1LL << (2 * sp.log2n);
        chosen.push_back({g.log2n * 2 + size_class(px), best_t});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(cudaStreamSynchronize(B.stream));
    purge_all();
    for (auto& c : chosen) g_tiles[B.precision][c.first & 1][c.first >> 1] = c.second;
    return INIM_OK;
}

static const char* kStageNames[] = {"crossings", "raster_rows", "density_table", "scan_phase1", "scan_carry",
                                     "scan_phase3", "gather_move", "areas_errors", "scan_fused"};
constexpr int kNumStages = 9;

const char* inim_stage_name(int32_t i) {
    return (i >= 0 && i < kNumStages) ? kStageNames[i] : "";
}

long long inim_launch_count(void) { return g_launches.load(); }

int inim_profile_stages(int32_t reps, float* ms, int32_t max_stages, int32_t* n_stages) {
    if (reps < 1 || !ms || max_stages < kNumStages) return fail(INIM_E_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (g_cache.empty() || !g_cache.front()->spec[0].map) return fail(INIM_E_STATE, "no map batch has run yet");
    Batch& B = *g_cache.front();
    const int nj = (int)B.spec.size();
    for (int k = 0; k < nj; ++k) {
        JobState& s = B.h_states[k];
        s.active = 1; s.stop_on_rule = 0; s.max_iters = INT_MAX; s.error = 0;
    }
    CUDA_TRY(cudaMemcpyAsync(B.d_states, B.h_states.data(), nj * sizeof(JobState), cudaMemcpyHostToDevice, B.stream));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    auto stage = [&](int i) -> cudaError_t {
        switch (i) {
            case 2: return launch_density_table(B.d_jobs, nj, B.stream);
            case 3: case 4: case 5: case 8: {
                // phases 1-3 of three-kernel groups; 8: the single-pass groups
                const int phase = i == 8 ? 4 : i - 2;
                cudaError_t e = cudaSuccess;
                for (auto& g : B.groups) {
                    if (B.precision == INIM_FIX64) e = launch_scan_fix64(B.d_jobs, g.band, g.carry, g.tile, nullptr, B.stream, phase);
                    else if (B.precision == INIM_KAHAN) e = launch_scan_kahan(B.d_jobs, g.band, g.carry, g.tile, nullptr, B.stream, phase);
                    else e = launch_scan_fp32(B.d_jobs, g.band, g.carry, g.tile, nullptr, B.stream, phase);
                    if (e != cudaSuccess) break;
                }
                return e;
            }
            // back-to-back moves: each reads its vertices before its launch
            // wait, so it may see the previous replay's moves half done (the
            // values only feed this timing run; every run restarts from its
            // start positions)
            case 6: return launch_gather(B.d_jobs, B.vert_blocks, B.precision, B.stream);
            default: return launch_areas_errors(B.d_jobs, B.region_blocks, 0, B.stream);
        }
    };
    int rc = INIM_OK;
    // reps launches captured into one CUDA graph (with the launches'
    // programmatic dependent-launch edges, as in the iteration graphs), timed
    // between two events around one replay: the host's launch rate does not
    // enter the per-launch time
    auto graph_ms = [&](const std::function<cudaError_t()>& fn, float* out) -> cudaError_t {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = fn();
        const cudaError_t e2 = cudaStreamEndCapture(B.stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, B.stream);                 // warm
        if (e == cudaSuccess) e = cudaEventRecord(e0, B.stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, B.stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, B.stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        *out = t / (float)reps;
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        return e;
    };
    // the rasteriser's two kernels run as pairs (the rows empty the buckets
    // the crossings fill); the crossing kernel alone is timed on its own graph
    // (its keys then overflow the buckets, whose guard skips the stores) and
    // the rows get the difference; the buckets are emptied afterwards
    {
        float t_pair = 0.0f, t_c = 0.0f;
        cudaError_t e = graph_ms([&] { return launch_raster_main(B.d_jobs, B.edge_blocks, B.row_blocks, B.max_n,
                                                                 B.stream); }, &t_pair);
        if (e == cudaSuccess) e = graph_ms([&] { return launch_raster_crossings(B.d_jobs, B.edge_blocks, B.stream); },
                                           &t_c);
        if (e == cudaSuccess) e = launch_raster_prologue(B.d_jobs, nj, B.edge_blocks, B.stream);
        if (e == cudaSuccess) e = launch_raster_main(B.d_jobs, B.edge_blocks, B.row_blocks, B.max_n, B.stream);
        if (e != cudaSuccess) rc = fail(INIM_E_CUDA, std::string("profile: ") + cudaGetErrorString(e));
        ms[0] = t_c;
        ms[1] = t_pair > t_c ? t_pair - t_c : 0.0f;
    }
    for (int i = 2; i < kNumStages && rc == INIM_OK; ++i) {
        if (i == 2 && B.fuse_table) { ms[i] = 0.0f; continue; }     // built by the scan's first phase
        bool any_fused = false, any_split = false;
        for (auto& g : B.groups) (g.tile.fused ? any_fused : any_split) = true;
        if ((i >= 3 && i <= 5 && !any_split) || (i == 8 && !any_fused)) { ms[i] = 0.0f; continue; }
        const cudaError_t e = graph_ms([&] { return stage(i); }, &ms[i]);
        if (e != cudaSuccess) rc = fail(INIM_E_CUDA, std::string("profile: ") + cudaGetErrorString(e));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_stages) *n_stages = kNumStages;
    return rc;
}

}  // extern "C"
