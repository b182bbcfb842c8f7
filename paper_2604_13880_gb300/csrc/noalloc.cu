// Allocation-free variant of the FP32 integral-image entry point.
//
// Some callers cannot allocate device memory: code that runs under another
// framework's memory manager which owns the whole device pool, or a
// latency-critical loop in which cudaMalloc / cudaFree (which can synchronise
// the device) are not acceptable.  inim_inims_noalloc serves them: the
// caller passes the texture and the output buffers, and every other byte the
// band scan needs (job descriptor, block tables, band aggregates and carries,
// row sums) lives in one fixed array compiled into this library.
//
// Limits and sharing:
//   - N <= 1024 (log2_res <= 10); larger textures are rejected.
//   - The array (kScratchBytes, about 1.6 MB) is held by every GPU that loads
//     the library until the process exits.
//   - Every call uses the same array and leaves its contents behind; calls
//     whose kernels overlap on the GPU (different streams, no ordering) race.
//   - The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current); make that first call
//     before any stream capture.  The address is kept for the life of the
//     process: a cudaDeviceReset between calls is not supported.
//   - A small set-up kernel writes the job descriptor and block tables into
//     the array; the first scan kernel after it is launched in plain stream
//     order (not as a programmatic dependent launch), because the scan
//     kernels read those tables before they wait on their predecessor.
#include <mutex>

#include "scan_impl.cuh"

namespace inim {

namespace {

constexpr int kNaMaxLog2 = 10;
constexpr int kNaMaxN = 1 << kNaMaxLog2;
constexpr int kNaH = 16;                                   // band height
constexpr int kNaMaxNb = kNaMaxN / kNaH;
constexpr int kNaMaxCarryBlocks = (kNaMaxN + 2 * (kNaMaxN + (kNaMaxNb - 1) * kNaH) + 255) / 256;

// layout of the scratch array (every part 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffJob = 0;
constexpr size_t kOffState = align256(kOffJob + sizeof(Job));
constexpr size_t kOffBandMap = align256(kOffState + sizeof(JobState));
constexpr size_t kOffCarryMap = align256(kOffBandMap + kNaMaxNb * sizeof(int2));
constexpr size_t kOffRowcum = align256(kOffCarryMap + kNaMaxCarryBlocks * sizeof(int2));
constexpr size_t kOffAgg = align256(kOffRowcum + kNaMaxN * sizeof(float));
constexpr size_t kOffCarry = align256(kOffAgg + (size_t)3 * kNaMaxNb * kNaMaxN * sizeof(float));
constexpr size_t kScratchBytes = align256(kOffCarry + (size_t)3 * kNaMaxNb * kNaMaxN * sizeof(float));

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// device address of g_scratch per device, looked up once
std::mutex g_mu;
void* g_addr[128] = {};

// writes the job descriptor, its state and the block tables into the scratch
__global__ void k_noalloc_setup(Job job, int nb, int carry_blocks, unsigned char* base) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *reinterpret_cast<Job*>(base + kOffJob) = job;
        JobState st{};
        st.active = 1;
        st.max_iters = 1;
        *reinterpret_cast<JobState*>(base + kOffState) = st;
    }
    int2* band = reinterpret_cast<int2*>(base + kOffBandMap);
    int2* carry = reinterpret_cast<int2*>(base + kOffCarryMap);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) band[b] = make_int2(0, b);
    for (int q = threadIdx.x; q < carry_blocks; q += blockDim.x) carry[q] = make_int2(0, q);
}

}  // namespace

}  // namespace inim

extern "C" int inim_inims_noalloc(const float* density, int32_t log2_res, float* S, float* T, float* A, float* B,
                                  void* stream) {
    using namespace inim;
    if (!density || !S || !T || !A || !B) return set_last_error(INIM_E_ARG, "inim_inims_noalloc: null pointer");
    if (log2_res < kMinLog2) return set_last_error(INIM_E_ARG, "inim_inims_noalloc: log2_res below 8");
    if (log2_res > kNaMaxLog2)                             // beyond the fixed scratch array
        return set_last_error(INIM_E_CAPACITY, "inim_inims_noalloc: log2_res above 10 (N <= 1024)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128)
        return set_last_error(INIM_E_CUDA, "inim_inims_noalloc: no current device");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p)
                return set_last_error(INIM_E_CUDA, "inim_inims_noalloc: cudaGetSymbolAddress failed");
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    const int n = 1 << log2_res;
    const int nb = n / kNaH;
    const int carry_blocks = (carry_qspace(n, nb, kNaH) + 255) / 256;
    constexpr int NT = 128;
    ScanTile tile{kNaH, log2_res == 8 ? 2 : (log2_res == 9 ? 4 : 8), NT};

    Job J{};
    J.n = n;
    J.log2n = log2_res;
    J.precision = INIM_FP32;
    J.S = S;
    J.T = T;
    J.A = A;
    J.B = B;
    J.rowcum = b + kOffRowcum;
    J.H = kNaH;
    J.nb = nb;
    J.agg = b + kOffAgg;
    J.carry = b + kOffCarry;
    J.st = reinterpret_cast<JobState*>(b + kOffState);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_noalloc_setup<<<1, 128, 0, s>>>(J, nb, carry_blocks, b);
    if (cudaGetLastError() != cudaSuccess) return set_last_error(INIM_E_CUDA, "inim_inims_noalloc: set-up launch");
    const Job* dj = reinterpret_cast<const Job*>(b + kOffJob);
    BlockMap band, carry;
    band.d_map = reinterpret_cast<int2*>(b + kOffBandMap);
    band.n_blocks = nb;
    carry.d_map = reinterpret_cast<int2*>(b + kOffCarryMap);
    carry.n_blocks = carry_blocks;
    // phase 1 in plain stream order: it starts only once the set-up kernel
    // has finished and its writes are visible
    const size_t ring = (size_t)kLabelDepth * n * 2;    // CPT * NT = n
    switch (tile.cpt) {
        case 2: k_scan_band<AccF32, 2, NT, 1><<<nb, NT, ring, s>>>(dj, band.d_map, density); break;
        case 4: k_scan_band<AccF32, 4, NT, 1><<<nb, NT, ring, s>>>(dj, band.d_map, density); break;
        default: k_scan_band<AccF32, 8, NT, 1><<<nb, NT, ring, s>>>(dj, band.d_map, density); break;
    }
    if (cudaGetLastError() != cudaSuccess) return set_last_error(INIM_E_CUDA, "inim_inims_noalloc: scan launch");
    if (launch_scan_fp32(dj, band, carry, tile, density, s, 2) != cudaSuccess ||
        launch_scan_fp32(dj, band, carry, tile, density, s, 3) != cudaSuccess)
        return set_last_error(INIM_E_CUDA, "inim_inims_noalloc: scan launch");
    if (launch_finalize_B(dj, INIM_FP32, s) != cudaSuccess)
        return set_last_error(INIM_E_CUDA, "inim_inims_noalloc: finalize launch");
    return INIM_OK;
}
