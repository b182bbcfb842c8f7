// Bulk asynchronous copies (the TMA engine's 1-D form, cp.async.bulk) from
// global into shared memory, completed on shared-memory mbarriers.  Used to
// stage texture rows ahead of the row loops of the scan: one thread issues
// the copy of a whole row, every thread of the block waits on the row's
// barrier phase.
//
// Every wait is bounded: after kTmaSpinCap polls it gives up and returns
// false, and the caller records INIM_E_TIMEOUT and leaves, so a copy that
// never lands cannot hang the GPU.  Copies need 16-byte aligned addresses
// and a size that is a multiple of 16 bytes (texture rows of N >= 256 u16
// pixels from a cudaMalloc base satisfy both).
#pragma once

#include <cstdint>

namespace inim {

constexpr unsigned kTmaSpinCap = 1u << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy (then a block barrier)
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one thread: expect `bytes` on the barrier's current phase, then start the copy
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// one thread: start a copy whose bytes an earlier expect_tx on the barrier announced
__device__ __forceinline__ void tma_copy_1d(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// wait until the barrier's phase with the given parity has completed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const unsigned a = smem_addr(bar);
    for (unsigned k = 0; k < kTmaSpinCap; ++k) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace inim
