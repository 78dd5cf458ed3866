// mbarrier and tensor-memory-accelerator (TMA) helpers, inline PTX for
// sm_103a: barrier set-up, bounded waits, and tiled global -> shared copies
// described by a tensor map and completed on an mbarrier (transaction bytes).
#pragma once

#include <cuda.h>   // CUtensorMap (the type only; maps are encoded on the host)
#include <stdint.h>

namespace bloch {

constexpr long long kMbarSpin = 1ll << 24;   // bound on mbarrier polls

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// bytes from p to the next 128-byte boundary of the shared window (TMA tile
// destinations); kernels that use it request kSmemAlignSlack extra bytes
constexpr int kSmemAlignSlack = 128;
__device__ __forceinline__ uint32_t smem_pad128(const void* p) { return (128u - (smem_u32(p) & 127u)) & 127u; }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < kMbarSpin; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// one arrival that also announces `bytes` of asynchronous transactions
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// orders this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy (TMA, tensor core) accesses
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Tiled copy of the box at coordinates (x, y, z) of the 3D tensor map into
// shared memory at dst; completion adds the box bytes to mbarrier bar.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

}  // namespace bloch
