// tma.cuh - mbarrier and 2-D TMA tensor-copy helpers shared by the replay kernels.
//
// Every wait is bounded by the %globaltimer clock: a wait that gives up returns false and
// the caller records MAGUS_ETIMEDOUT instead of spinning forever.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "replay_core.cuh"

namespace magus {
namespace tma {

constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded waits: 2 s

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(core::smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(core::smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(core::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(core::smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Non-blocking probe of the phase (test_wait returns at once; try_wait may suspend the
// thread until the phase completes, which a short limit must not wait for).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(core::smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for `parity` of `bar` with a time limit (default 2 s); false on timeout.  A limit
// below the default polls with test_wait and measures it in SM cycles (two per ns, so the
// wait lasts at least the limit at any clock up to 2 GHz; the cycle counter advances every
// cycle, where the global timer may advance in coarser steps).
static __device__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned long long limit_ns = kWaitNs) {
    if (limit_ns < kWaitNs) {
        const long long c0 = clock64();
        const long long lim = (long long)(2 * limit_ns);
        while (true) {
            if (mbar_test_wait(bar, parity)) return true;
            if (clock64() - c0 >= lim) return false;
        }
    }
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
}
// 2-D tensor copy of the box at (x = 0, y = row) of the trace buffer into shared memory.
// Every trace byte is read once, so the copy asks L2 to evict its lines first: the lines
// that stay are the outputs being written (change-log entries arrive a few at a time and
// are merged in L2 instead of reaching DRAM as partial sectors).
__device__ __forceinline__ void tma_rows(uint32_t dst, const CUtensorMap *tmap, int y, uint64_t *bar) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(tmap), "r"(0), "r"(y), "r"(core::smem_u32(bar)), "l"(pol)
        : "memory");
}

}  // namespace tma
}  // namespace magus
