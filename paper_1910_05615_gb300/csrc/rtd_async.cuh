// rtd_async.cuh - bulk asynchronous global -> shared copies completed on an
// mbarrier (sm_90 and later), with waits bounded in wall time.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rtd {

// Limit of every wait on a copy: a copy that has not landed after this long
// is treated as failed (the kernel records an error and returns).
constexpr unsigned long long ASYNC_WAIT_NS = 2000000000ull;

__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes barrier initialisation visible to the asynchronous proxy
__device__ inline void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this thread's earlier shared-memory accesses before later
// asynchronous-proxy writes to the same memory
__device__ inline void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One contiguous copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) that completes `bytes` transactions on `bar`.
__device__ inline void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// One bounded probe of the phase: the thread may be suspended until the
// phase completes or about 1 ms passes (suspend-time hint, in ns), so a
// waiting warp issues few instructions.
__device__ inline bool mbar_test(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity to complete; false if it
// did not within ASYNC_WAIT_NS.
__device__ inline bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > ASYNC_WAIT_NS) return false;
    }
    return true;
}

}  // namespace rtd
