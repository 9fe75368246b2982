// Bulk asynchronous copies (cp.async.bulk, the Tensor Memory Accelerator's
// untiled form) from global to shared memory with completion on an mbarrier,
// and the mbarrier operations around them (device code only).  Every copy
// wants 16-byte aligned addresses and a size that is a multiple of 16 bytes;
// callers arrange their layouts for it.
#pragma once

#include <cuda_runtime.h>

namespace gnk {

static __device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// An mbarrier expecting `count` arrivals per phase; fenced so that the copy
// engine sees the initialised barrier.  Callers synchronise the block after.
static __device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of copies completing on this phase.
static __device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

static __device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared memory
static __device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                                 unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// bulk_load of data read once (a stream larger than L2): the L2 lines it brings
// in are marked evict-first, so that the stream does not push out data that is
// reused.
static __device__ __forceinline__ void bulk_load_stream(void* dst, const void* src, unsigned bytes,
                                                        unsigned long long* bar) {
    unsigned long long policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// True once the phase of parity `parity` has completed.
static __device__ __forceinline__ bool mbar_done(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for that phase with at most `limit` polls; false when it gave up.
static __device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit) {
    for (int it = 0; !mbar_done(bar, parity); ++it)
        if (it >= limit) return false;
    return true;
}

}  // namespace gnk
