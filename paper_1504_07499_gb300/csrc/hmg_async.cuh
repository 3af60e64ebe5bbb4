// Asynchronous bulk copies global -> shared memory (the Hopper/Blackwell bulk-copy
// engine) completed through a shared-memory mbarrier, with a bounded wait.
//
// One thread arms the barrier with the byte count it expects and issues the copies;
// every consumer waits for the barrier's phase to complete.  A wait gives up after a
// fixed number of polls (far longer than any copy takes), so a kernel never spins
// without end: the caller then records the failure and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hmg {
namespace async {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Initialize a barrier that completes a phase after one arrival and its expected bytes.
__device__ __forceinline__ void mbar_init(uint32_t mb) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    // make the initialized barrier visible to the bulk-copy engine (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive once and expect `bytes` more from bulk copies in this phase.
__device__ __forceinline__ void mbar_expect(uint32_t mb, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mb),
        "r"(bytes)
        : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from global
// memory to this CTA's shared memory, completing on barrier mb.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mb) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mb)
        : "memory");
}

// Tiled 4D tensor copy (the tensor map describes the global array and the box) to this
// CTA's shared memory at dst, completing on barrier mb.  x is the innermost coordinate.
__device__ __forceinline__ void tensor_g2s_4d(uint32_t dst, const void* map, int x, int y, int z, int w, uint32_t mb) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(mb)
        : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mb, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}

// Polls before a wait gives up: each try_wait suspends for up to a hardware-defined
// time slice, so this bounds a wait to seconds, orders of magnitude above a copy.
constexpr long long kWaitPolls = 1ll << 24;

// Wait for the phase of the given parity to complete; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity) {
    for (long long i = 0; i < kWaitPolls; ++i)
        if (mbar_try(mb, parity)) return true;
    return false;
}

}  // namespace async
}  // namespace hmg
