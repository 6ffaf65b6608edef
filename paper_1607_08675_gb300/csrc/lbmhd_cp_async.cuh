// lbmhd_cp_async.cuh -- per-thread asynchronous copies into shared memory.
//
// One 4- or 8-byte cp.async (the L1-allocating form, the one that takes
// sizes below 16 bytes) or a 16-byte one, the commit, and a wait until at
// most N of the thread's most recent groups are pending.  A thread's
// wait_group covers its own copies; values another thread copied need a
// barrier after the waits (and a slot is refilled only after a barrier
// that follows its last read).
#pragma once

namespace lbmhd {

template <int B>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
    static_assert(B == 4 || B == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B)
                 : "memory");
}
// 16 bytes, cached in L2 only (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace lbmhd
