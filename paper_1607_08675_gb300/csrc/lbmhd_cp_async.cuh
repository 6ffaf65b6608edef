// lbmhd_cp_async.cuh -- per-thread asynchronous copies into shared memory.
//
// One 4- or 8-byte cp.async (the L1-allocating form, the one that takes
// sizes below 16 bytes), its commit, and a wait until at most N of the
// thread's most recent groups are pending.  The kernels that use these read
// back only the values the same thread copied, so the thread's own
// wait_group is all the synchronisation a slot needs; a slot is reused only
// after its values have been read into registers (program order).
#pragma once

namespace lbmhd {

template <int B>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
    static_assert(B == 4 || B == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace lbmhd
