// Asynchronous global -> shared copies (cp.async): the copy is in flight
// without holding a register, so a thread can have many outstanding at once.
#pragma once

namespace glls {

// One value of 4 or 8 bytes; both addresses aligned to its size.
template <typename T>
__device__ __forceinline__ void cp_async(T* sdst, const T* gsrc) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte values");
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}

// Waits for every copy this thread has issued (others' copies need a barrier
// after their own waits).
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace glls
