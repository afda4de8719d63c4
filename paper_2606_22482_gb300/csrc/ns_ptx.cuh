// ns_ptx.cuh -- asynchronous-copy PTX wrappers shared by the execute paths.
#pragma once
#include "ns_internal.cuh"

namespace ns {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <bool HINT>
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid, uint64_t pol)
{
    const uint32_t d = smem_u32(dst);
    const int n = valid ? 16 : 0;  // 0: fill the 16 bytes with zeros, read nothing
    if (HINT)
        asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;"
                     :: "r"(d), "l"(src), "r"(n), "l"(pol) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

}  // namespace ns
