// lat_async.cuh -- per-thread asynchronous global->shared copies (cp.async)
// and small index helpers shared by the plane-ring step kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lat {

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// 16-byte copy that bypasses L1 (cg); both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
// 4- or 8-byte copy through L1 (ca); both addresses aligned to the size
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem)
{
    static_assert(BYTES == 4 || BYTES == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem), "n"(BYTES)
                 : "memory");
}
// v, or the shared-memory value at a where p holds: a predicated load, no branch
__device__ __forceinline__ float ld_shared_if(bool p, const float* a, float v)
{
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.shared.f32 %0, [%1];\n\t}"
        : "+f"(v)
        : "r"((uint32_t)__cvta_generic_to_shared(a)), "r"((int)p));
    return v;
}
__device__ __forceinline__ double ld_shared_if(bool p, const double* a, double v)
{
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.shared.f64 %0, [%1];\n\t}"
        : "+d"(v)
        : "r"((uint32_t)__cvta_generic_to_shared(a)), "r"((int)p));
    return v;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most `pending` of the most recent groups are still in flight
__device__ __forceinline__ void cp_async_wait(int pending)
{
    switch (pending) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    }
}

} // namespace lat
