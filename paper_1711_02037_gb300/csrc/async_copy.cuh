// async_copy.cuh - global -> shared copies that do not stall the issuing thread.
//
// A loop of "load global, store shared" waits for every load before it can issue
// the next one; cp.async moves the data without a register round trip, so all of
// a thread's copies are in flight at once.  Out-of-range elements are written as
// zeros (source size 0: nothing is read from `src`).
#pragma once
#include <stdint.h>

__device__ __forceinline__ uint32_t ac_smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(ac_smem_u32(smem_dst)), "l"(gmem_src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(ac_smem_u32(smem_dst)), "l"(gmem_src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// 16-byte copy of which only the first `bytes` (0, 4, 8, 12 or 16) are read; the
// rest of the 16 destination bytes are written as zeros.
__device__ __forceinline__ void cp_async16_n(void* smem_dst, const void* gmem_src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(ac_smem_u32(smem_dst)), "l"(gmem_src),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most one committed group is still in flight.
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
