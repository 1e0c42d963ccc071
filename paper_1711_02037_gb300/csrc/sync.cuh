// sync.cuh - grid-wide barrier with a bounded wait.
//
// Blocks of one persistent launch (all co-resident: the grid never exceeds
// SMs x occupancy) meet at a monotone arrival counter.  Thread 0 of each block
// publishes its writes (__threadfence), arrives (atomicAdd), and polls the
// counter with acquire loads until it reaches `target`.  The wait is bounded
// by `spin_limit` SM clock cycles and by the status word: on a timeout the
// block records RNMF_DEV_TIMEOUT and the whole block returns false, so a block
// that never arrives produces an error status instead of a hang.
#pragma once
#include "rnmf_internal.cuh"

__device__ __forceinline__ unsigned rnmf_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int rnmf_ld_volatile(const int* p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool rnmf_grid_barrier(unsigned* bar, unsigned target, int* status, long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int ok = 1;
        const long long t0 = clock64();
        while (rnmf_ld_acquire(bar) < target) {
            if (clock64() - t0 > spin_limit || rnmf_ld_volatile(status) != RNMF_DEV_OK) {
                atomicCAS(status, RNMF_DEV_OK, RNMF_DEV_TIMEOUT);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}
