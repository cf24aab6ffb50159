// Bounded grid-wide barrier for cooperative launches (every block resident).
#pragma once

#include <cuda_runtime.h>

// Generation barrier: each block's thread 0 reads the generation word, arrives on the
// counter with one acquire-release atomic; the last arrival resets the counter and
// publishes the next generation with a release store; the others poll the generation with
// acquire loads.  The wait is bounded: `limit` counts units of 64 ns of the global timer
// (200,000 ~ 13 ms, 20,000,000 ~ 1.3 s); a block whose wait runs out records a timeout in
// *err, and every block leaves the kernel at its next barrier.
struct GridBar {
    unsigned int count;      // arrivals, with the error flag on one 128-byte line
    int err;
    int pad0[30];
    unsigned int gen;        // the polled generation word on a line of its own
    int pad1[31];
};

__device__ __forceinline__ unsigned int gb_ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int gb_arrive(unsigned int *p) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

__device__ __forceinline__ void gb_st_release(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long gb_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool grid_barrier(GridBar *bar, unsigned int nblocks, long long limit) {
    __shared__ int s_ok;     // one outcome per block, read by all of its threads
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int g = gb_ld_acquire(&bar->gen);
        const unsigned int arrived = gb_arrive(&bar->count);
        if (arrived == nblocks - 1) {
            bar->count = 0u;                       // ordered before the release below
            gb_st_release(&bar->gen, g + 1u);
        } else {
            const unsigned long long deadline = gb_clock_ns() + 64ull * (unsigned long long)limit;
            unsigned int polls = 0;
            while (gb_ld_acquire(&bar->gen) == g) {
                if ((++polls & 63u) == 0u) {
                    if (gb_clock_ns() > deadline || *(volatile int *)&bar->err) {
                        atomicExch(&bar->err, 1);
                        break;
                    }
                }
            }
        }
        s_ok = *(volatile int *)&bar->err == 0;
    }
    __syncthreads();
    return s_ok != 0;
}
