// Bounded grid-wide barrier for cooperative launches (every block resident).
#pragma once

#include <cuda_runtime.h>

// The spin on the generation word is bounded: after `limit` polls the block records a
// timeout in *err and every block leaves the kernel at its next barrier.
struct GridBar {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

__device__ __forceinline__ bool grid_barrier(GridBar *bar, unsigned int nblocks, long long limit) {
    __shared__ int s_ok;     // one verdict per block, read by all of its threads
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &bar->gen;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == g) {
                if (++it > limit || *(volatile int *)&bar->err) {
                    atomicExch(&bar->err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = *(volatile int *)&bar->err == 0;
    }
    __syncthreads();
    return s_ok != 0;
}
