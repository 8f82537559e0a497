// Grid-wide barrier with bounded waits for cooperative (co-resident) grids,
// shared by the persistent solver kernels.
#pragma once

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr long long kSpinLimit = 16000000;
struct GridSync {
    unsigned int* count;
    unsigned int* gen;
    int* err;
};

__device__ __forceinline__ unsigned int vload(const unsigned int* p) {
    return *(const volatile unsigned int*)p;
}
__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false (in every thread of the block) if a barrier timed out.  One
// thread per block (flat index 0, for 1-D and 2-D blocks alike) arrives; a
// waiting block gives up after kSpinLimit polls or kWaitNs of global time,
// whichever comes first, and records GS_TIMEOUT for every block to see.
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s
__device__ bool grid_sync(const GridSync& g) {
    __shared__ int s_ok;
    __syncthreads();
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
    if (leader) {
        int ok = 1;
        const unsigned int my_gen = vload(g.gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(g.count, 1u) + 1u;
        if (arrived == gridDim.x * gridDim.y * gridDim.z) {
            atomicExch(g.count, 0u);
            __threadfence();
            atomicAdd(g.gen, 1u);
        } else {
            long long spins = 0;
            const unsigned long long t0 = global_ns();
            while (vload(g.gen) == my_gen) {
                if (vload(g.err) != 0) {
                    ok = 0;
                    break;
                }
                if (++spins > kSpinLimit || global_ns() - t0 > kWaitNs) {
                    atomicExch(g.err, (int)GS_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (vload(g.err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace
}  // namespace gs
