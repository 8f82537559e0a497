// Grid-wide barrier with bounded waits for cooperative (co-resident) grids,
// shared by the persistent solver kernels.
#pragma once

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr long long kSpinLimit = 16000000;
struct GridSync {
    unsigned int* count;  // arrivals since the launch began
    unsigned int* gen;    // unused (kept zero)
    int* err;             // GS_TIMEOUT once any block gave up
    unsigned long long wait_ns;  // bound on one wait (0: kWaitNs)
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
// thread per block (flat index 0, for 1-D and 2-D blocks alike) arrives by a
// release add on a counter that only grows during a launch (zeroed by the
// host before it): the value it returns tells the block which barrier this
// is (no block can arrive at barrier k + 1 before every block has arrived at
// barrier k), so the block waits, with acquire loads, for the count of that
// barrier's last arrival.  A waiting block gives up after kSpinLimit polls or
// g.wait_ns of global time (the context's wait limit; kWaitNs if 0),
// whichever comes first, and records GS_TIMEOUT; a block that sees the error
// word set leaves as well.
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s
__device__ bool grid_sync(const GridSync& g) {
    __shared__ int s_ok;
    __syncthreads();
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
    if (leader) {
        int ok = 1;
        const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
        unsigned int old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(g.count) : "memory");
        const unsigned int target = (old / nb + 1u) * nb;
        const unsigned long long limit = g.wait_ns ? g.wait_ns : kWaitNs;
        long long spins = 0;
        const unsigned long long t0 = global_ns();
        for (;;) {
            unsigned int cur;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(g.count) : "memory");
            if ((int)(cur - target) >= 0) break;
            if ((spins & 63) == 63 && vload(g.err) != 0) {
                ok = 0;
                break;
            }
            if (++spins > kSpinLimit || global_ns() - t0 > limit) {
                atomicExch(g.err, (int)GS_TIMEOUT);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace
}  // namespace gs
