// wilson_apply_noalloc: y = D x on the full lattice for callers that cannot
// allocate device memory.  It runs the same stencil kernel as wilson_apply;
// the two tables that kernel reads besides its inputs and outputs -- the
// neighbour table and the packed (-1/2 U) links -- live in one file-scope
// device array instead of context-owned allocations.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int64_t kNoAllocMaxSites = 8192;
constexpr size_t kNbrBytes = (size_t)kNoAllocMaxSites * 4 * sizeof(int2);        // 256 KiB
constexpr size_t kLinkBytes = (size_t)kNoAllocMaxSites * 36 * sizeof(double2);   // 4.5 MiB
constexpr size_t kScratchBytes = kNbrBytes + kLinkBytes;

// Held by every GPU that loads the library, until the process exits.  In host
// code this name is only a host-side stand-in: the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array in the current device's context.  The
// first call on a device loads the library's module there (the set-up, which
// is why that first call must come before any stream capture); after that the
// lookup is a cheap query.  It is made on every call, so a device that was
// reset, or a primary context destroyed and created again (the module then
// reloads, possibly at another address), never sees a stale pointer.
gs_status scratch_address(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return GS_ECUDA;
    }
    *out = p;
    return GS_OK;
}

struct Dims4 {
    int L[4];
};

// Site-order neighbour table and -1/2 U, written over the whole table each call.
__global__ void k_site_tables(Dims4 d, int64_t V, const double2* __restrict__ U,
                              int2* __restrict__ nbr, double2* __restrict__ links) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V;
         s += (int64_t)gridDim.x * blockDim.x) {
        int x[4];
        int64_t t = s;
        for (int mu = 0; mu < 4; ++mu) {
            x[mu] = (int)(t % d.L[mu]);
            t /= d.L[mu];
        }
        int64_t stride = 1;
        for (int mu = 0; mu < 4; ++mu) {
            const int64_t fwd = s + ((x[mu] + 1 == d.L[mu]) ? -(int64_t)(d.L[mu] - 1) : 1) * stride;
            const int64_t bwd = s + ((x[mu] == 0) ? (int64_t)(d.L[mu] - 1) : -1) * stride;
            nbr[s * 4 + mu] = make_int2((int)fwd, (int)bwd);
            stride *= d.L[mu];
        }
        for (int k = 0; k < 36; ++k) {
            const double2 u = U[s * 36 + k];
            links[s * 36 + k] = make_double2(-0.5 * u.x, -0.5 * u.y);
        }
    }
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status wilson_apply_noalloc(const int dims[4], double m0, const void* U_dev,
                                          const void* x_dev, void* y_dev, void* stream) {
    if (!dims || !U_dev || !x_dev || !y_dev || !isfinite(m0)) return GS_EINVAL;
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] < 2) return GS_EINVAL;
    // every factor is checked against the bound before it multiplies V, so the
    // product never overflows whatever the extents
    int64_t V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] > kNoAllocMaxSites / V) return GS_ETOOLARGE;
        V *= dims[mu];
    }
    void* base = nullptr;
    gs_status s = scratch_address(&base);
    if (s != GS_OK) return s;
    int2* nbr = (int2*)base;
    double2* links = (double2*)((unsigned char*)base + kNbrBytes);
    cudaStream_t st = (cudaStream_t)stream;
    Dims4 d;
    for (int mu = 0; mu < 4; ++mu) d.L[mu] = dims[mu];
    k_site_tables<<<(int)((V + 127) / 128), 128, 0, st>>>(d, V, (const double2*)U_dev, nbr, links);
    if (cudaGetLastError() != cudaSuccess) return GS_ECUDA;
    StencilArgs a;
    memset(&a, 0, sizeof a);
    a.out = (double2*)y_dev;
    a.o0 = 0;
    a.n_out = V;
    a.inA = (const double2*)x_dev;
    a.a0 = 0;
    a.a1 = V;
    a.b1 = V;
    a.diag = m0 + 4.0;
    a.nbr = nbr;
    a.links = links;
    return launch_stencil_f64_on(a, st);
}
