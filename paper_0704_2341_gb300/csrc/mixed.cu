// Mixed-precision inner solve of D_rr z = t.
//
// FP64 defect correction around a low-precision BiCGStab:
//   z = 0, r = t;  repeat { solve D_rr e = r / ||r|| approximately in FP32
//   arithmetic with FP32 or BF16 storage;  z += ||r|| e;  r = t - D_rr z in
//   FP64 }  until ||r|| <= tol ||t||.
// The true residual is recomputed with the FP64 stencil every cycle, so the
// result meets the same FP64 tolerance as the plain solve; the low-precision
// solve only has to reduce the residual by a few digits per cycle.  If a
// cycle stops making progress, the remaining correction is computed by the
// plain FP64 BiCGStab (the fallback and the judge of the result).
//
// Low-precision layouts (compact rest-set index k = label - n_b):
//   spinors: SoA of 16-byte vectors, component-major: FP32 -> 6 float4 per
//            site ([6][n]), BF16 -> 3 x (8 bf16) per site ([3][n]);
//   links:   two rows of -1/2 U (12 reals), the third row rebuilt as
//            -2 conj(row0 x row1) (SU(3)); FP32 -> 3 float4 ([mu][3][n]),
//            BF16 -> 3 x (4 bf16) ([mu][3][n]);
//   neighbours: int2 [n][mu] compact indices, -1 for a neighbour outside r.
// One thread per site accumulates all eight hops in FP32 registers; the
// kernel is HBM bound (384 B/site FP32, 192 B/site BF16 algorithmic).
#include <cuda_bf16.h>
#include <math.h>

#include "gs_internal.cuh"

namespace gs {

struct LpState;

namespace {

constexpr int kLpRed = 256;  // block size of the low-precision BLAS kernels

// ---------------------------------------------------------------------------
// storage traits
// ---------------------------------------------------------------------------
template <class S>
struct Store;

template <>
struct Store<float> {
    static constexpr int kSpinVec = 6;  // float4 per spinor
    static constexpr int kLinkVec = 3;  // float4 per 12-real link
    using SV = float4;
    using LV = float4;
    __device__ __forceinline__ static void load_spinor(const void* base, int64_t n, int64_t k,
                                                       float (&f)[24]) {
        const float4* b = (const float4*)base;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float4 v = __ldg(b + c * n + k);
            f[4 * c + 0] = v.x;
            f[4 * c + 1] = v.y;
            f[4 * c + 2] = v.z;
            f[4 * c + 3] = v.w;
        }
    }
    __device__ __forceinline__ static void store_spinor(void* base, int64_t n, int64_t k,
                                                        const float (&f)[24]) {
        float4* b = (float4*)base;
#pragma unroll
        for (int c = 0; c < 6; ++c)
            b[c * n + k] = make_float4(f[4 * c + 0], f[4 * c + 1], f[4 * c + 2], f[4 * c + 3]);
    }
    __device__ __forceinline__ static void load_link(const void* base, int64_t n, int mu,
                                                     int64_t k, float (&f)[12]) {
        const float4* b = (const float4*)base + (int64_t)mu * 3 * n;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 v = __ldg(b + c * n + k);
            f[4 * c + 0] = v.x;
            f[4 * c + 1] = v.y;
            f[4 * c + 2] = v.z;
            f[4 * c + 3] = v.w;
        }
    }
    __device__ __forceinline__ static void store_link(void* base, int64_t n, int mu, int64_t k,
                                                      const float (&f)[12]) {
        float4* b = (float4*)base + (int64_t)mu * 3 * n;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            b[c * n + k] = make_float4(f[4 * c + 0], f[4 * c + 1], f[4 * c + 2], f[4 * c + 3]);
    }
    static constexpr size_t spinor_bytes = 96;
    static constexpr size_t link_bytes = 48;
};

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_bf2(uint32_t u) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(h);
}

template <>
struct Store<__nv_bfloat16> {
    static constexpr int kSpinVec = 3;  // uint4 (8 bf16) per spinor component group
    static constexpr int kLinkVec = 3;  // uint2 (4 bf16)
    __device__ __forceinline__ static void load_spinor(const void* base, int64_t n, int64_t k,
                                                       float (&f)[24]) {
        const uint4* b = (const uint4*)base;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint4 v = __ldg(b + c * n + k);
            float2 t;
            t = unpack_bf2(v.x); f[8 * c + 0] = t.x; f[8 * c + 1] = t.y;
            t = unpack_bf2(v.y); f[8 * c + 2] = t.x; f[8 * c + 3] = t.y;
            t = unpack_bf2(v.z); f[8 * c + 4] = t.x; f[8 * c + 5] = t.y;
            t = unpack_bf2(v.w); f[8 * c + 6] = t.x; f[8 * c + 7] = t.y;
        }
    }
    __device__ __forceinline__ static void store_spinor(void* base, int64_t n, int64_t k,
                                                        const float (&f)[24]) {
        uint4* b = (uint4*)base;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            b[c * n + k] = make_uint4(pack_bf2(f[8 * c + 0], f[8 * c + 1]),
                                      pack_bf2(f[8 * c + 2], f[8 * c + 3]),
                                      pack_bf2(f[8 * c + 4], f[8 * c + 5]),
                                      pack_bf2(f[8 * c + 6], f[8 * c + 7]));
    }
    __device__ __forceinline__ static void load_link(const void* base, int64_t n, int mu,
                                                     int64_t k, float (&f)[12]) {
        const uint2* b = (const uint2*)base + (int64_t)mu * 3 * n;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint2 v = __ldg(b + c * n + k);
            float2 t;
            t = unpack_bf2(v.x); f[4 * c + 0] = t.x; f[4 * c + 1] = t.y;
            t = unpack_bf2(v.y); f[4 * c + 2] = t.x; f[4 * c + 3] = t.y;
        }
    }
    __device__ __forceinline__ static void store_link(void* base, int64_t n, int mu, int64_t k,
                                                      const float (&f)[12]) {
        uint2* b = (uint2*)base + (int64_t)mu * 3 * n;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            b[c * n + k] = make_uint2(pack_bf2(f[4 * c + 0], f[4 * c + 1]),
                                      pack_bf2(f[4 * c + 2], f[4 * c + 3]));
    }
    static constexpr size_t spinor_bytes = 48;
    static constexpr size_t link_bytes = 24;
};

// ---------------------------------------------------------------------------
// FP32 complex helpers on (re, im) pairs held in float arrays
// ---------------------------------------------------------------------------
struct cf {
    float x, y;
};
__device__ __forceinline__ cf mk(float a, float b) { return cf{a, b}; }
__device__ __forceinline__ cf operator+(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cf operator-(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cf muli(cf a) { return cf{-a.y, a.x}; }
__device__ __forceinline__ cf mulmi(cf a) { return cf{a.y, -a.x}; }
__device__ __forceinline__ cf cneg(cf a) { return cf{-a.x, -a.y}; }
__device__ __forceinline__ cf conjf_(cf a) { return cf{a.x, -a.y}; }
__device__ __forceinline__ cf cmul(cf a, cf b) {
    return cf{fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)};
}
__device__ __forceinline__ void cfma_(cf& acc, cf a, cf b) {  // acc += a b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void ccfma_(cf& acc, cf a, cf b) {  // acc += conj(a) b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}

__device__ __forceinline__ cf get(const float (&f)[24], int spin, int col) {
    return cf{f[2 * (3 * spin + col)], f[2 * (3 * spin + col) + 1]};
}

// h = psi_up -+ X_mu psi_lo (the DeGrand-Rossi projection, as in the FP64 kernel)
template <int MU, bool FWD>
__device__ __forceinline__ void project(const float (&p)[24], cf (&h)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cf s0 = get(p, 0, c), s1 = get(p, 1, c), s2 = get(p, 2, c), s3 = get(p, 3, c);
        if (MU == 0) {  // X psi_lo = (i s3, i s2)
            h[0][c] = FWD ? s0 - muli(s3) : s0 + muli(s3);
            h[1][c] = FWD ? s1 - muli(s2) : s1 + muli(s2);
        } else if (MU == 1) {  // (-s3, s2)
            h[0][c] = FWD ? s0 + s3 : s0 - s3;
            h[1][c] = FWD ? s1 - s2 : s1 + s2;
        } else if (MU == 2) {  // (i s2, -i s3)
            h[0][c] = FWD ? s0 - muli(s2) : s0 + muli(s2);
            h[1][c] = FWD ? s1 + muli(s3) : s1 - muli(s3);
        } else {  // (s2, s3)
            h[0][c] = FWD ? s0 - s2 : s0 + s2;
            h[1][c] = FWD ? s1 - s3 : s1 + s3;
        }
    }
}

// acc (24 floats) += [g ; sign X_mu^dag g]
template <int MU, int SIGN>
__device__ __forceinline__ void accumulate(float (&acc)[24], const cf (&g)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[2 * (0 + c)] += g[0][c].x;
        acc[2 * (0 + c) + 1] += g[0][c].y;
        acc[2 * (3 + c)] += g[1][c].x;
        acc[2 * (3 + c) + 1] += g[1][c].y;
        cf l0, l1;
        if (MU == 0) {  // X^dag = [[0,-i],[-i,0]]
            l0 = mulmi(g[1][c]);
            l1 = mulmi(g[0][c]);
        } else if (MU == 1) {  // [[0,1],[-1,0]]
            l0 = g[1][c];
            l1 = cneg(g[0][c]);
        } else if (MU == 2) {  // diag(-i, i)
            l0 = mulmi(g[0][c]);
            l1 = muli(g[1][c]);
        } else {
            l0 = g[0][c];
            l1 = g[1][c];
        }
        if (SIGN > 0) {
            acc[2 * (6 + c)] += l0.x;
            acc[2 * (6 + c) + 1] += l0.y;
            acc[2 * (9 + c)] += l1.x;
            acc[2 * (9 + c) + 1] += l1.y;
        } else {
            acc[2 * (6 + c)] -= l0.x;
            acc[2 * (6 + c) + 1] -= l0.y;
            acc[2 * (9 + c)] -= l1.x;
            acc[2 * (9 + c) + 1] -= l1.y;
        }
    }
}

// rows 0, 1 of -1/2 U from 12 reals; row 2 = -2 conj(row0 x row1)
__device__ __forceinline__ void rebuild(const float (&f)[12], cf (&u)[3][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        u[0][c] = cf{f[2 * c], f[2 * c + 1]};
        u[1][c] = cf{f[6 + 2 * c], f[6 + 2 * c + 1]};
    }
    const cf x0 = cmul(u[0][1], u[1][2]) - cmul(u[0][2], u[1][1]);
    const cf x1 = cmul(u[0][2], u[1][0]) - cmul(u[0][0], u[1][2]);
    const cf x2 = cmul(u[0][0], u[1][1]) - cmul(u[0][1], u[1][0]);
    u[2][0] = cf{-2.f * x0.x, 2.f * x0.y};
    u[2][1] = cf{-2.f * x1.x, 2.f * x1.y};
    u[2][2] = cf{-2.f * x2.x, 2.f * x2.y};
}

struct LpArgs {
    void* out;
    const void* in;
    const void* links;
    const int2* nbr;     // [n][4]
    int64_t n;           // rest-set sites
    float diag;          // m0 + 4
    int epi;
    const void* epi_vec;
    LpState* st;
    float* partial;
    unsigned int* counter;
    int* ran;
};

}  // namespace

// Device state of the low-precision BiCGStab (FP32 scalars).
struct LpState {
    float2 rho, alpha, omega, beta;
    float rr, bb, tol2;
    int done, status, iter, pad;
    BicgPublic* pub;
};

namespace {

__device__ __forceinline__ void lp_publish(LpState* st) {
    BicgPublic* p = st->pub;
    if (p) {
        p->rr = st->rr;
        p->bb = st->bb;
        p->iter = st->iter;
        p->status = st->status;
        __threadfence_system();
        p->done = st->done;
        __threadfence_system();
    }
}

// FP32 block reduction; the last block gets the totals in thread 0.
template <int NV>
__device__ bool lp_reduce_last(float (&v)[NV], float* partial, unsigned int* counter,
                               float (&tot)[NV]) {
    __shared__ float sm[32][NV];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        float x = v[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) sm[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float x = 0.f;
            for (int w = 0; w < nw; ++w) x += sm[w][q];
            partial[(int64_t)blockIdx.x * kMaxRedVals + q] = x;
        }
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    float s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = 0.f;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile float* p = partial + (int64_t)b * kMaxRedVals;
#pragma unroll
        for (int q = 0; q < NV; ++q) s[q] += p[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        float x = s[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) sm[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float x = 0.f;
            for (int w = 0; w < nw; ++w) x += sm[w][q];
            tot[q] = x;
        }
        *counter = 0u;
    }
    return true;
}

__device__ __forceinline__ float2 cdivf_(float2 a, float2 b) {
    const float inv = 1.0f / (b.x * b.x + b.y * b.y);
    return make_float2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ float2 cmulf2(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------------------
// the low-precision stencil: a block of 4 warps covers 32 sites, warp w owns
// direction mu = w (forward and backward hop) for all 32 sites.  All loads of
// a warp's two hops are issued before any is used (out-of-set neighbours read
// a valid dummy site and are masked afterwards), so each thread waits for
// memory about twice instead of once per hop; the four 24-float partial
// results meet in shared memory and are summed per 16-byte output group.
// ---------------------------------------------------------------------------
constexpr int kLpSites = 32;
constexpr int kLpThreads = 128;

template <class S, int MU>
__device__ __forceinline__ void lp_dir(const LpArgs& a, int64_t k, bool valid, float (&acc)[24]) {
#pragma unroll
    for (int q = 0; q < 24; ++q) acc[q] = 0.f;
    const int2 nb = valid ? __ldg(a.nbr + k * 4 + MU) : make_int2(-1, -1);
    const bool hf = nb.x >= 0, hb = nb.y >= 0;
    const int64_t jf = hf ? nb.x : 0, jb = hb ? nb.y : 0, jk = valid ? k : 0;
    float pf[24], pb[24], lf[12], lb[12];
    Store<S>::load_spinor(a.in, a.n, jf, pf);
    Store<S>::load_spinor(a.in, a.n, jb, pb);
    Store<S>::load_link(a.links, a.n, MU, jk, lf);
    Store<S>::load_link(a.links, a.n, MU, jb, lb);
    if (hf) {
        cf h[2][3], u[3][3], g[2][3];
        project<MU, true>(pf, h);
        rebuild(lf, u);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cf t = cmul(u[r][0], h[s][0]);
                cfma_(t, u[r][1], h[s][1]);
                cfma_(t, u[r][2], h[s][2]);
                g[s][r] = t;
            }
        accumulate<MU, -1>(acc, g);
    }
    if (hb) {
        cf h[2][3], u[3][3], g[2][3];
        project<MU, false>(pb, h);
        rebuild(lb, u);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cf t = cf{0.f, 0.f};
                ccfma_(t, u[0][r], h[s][0]);
                ccfma_(t, u[1][r], h[s][1]);
                ccfma_(t, u[2][r], h[s][2]);
                g[s][r] = t;
            }
        accumulate<MU, +1>(acc, g);
    }
}

// Variant "site": one thread per site, all eight hops in registers.  The
// neighbour indices of all four directions are loaded first; each direction's
// two spinors and two links are then loaded together (out-of-set neighbours
// read a valid dummy site and are masked), so a thread waits for memory about
// five times per site instead of sixteen.
template <class S, int MU>
__device__ __forceinline__ void site_dir(const LpArgs& a, int64_t k, int2 nb, float (&acc)[24]) {
    const bool hf = nb.x >= 0, hb = nb.y >= 0;
    const int64_t jf = hf ? nb.x : k, jb = hb ? nb.y : k;
    float pf[24], pb[24], lf[12], lb[12];
    Store<S>::load_spinor(a.in, a.n, jf, pf);
    Store<S>::load_spinor(a.in, a.n, jb, pb);
    Store<S>::load_link(a.links, a.n, MU, k, lf);
    Store<S>::load_link(a.links, a.n, MU, jb, lb);
    if (hf) {
        cf h[2][3], u[3][3], g[2][3];
        project<MU, true>(pf, h);
        rebuild(lf, u);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cf t = cmul(u[r][0], h[s][0]);
                cfma_(t, u[r][1], h[s][1]);
                cfma_(t, u[r][2], h[s][2]);
                g[s][r] = t;
            }
        accumulate<MU, -1>(acc, g);
    }
    if (hb) {
        cf h[2][3], u[3][3], g[2][3];
        project<MU, false>(pb, h);
        rebuild(lb, u);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cf t = cf{0.f, 0.f};
                ccfma_(t, u[0][r], h[s][0]);
                ccfma_(t, u[1][r], h[s][1]);
                ccfma_(t, u[2][r], h[s][2]);
                g[s][r] = t;
            }
        accumulate<MU, +1>(acc, g);
    }
}

template <class S, int EPI>
__device__ __forceinline__ void lp_finish(const LpArgs& a, LpState* st, float (&tot)[3]);

template <class S, int EPI, int MINB>
__global__ void __launch_bounds__(128, MINB) k_dslash_lp_site(LpArgs a) {
    const bool skip = a.st != nullptr && a.st->done;
    if (a.ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.ran = skip ? 0 : 1;
    if (skip) return;
    float e[3] = {0.f, 0.f, 0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int4 n01 = __ldg((const int4*)(a.nbr + k * 4));
        const int4 n23 = __ldg((const int4*)(a.nbr + k * 4) + 1);
        float acc[24];
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[q] = 0.f;
        site_dir<S, 0>(a, k, make_int2(n01.x, n01.y), acc);
        site_dir<S, 1>(a, k, make_int2(n01.z, n01.w), acc);
        site_dir<S, 2>(a, k, make_int2(n23.x, n23.y), acc);
        site_dir<S, 3>(a, k, make_int2(n23.z, n23.w), acc);
        float self[24];
        Store<S>::load_spinor(a.in, a.n, k, self);
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[q] = fmaf(a.diag, self[q], acc[q]);
        Store<S>::store_spinor(a.out, a.n, k, acc);
        if (EPI == EPI_DOT_RHAT_V) {
            float rv[24];
            Store<S>::load_spinor(a.epi_vec, a.n, k, rv);
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                e[0] = fmaf(rv[2 * q], acc[2 * q], fmaf(rv[2 * q + 1], acc[2 * q + 1], e[0]));
                e[1] = fmaf(rv[2 * q], acc[2 * q + 1], fmaf(-rv[2 * q + 1], acc[2 * q], e[1]));
            }
        } else if (EPI == EPI_DOT_TS) {
            float sv[24];
            Store<S>::load_spinor(a.epi_vec, a.n, k, sv);
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                const float tr = acc[2 * q], ti = acc[2 * q + 1];
                e[0] = fmaf(tr, sv[2 * q], fmaf(ti, sv[2 * q + 1], e[0]));
                e[1] = fmaf(tr, sv[2 * q + 1], fmaf(-ti, sv[2 * q], e[1]));
                e[2] = fmaf(tr, tr, fmaf(ti, ti, e[2]));
            }
        }
    }
    if constexpr (EPI != EPI_NONE) {
        float tot[3];
        if (lp_reduce_last<3>(e, a.partial, a.counter, tot) && threadIdx.x == 0)
            lp_finish<S, EPI>(a, a.st, tot);
    }
}

// One 16-byte output group (4 reals for FP32, 8 for BF16) of site k.
template <class S>
struct Group;
template <>
struct Group<float> {
    static constexpr int kReals = 4, kGroups = 6;
    __device__ __forceinline__ static void load(const void* b, int64_t n, int g, int64_t k,
                                                float (&f)[8]) {
        const float4 v = __ldg((const float4*)b + g * n + k);
        f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
    }
    __device__ __forceinline__ static void store(void* b, int64_t n, int g, int64_t k,
                                                 const float (&f)[8]) {
        ((float4*)b)[g * n + k] = make_float4(f[0], f[1], f[2], f[3]);
    }
};
template <>
struct Group<__nv_bfloat16> {
    static constexpr int kReals = 8, kGroups = 3;
    __device__ __forceinline__ static void load(const void* b, int64_t n, int g, int64_t k,
                                                float (&f)[8]) {
        const uint4 v = __ldg((const uint4*)b + g * n + k);
        float2 t;
        t = unpack_bf2(v.x); f[0] = t.x; f[1] = t.y;
        t = unpack_bf2(v.y); f[2] = t.x; f[3] = t.y;
        t = unpack_bf2(v.z); f[4] = t.x; f[5] = t.y;
        t = unpack_bf2(v.w); f[6] = t.x; f[7] = t.y;
    }
    __device__ __forceinline__ static void store(void* b, int64_t n, int g, int64_t k,
                                                 const float (&f)[8]) {
        ((uint4*)b)[g * n + k] = make_uint4(pack_bf2(f[0], f[1]), pack_bf2(f[2], f[3]),
                                            pack_bf2(f[4], f[5]), pack_bf2(f[6], f[7]));
    }
};

template <class S, int EPI>
__global__ void __launch_bounds__(kLpThreads) k_dslash_lp_dir(LpArgs a) {
    const bool skip = a.st != nullptr && a.st->done;
    if (a.ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.ran = skip ? 0 : 1;
    if (skip) return;
    __shared__ float red[4][24][kLpSites];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float e[3] = {0.f, 0.f, 0.f};
    constexpr int R = Group<S>::kReals, G = Group<S>::kGroups;
    for (int64_t base = (int64_t)blockIdx.x * kLpSites; base < a.n;
         base += (int64_t)gridDim.x * kLpSites) {
        const int64_t k = base + lane;
        const bool valid = k < a.n;
        {
            float acc[24];
            switch (warp) {
                case 0: lp_dir<S, 0>(a, k, valid, acc); break;
                case 1: lp_dir<S, 1>(a, k, valid, acc); break;
                case 2: lp_dir<S, 2>(a, k, valid, acc); break;
                default: lp_dir<S, 3>(a, k, valid, acc); break;
            }
#pragma unroll
            for (int q = 0; q < 24; ++q) red[warp][q][lane] = acc[q];
        }
        __syncthreads();
        if (valid) {
            for (int g = warp; g < G; g += 4) {
                float self[8], out[8];
                Group<S>::load(a.in, a.n, g, k, self);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const int q = g * R + j;
                    out[j] = fmaf(a.diag, self[j],
                                  (red[0][q][lane] + red[1][q][lane]) + (red[2][q][lane] + red[3][q][lane]));
                }
                Group<S>::store(a.out, a.n, g, k, out);
                if (EPI == EPI_DOT_RHAT_V) {  // <rhat, v>
                    float rv[8];
                    Group<S>::load(a.epi_vec, a.n, g, k, rv);
#pragma unroll
                    for (int j = 0; j < R; j += 2) {
                        e[0] = fmaf(rv[j], out[j], fmaf(rv[j + 1], out[j + 1], e[0]));
                        e[1] = fmaf(rv[j], out[j + 1], fmaf(-rv[j + 1], out[j], e[1]));
                    }
                } else if (EPI == EPI_DOT_TS) {  // <t, s>, <t, t>
                    float sv[8];
                    Group<S>::load(a.epi_vec, a.n, g, k, sv);
#pragma unroll
                    for (int j = 0; j < R; j += 2) {
                        const float tr = out[j], ti = out[j + 1];
                        e[0] = fmaf(tr, sv[j], fmaf(ti, sv[j + 1], e[0]));
                        e[1] = fmaf(tr, sv[j + 1], fmaf(-ti, sv[j], e[1]));
                        e[2] = fmaf(tr, tr, fmaf(ti, ti, e[2]));
                    }
                }
            }
        }
        __syncthreads();
    }
    if constexpr (EPI == EPI_NONE) {
        return;
    } else {
        float tot[3];
        if (lp_reduce_last<3>(e, a.partial, a.counter, tot) && threadIdx.x == 0)
            lp_finish<S, EPI>(a, a.st, tot);
    }
}

// alpha = rho / <rhat, v>  or  omega = <t, s> / <t, t>, in the last block
template <class S, int EPI>
__device__ __forceinline__ void lp_finish(const LpArgs& a, LpState* st, float (&tot)[3]) {
    if (EPI == EPI_DOT_RHAT_V) {
        const float2 den = make_float2(tot[0], tot[1]);
        if (den.x == 0.f && den.y == 0.f) {
            st->status = GS_BREAKDOWN;
            st->done = 1;
        } else {
            st->alpha = cdivf_(st->rho, den);
            if (!isfinite(st->alpha.x) || !isfinite(st->alpha.y)) {
                st->status = GS_NONFINITE;
                st->done = 1;
            }
        }
    } else {
        st->omega = tot[2] > 0.f ? make_float2(tot[0] / tot[2], tot[1] / tot[2])
                                 : make_float2(0.f, 0.f);
        if (!isfinite(st->omega.x) || !isfinite(st->omega.y)) {
            st->status = GS_NONFINITE;
            st->done = 1;
        }
    }
    if (st->done) lp_publish(st);
}

// ---------------------------------------------------------------------------
// low-precision BiCGStab vector kernels (thread per site)
// ---------------------------------------------------------------------------

// r = rhat = p = scale * r64 (AoS FP64 -> SoA S), x = 0, rho = ||r||^2.
template <class S>
__global__ void k_lp_init(const double2* __restrict__ r64, const double* __restrict__ rr64,
                          void* r, void* rhat, void* p, void* x, int64_t n, float tol,
                          LpState* st, float* partial, unsigned int* counter) {
    const double nrm2 = *rr64;
    const float scale = nrm2 > 0.0 ? (float)(1.0 / sqrt(nrm2)) : 0.f;
    float acc[1] = {0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[24], z[24];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const double2 v = r64[k * 12 + q];
            f[2 * q] = (float)v.x * scale;
            f[2 * q + 1] = (float)v.y * scale;
            z[2 * q] = z[2 * q + 1] = 0.f;
        }
        Store<S>::store_spinor(r, n, k, f);
        Store<S>::store_spinor(rhat, n, k, f);
        Store<S>::store_spinor(p, n, k, f);
        Store<S>::store_spinor(x, n, k, z);
        // norms of the stored (rounded) values
        Store<S>::load_spinor(r, n, k, f);
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[0] = fmaf(f[q], f[q], acc[0]);
    }
    float tot[1];
    if (lp_reduce_last<1>(acc, partial, counter, tot) && threadIdx.x == 0) {
        st->bb = tot[0];
        st->rr = tot[0];
        st->rho = make_float2(tot[0], 0.f);
        st->alpha = st->omega = st->beta = make_float2(0.f, 0.f);
        st->tol2 = tol * tol * tot[0];
        st->iter = 0;
        st->status = isfinite(tot[0]) ? GS_OK : GS_NONFINITE;
        st->done = (tot[0] == 0.f || !isfinite(tot[0])) ? 1 : 0;
        lp_publish(st);
    }
}

// s = r - alpha v ; x += alpha p ; ||s||^2
template <class S>
__global__ void k_lp_s(const void* r, const void* v, const void* p, void* s, void* x, int64_t n,
                       LpState* st, float* partial, unsigned int* counter) {
    if (st->done) return;
    const float2 al = st->alpha;
    float acc[1] = {0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float fr[24], fv[24], fp[24], fx[24];
        Store<S>::load_spinor(r, n, k, fr);
        Store<S>::load_spinor(v, n, k, fv);
        Store<S>::load_spinor(p, n, k, fp);
        Store<S>::load_spinor(x, n, k, fx);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float vr = fv[2 * q], vi = fv[2 * q + 1];
            fr[2 * q] -= al.x * vr - al.y * vi;
            fr[2 * q + 1] -= al.x * vi + al.y * vr;
            const float pr = fp[2 * q], pi = fp[2 * q + 1];
            fx[2 * q] = fmaf(al.x, pr, fmaf(-al.y, pi, fx[2 * q]));
            fx[2 * q + 1] = fmaf(al.x, pi, fmaf(al.y, pr, fx[2 * q + 1]));
        }
        Store<S>::store_spinor(s, n, k, fr);
        Store<S>::store_spinor(x, n, k, fx);
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[0] = fmaf(fr[q], fr[q], acc[0]);
    }
    float tot[1];
    if (lp_reduce_last<1>(acc, partial, counter, tot) && threadIdx.x == 0) {
        if (!isfinite(tot[0])) {
            st->status = GS_NONFINITE;
            st->done = 1;
        } else if (tot[0] <= st->tol2) {
            st->rr = tot[0];
            st->iter += 1;
            st->done = 1;
        }
        if (st->done) lp_publish(st);
    }
}

// x += omega s ; r = s - omega t ; rho' = <rhat, r> ; ||r||^2 ; beta
template <class S>
__global__ void k_lp_xr(const void* s, const void* t, const void* rhat, void* x, void* r,
                        int64_t n, LpState* st, float* partial, unsigned int* counter) {
    if (st->done) return;
    const float2 om = st->omega;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float fs[24], ft[24], fh[24], fx[24];
        Store<S>::load_spinor(s, n, k, fs);
        Store<S>::load_spinor(t, n, k, ft);
        Store<S>::load_spinor(rhat, n, k, fh);
        Store<S>::load_spinor(x, n, k, fx);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float sr = fs[2 * q], si = fs[2 * q + 1];
            fx[2 * q] = fmaf(om.x, sr, fmaf(-om.y, si, fx[2 * q]));
            fx[2 * q + 1] = fmaf(om.x, si, fmaf(om.y, sr, fx[2 * q + 1]));
            const float tr = ft[2 * q], ti = ft[2 * q + 1];
            const float rr = sr - (om.x * tr - om.y * ti);
            const float ri = si - (om.x * ti + om.y * tr);
            fs[2 * q] = rr;
            fs[2 * q + 1] = ri;
            acc[0] = fmaf(fh[2 * q], rr, fmaf(fh[2 * q + 1], ri, acc[0]));
            acc[1] = fmaf(fh[2 * q], ri, fmaf(-fh[2 * q + 1], rr, acc[1]));
            acc[2] = fmaf(rr, rr, fmaf(ri, ri, acc[2]));
        }
        Store<S>::store_spinor(x, n, k, fx);
        Store<S>::store_spinor(r, n, k, fs);
    }
    float tot[3];
    if (lp_reduce_last<3>(acc, partial, counter, tot) && threadIdx.x == 0) {
        const float2 rho_new = make_float2(tot[0], tot[1]);
        st->rr = tot[2];
        st->iter += 1;
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
            st->status = GS_NONFINITE;
            st->done = 1;
        } else if (tot[2] <= st->tol2) {
            st->done = 1;
        } else if ((om.x == 0.f && om.y == 0.f) || (rho_new.x == 0.f && rho_new.y == 0.f)) {
            st->status = GS_BREAKDOWN;
            st->done = 1;
        } else {
            st->beta = cmulf2(cdivf_(rho_new, st->rho), cdivf_(st->alpha, om));
            st->rho = rho_new;
        }
        lp_publish(st);
    }
}

// p = r + beta (p - omega v)
template <class S>
__global__ void k_lp_p(const void* r, const void* v, void* p, int64_t n, const LpState* st) {
    if (st->done) return;
    const float2 be = st->beta, om = st->omega;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float fr[24], fv[24], fp[24];
        Store<S>::load_spinor(r, n, k, fr);
        Store<S>::load_spinor(v, n, k, fv);
        Store<S>::load_spinor(p, n, k, fp);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float vr = fv[2 * q], vi = fv[2 * q + 1];
            const float qr = fp[2 * q] - (om.x * vr - om.y * vi);
            const float qi = fp[2 * q + 1] - (om.x * vi + om.y * vr);
            fp[2 * q] = fmaf(be.x, qr, fmaf(-be.y, qi, fr[2 * q]));
            fp[2 * q + 1] = fmaf(be.x, qi, fmaf(be.y, qr, fr[2 * q + 1]));
        }
        Store<S>::store_spinor(p, n, k, fp);
    }
}

// z64 += sqrt(rr64) * e   (undo the normalisation of the cycle's right-hand side)
template <class S>
__global__ void k_lp_accum(const void* e, const double* __restrict__ rr64, double2* z64,
                           int64_t n) {
    const double scale = sqrt(*rr64);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[24];
        Store<S>::load_spinor(e, n, k, f);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            double2 z = z64[k * 12 + q];
            z.x = fma(scale, (double)f[2 * q], z.x);
            z.y = fma(scale, (double)f[2 * q + 1], z.y);
            z64[k * 12 + q] = z;
        }
    }
}

// complex128 AoS (n sites) <-> low-precision SoA
template <class S>
__global__ void k_lp_pack(const double2* __restrict__ x, void* y, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[24];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const double2 v = x[k * 12 + q];
            f[2 * q] = (float)v.x;
            f[2 * q + 1] = (float)v.y;
        }
        Store<S>::store_spinor(y, n, k, f);
    }
}

template <class S>
__global__ void k_lp_unpack(const void* x, double2* __restrict__ y, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[24];
        Store<S>::load_spinor(x, n, k, f);
#pragma unroll
        for (int q = 0; q < 12; ++q) y[k * 12 + q] = make_double2((double)f[2 * q], (double)f[2 * q + 1]);
    }
}

// compact rest-set neighbour table and low-precision links from a plan
template <class S>
__global__ void k_lp_tables(int64_t nb, int64_t n, const int2* __restrict__ nbr,
                            const double2* __restrict__ links64, int2* __restrict__ nbr_r,
                            void* links_lp) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = nb + k;
        for (int mu = 0; mu < 4; ++mu) {
            const int2 q = nbr[j * 4 + mu];
            nbr_r[k * 4 + mu] = make_int2(q.x >= nb ? (int)(q.x - nb) : -1,
                                          q.y >= nb ? (int)(q.y - nb) : -1);
            float f[12];
            const double2* u = links64 + (j * 4 + mu) * 9;  // rows 0 and 1
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                f[2 * c] = (float)u[c].x;
                f[2 * c + 1] = (float)u[c].y;
            }
            Store<S>::store_link(links_lp, n, mu, k, f);
        }
    }
}

int lp_block(int64_t n, int sms) {
    if (n >= (int64_t)sms * 4 * 128) return 128;
    if (n >= (int64_t)sms * 2 * 64) return 64;
    return 32;
}

// Launch the low-precision stencil (variant 1: thread per site; 2: warp per
// direction); with profiling on, bracket it by events and count its
// algorithmic work (168 flop per in-set hop + 48 per site; bytes: spinor in +
// out, one 12-real link per link used, each datum once).
template <class S>
gs_status launch_lp_stencil(gs_ctx* c, LpArgs a, long long hops, int variant, long long* launches) {
    int slot = -1;
    a.ran = nullptr;
    if (c->prof.on) {
        gs_status s = prof_begin(c, &slot);
        if (s != GS_OK) return s;
        a.ran = c->prof.ran_dev + slot;
    }
    if (variant == 2) {
        int64_t g = (a.n + kLpSites - 1) / kLpSites;
        if (a.epi != EPI_NONE && g > kMaxRedBlocks) g = kMaxRedBlocks;
        switch (a.epi) {
            case EPI_NONE: k_dslash_lp_dir<S, EPI_NONE><<<(int)g, kLpThreads, 0, c->stream>>>(a); break;
            case EPI_DOT_RHAT_V: k_dslash_lp_dir<S, EPI_DOT_RHAT_V><<<(int)g, kLpThreads, 0, c->stream>>>(a); break;
            default: k_dslash_lp_dir<S, EPI_DOT_TS><<<(int)g, kLpThreads, 0, c->stream>>>(a); break;
        }
    } else {
        // variants 1, 3, 4: thread per site with a register budget for
        // 4, 6 or 8 blocks of 128 threads per SM
        const int b = lp_block(a.n, c->num_sms);
        int64_t g = (a.n + b - 1) / b;
        if (a.epi != EPI_NONE && g > kMaxRedBlocks) g = kMaxRedBlocks;
#define GS_SITE_LAUNCH(MB)                                                                       \
        switch (a.epi) {                                                                         \
            case EPI_NONE: k_dslash_lp_site<S, EPI_NONE, MB><<<(int)g, b, 0, c->stream>>>(a); break; \
            case EPI_DOT_RHAT_V:                                                                 \
                k_dslash_lp_site<S, EPI_DOT_RHAT_V, MB><<<(int)g, b, 0, c->stream>>>(a); break;  \
            default: k_dslash_lp_site<S, EPI_DOT_TS, MB><<<(int)g, b, 0, c->stream>>>(a); break; \
        }
        if (variant == 3) {
            GS_SITE_LAUNCH(6)
        } else if (variant == 4) {
            GS_SITE_LAUNCH(8)
        } else {
            GS_SITE_LAUNCH(4)
        }
#undef GS_SITE_LAUNCH
    }
    ++*launches;
    GS_CHECK_LAUNCH(c);
    if (slot >= 0) {
        const double sb = (double)Store<S>::spinor_bytes, lb = (double)Store<S>::link_bytes;
        const int prec = sizeof(S) == 4 ? GS_F32 : GS_BF16;
        return prof_end_work(c, slot, prec, a.n, hops, 168.0 * hops + 48.0 * a.n,
                             2.0 * sb * a.n + lb * 0.5 * hops);
    }
    return GS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct LpWork {
    int prec = -1;
    int64_t cap = 0;
    void *x = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr,
         *t = nullptr;
    LpState* st = nullptr;
    float* partial = nullptr;
    unsigned int* counter = nullptr;
    double* rr64 = nullptr;       // device ||r||^2 of the current FP64 residual
    double* rr64_host = nullptr;  // pinned
};

struct LpPlanData {
    const Plan* plan = nullptr;
    int prec = -1;
    int64_t nb = 0;        // labels below nb are excluded (0 for the full lattice)
    int64_t n = 0;         // sites of the set
    long long hops = 0;    // in-set neighbour terms of one D application
    int variant = 0;       // stencil variant: 1/3/4 = thread per site (register budget for
                           // 4/6/8 blocks per SM), 2 = warp per direction
    int2* nbr_r = nullptr;
    void* links = nullptr;
};

static size_t spinor_bytes(int prec) { return prec == GS_BF16 ? 48 : 96; }
static gs_status ensure_lp(gs_ctx* c, int prec, int64_t n);
static size_t link_bytes(int prec) { return prec == GS_BF16 ? 24 : 48; }

struct MixedState {
    LpWork w;
    std::vector<LpPlanData> plans;
    double2* e64 = nullptr;  // FP64 correction of the fallback solve (rest set)
    int64_t e64_cap = 0;
};

static MixedState* mixed_of(gs_ctx* c) {
    if (!c->mixed) c->mixed = new MixedState();
    return (MixedState*)c->mixed;
}

void free_mixed(gs_ctx* c) {
    MixedState* m = (MixedState*)c->mixed;
    if (!m) return;
    void* bufs[] = {m->w.x, m->w.r, m->w.rhat, m->w.p, m->w.v, m->w.s, m->w.t};
    for (void* b : bufs) cudaFree(b);
    cudaFree(m->w.st);
    cudaFree(m->w.partial);
    cudaFree(m->w.counter);
    cudaFree(m->w.rr64);
    cudaFree(m->e64);
    if (m->w.rr64_host) cudaFreeHost(m->w.rr64_host);
    for (auto& pd : m->plans) {
        cudaFree(pd.nbr_r);
        cudaFree(pd.links);
    }
    delete m;
    c->mixed = nullptr;
}

static gs_status ensure_lp(gs_ctx* c, int prec, int64_t n) {
    MixedState* m = mixed_of(c);
    LpWork& w = m->w;
    if (w.st == nullptr) {
        if (cudaMalloc(&w.st, sizeof(LpState)) != cudaSuccess ||
            cudaMalloc(&w.partial, kMaxRedBlocks * kMaxRedVals * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&w.counter, sizeof(unsigned int)) != cudaSuccess ||
            cudaMalloc(&w.rr64, sizeof(double)) != cudaSuccess ||
            cudaHostAlloc(&w.rr64_host, sizeof(double), 0) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GS_ENOMEM, "allocating the mixed-precision state failed");
        }
        GS_CUDA(c, cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), c->stream));
        // the low-precision state publishes through the inner solver's mapped mirror
        gs_status s = ensure_inner(c, 1);
        if (s != GS_OK) return s;
        LpState init;
        memset(&init, 0, sizeof init);
        init.pub = c->inner.pub_dev;
        GS_CUDA(c, cudaMemcpyAsync(w.st, &init, sizeof init, cudaMemcpyHostToDevice, c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    const size_t need = (size_t)n * spinor_bytes(prec);
    if (w.cap < (int64_t)need) {
        void** bufs[] = {&w.x, &w.r, &w.rhat, &w.p, &w.v, &w.s, &w.t};
        for (void** b : bufs) {
            cudaFree(*b);
            *b = nullptr;
        }
        for (void** b : bufs)
            if (cudaMalloc(b, need) != cudaSuccess) {
                cudaGetLastError();
                return set_err(c, GS_ENOMEM, "allocating low-precision vectors failed");
            }
        w.cap = (int64_t)need;
    }
    return GS_OK;
}

// The autotuner: time both stencil variants on this set (2 warm-up and 5
// timed launches each, CUDA events, zeroed operands) and keep the faster one;
// a variant forced with gs_set_option skips the timing.
static gs_status lp_tune(gs_ctx* c, LpPlanData& pd) {
    if (c->opt_stencil_variant == 1 || c->opt_stencil_variant == 2) {
        pd.variant = c->opt_stencil_variant;
        return GS_OK;
    }
    gs_status s = ensure_lp(c, pd.prec, pd.n);
    if (s != GS_OK) return s;
    MixedState* m = mixed_of(c);
    const size_t bytes = (size_t)pd.n * spinor_bytes(pd.prec);
    GS_CUDA(c, cudaMemsetAsync(m->w.p, 0, bytes, c->stream));
    LpArgs a;
    memset(&a, 0, sizeof a);
    a.out = m->w.v;
    a.in = m->w.p;
    a.links = pd.links;
    a.nbr = pd.nbr_r;
    a.n = pd.n;
    a.diag = (float)(c->m0 + 4.0);
    a.epi = EPI_NONE;
    cudaEvent_t e0, e1;
    GS_CUDA(c, cudaEventCreate(&e0));
    GS_CUDA(c, cudaEventCreate(&e1));
    float best = 0.f;
    const bool was_on = c->prof.on;
    c->prof.on = false;
    for (int v = 1; v <= 4; ++v) {
        long long l = 0;
        for (int r = 0; r < 7; ++r) {
            if (r == 2) GS_CUDA(c, cudaEventRecord(e0, c->stream));
            s = (pd.prec == GS_BF16) ? launch_lp_stencil<__nv_bfloat16>(c, a, pd.hops, v, &l)
                                     : launch_lp_stencil<float>(c, a, pd.hops, v, &l);
            if (s != GS_OK) break;
        }
        c->launches += l;
        if (s != GS_OK) break;
        GS_CUDA(c, cudaEventRecord(e1, c->stream));
        GS_CUDA(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        GS_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        if (v == 1 || ms < best) {
            best = ms;
            pd.variant = v;
        }
    }
    c->prof.on = was_on;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tuned_variant = pd.variant;
    return s;
}

static gs_status lp_plan(gs_ctx* c, const Plan* p, int prec, LpPlanData** out) {
    MixedState* m = mixed_of(c);
    for (auto& pd : m->plans)
        if (pd.plan == p && pd.prec == prec) {
            *out = &pd;
            return GS_OK;
        }
    LpPlanData pd;
    pd.plan = p;
    pd.prec = prec;
    // the identity plan stands for the whole lattice; a permutation for its rest set
    pd.nb = (p->type == 0) ? 0 : p->nb;
    pd.n = c->V - pd.nb;
    pd.hops = (p->type == 0) ? p->hops[0][0] : p->hops[1][1];
    const int64_t n = pd.n;
    if (cudaMalloc(&pd.nbr_r, (size_t)n * 4 * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&pd.links, (size_t)n * 4 * link_bytes(prec)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, GS_ENOMEM, "allocating low-precision links failed");
    }
    const int g = grid_for(n, 256, c->num_sms * 8);
    if (prec == GS_BF16)
        k_lp_tables<__nv_bfloat16><<<g, 256, 0, c->stream>>>(pd.nb, n, p->nbr, p->links, pd.nbr_r,
                                                             pd.links);
    else
        k_lp_tables<float><<<g, 256, 0, c->stream>>>(pd.nb, n, p->nbr, p->links, pd.nbr_r, pd.links);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    gs_status s = lp_tune(c, pd);
    if (s != GS_OK) return s;
    m->plans.push_back(pd);
    *out = &m->plans.back();
    return GS_OK;
}

void invalidate_mixed_links(gs_ctx* c) {
    MixedState* m = (MixedState*)c->mixed;
    if (!m) return;
    for (auto& pd : m->plans) {
        cudaFree(pd.nbr_r);
        cudaFree(pd.links);
    }
    m->plans.clear();
}

template <class S>
static gs_status lp_bicgstab(gs_ctx* c, LpPlanData* pd, int64_t n, float tol, int maxit,
                             int depth, int* iters_out, int* status_out) {
    MixedState* m = mixed_of(c);
    LpWork& w = m->w;
    const int bb = kLpRed;
    int gr = grid_for(n, bb, c->num_sms * 4 < kMaxRedBlocks ? c->num_sms * 4 : kMaxRedBlocks);
    int gp = grid_for(n, bb, c->num_sms * 16);
    LpArgs k1;
    memset(&k1, 0, sizeof k1);
    k1.out = w.v;
    k1.in = w.p;
    k1.links = pd->links;
    k1.nbr = pd->nbr_r;
    k1.n = n;
    k1.diag = (float)(c->m0 + 4.0);
    k1.epi = EPI_DOT_RHAT_V;
    k1.epi_vec = w.rhat;
    k1.st = w.st;
    k1.partial = w.partial;
    k1.counter = w.counter;
    LpArgs k3 = k1;
    k3.out = w.t;
    k3.in = w.s;
    k3.epi = EPI_DOT_TS;
    k3.epi_vec = w.s;
    InnerWork& iw = c->inner;
    volatile BicgPublic* pub = iw.pub_host;
    long long dummy = 0;
    gs_status s;
    int enq = 0;
    GS_CUDA(c, cudaEventRecord(iw.ev[0], c->stream));
    GS_CUDA(c, cudaEventSynchronize(iw.ev[0]));
    if (!pub->done) {
        for (int it = 0; it < maxit; ++it) {
            if (it >= depth) {
                GS_CUDA(c, cudaEventSynchronize(iw.ev[(it - depth) % 4]));
                if (pub->done) break;
            }
            if ((s = launch_lp_stencil<S>(c, k1, pd->hops, pd->variant, &dummy)) != GS_OK) return s;
            k_lp_s<S><<<gr, bb, 0, c->stream>>>(w.r, w.v, w.p, w.s, w.x, n, w.st, w.partial,
                                                 w.counter);
            if ((s = launch_lp_stencil<S>(c, k3, pd->hops, pd->variant, &dummy)) != GS_OK) return s;
            k_lp_xr<S><<<gr, bb, 0, c->stream>>>(w.s, w.t, w.rhat, w.x, w.r, n, w.st, w.partial,
                                                  w.counter);
            k_lp_p<S><<<gp, bb, 0, c->stream>>>(w.r, w.v, w.p, n, w.st);
            c->launches += 3;
            c->stencil_sites += 2 * n;
            GS_CHECK_LAUNCH(c);
            GS_CUDA(c, cudaEventRecord(iw.ev[it % 4], c->stream));
            enq = it + 1;
        }
        if (enq > 0) GS_CUDA(c, cudaEventSynchronize(iw.ev[(enq - 1) % 4]));
    }
    c->launches += dummy;
    *iters_out = pub->iter;
    *status_out = pub->status;
    return GS_OK;
}

// z = D_rr^-1 t to FP64 tolerance o.inner_tol, low-precision inner iterations.
gs_status inner_solve_mixed(gs_ctx* c, const Plan* p, const double2* t, double2* z,
                            const gs_solve_opts& o, gs_solve_stats& st) {
    const int prec = o.inner_prec;
    const int64_t n = c->V - p->nb;
    gs_status s = ensure_inner(c, n);
    if (s != GS_OK) return s;
    if ((s = ensure_lp(c, prec, n)) != GS_OK) return s;
    LpPlanData* pd = nullptr;
    if ((s = lp_plan(c, p, prec, &pd)) != GS_OK) return s;
    MixedState* m = mixed_of(c);
    LpWork& w = m->w;
    InnerWork& iw = c->inner;
    double2* r64 = iw.r;  // FP64 residual (rest set)
    const size_t vbytes = (size_t)n * kSiteC * sizeof(double2);
    GS_CUDA(c, cudaMemsetAsync(z, 0, vbytes, c->stream));
    GS_CUDA(c, cudaMemcpyAsync(r64, t, vbytes, cudaMemcpyDeviceToDevice, c->stream));
    RedScratch red = iw.red;
    if ((s = launch_norm2(c, red, r64, n * kSiteC, w.rr64)) != GS_OK) return s;
    GS_CUDA(c, cudaMemcpyAsync(w.rr64_host, w.rr64, sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    const double tt = *w.rr64_host;
    st.inner_solves += 1;
    if (!isfinite(tt)) return set_err(c, GS_NONFINITE, "non-finite right-hand side");
    if (tt == 0.0) return GS_OK;
    const double target = o.inner_tol * o.inner_tol * tt;
    const float lo_tol = (float)(o.lowp_tol > 0.0 ? o.lowp_tol : (prec == GS_BF16 ? 3e-2 : 1e-5));
    const int depth = (o.check_every >= 1 && o.check_every <= 4) ? o.check_every : 2;
    double rr = tt;
    int stalls = 0;
    long long iters_total = 0;
    const int gs_ = grid_for(n, kLpRed, c->num_sms * 4 < kMaxRedBlocks ? c->num_sms * 4 : kMaxRedBlocks);
    const int gp = grid_for(n, kLpRed, c->num_sms * 16);
    StencilArgs ra;
    memset(&ra, 0, sizeof ra);
    ra.out = r64;
    ra.o0 = p->nb;
    ra.n_out = n;
    ra.inA = z;
    ra.a0 = p->nb;
    ra.a1 = c->V;
    ra.b1 = c->V;
    ra.diag = c->m0 + 4.0;
    ra.negate = 1;
    ra.addend = t;
    ra.plan = p;
    ra.nbr = p->nbr;
    ra.links = p->links;
    int cycles = 0;
    for (; cycles < 100 && rr > target; ++cycles) {
        if (stalls >= 2) break;
        if (prec == GS_BF16)
            k_lp_init<__nv_bfloat16><<<gs_, kLpRed, 0, c->stream>>>(
                r64, w.rr64, w.r, w.rhat, w.p, w.x, n, lo_tol, w.st, w.partial, w.counter);
        else
            k_lp_init<float><<<gs_, kLpRed, 0, c->stream>>>(r64, w.rr64, w.r, w.rhat, w.p, w.x, n,
                                                            lo_tol, w.st, w.partial, w.counter);
        c->launches++;
        GS_CHECK_LAUNCH(c);
        int it = 0, status = 0;
        if (prec == GS_BF16)
            s = lp_bicgstab<__nv_bfloat16>(c, pd, n, lo_tol, o.inner_max_iter, depth, &it, &status);
        else
            s = lp_bicgstab<float>(c, pd, n, lo_tol, o.inner_max_iter, depth, &it, &status);
        if (s != GS_OK) return s;
        iters_total += it;
        // z += ||r|| e ; r = t - D_rr z (FP64) ; ||r||^2
        if (prec == GS_BF16)
            k_lp_accum<__nv_bfloat16><<<gp, kLpRed, 0, c->stream>>>(w.x, w.rr64, z, n);
        else
            k_lp_accum<float><<<gp, kLpRed, 0, c->stream>>>(w.x, w.rr64, z, n);
        c->launches++;
        GS_CHECK_LAUNCH(c);
        if ((s = launch_stencil_f64(c, ra)) != GS_OK) return s;
        if ((s = launch_norm2(c, red, r64, n * kSiteC, w.rr64)) != GS_OK) return s;
        GS_CUDA(c, cudaMemcpyAsync(w.rr64_host, w.rr64, sizeof(double), cudaMemcpyDeviceToHost,
                                   c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        const double rr_new = *w.rr64_host;
        if (!isfinite(rr_new)) return set_err(c, GS_NONFINITE, "non-finite mixed residual");
        stalls = (rr_new > 0.25 * rr) ? stalls + 1 : 0;
        rr = rr_new;
    }
    st.inner_iters += iters_total;
    st.lowp_cycles += cycles;
    if (iters_total > st.inner_max_seen) st.inner_max_seen = (int)iters_total;
    if (rr > target) {
        // the plain FP64 solve finishes the correction: z += D_rr^-1 r
        gs_solve_opts o64 = o;
        o64.inner_prec = GS_F64;
        o64.inner_tol = sqrt(target / rr);
        if (m->e64_cap < n) {
            cudaFree(m->e64);
            m->e64 = nullptr;
            if (cudaMalloc(&m->e64, (size_t)n * kSiteC * sizeof(double2)) != cudaSuccess) {
                cudaGetLastError();
                return set_err(c, GS_ENOMEM, "allocating the FP64 correction failed");
            }
            m->e64_cap = n;
        }
        gs_solve_stats sub;
        memset(&sub, 0, sizeof sub);
        st.lowp_fallbacks += 1;
        gs_status si = inner_solve_f64(c, p, r64, m->e64, o64, sub);
        st.inner_iters += sub.inner_iters;
        if (si != GS_OK && si != GS_MAXITER) return si;
        if ((s = launch_axpby(c, make_double2(1.0, 0.0), m->e64, make_double2(1.0, 0.0), z,
                              n * kSiteC)) != GS_OK)
            return s;
        rr *= sub.inner_residual * sub.inner_residual;
        if (si == GS_MAXITER) return si;
    }
    const double rel = sqrt(rr / tt);
    if (rel > st.inner_residual) st.inner_residual = rel;
    return GS_OK;
}

// ---------------------------------------------------------------------------
// ABI: low-precision vectors and the low-precision stencil
// ---------------------------------------------------------------------------
static gs_status lp_entry(gs_ctx* c, int type, int dir, int inverse, int prec, LpPlanData** pd) {
    if (!c) return GS_EINVAL;
    if (prec != GS_F32 && prec != GS_BF16)
        return set_err(c, GS_EINVAL, "low-precision calls take GS_F32 or GS_BF16, not %d", prec);
    if (type != 0 && type != GS_TYPE_I && type != GS_TYPE_II)
        return set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    return lp_plan(c, p, prec, pd);
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_lowp_pack(gs_ctx* c, int type, int dir, int inverse, int prec, const void* x_dev,
                       void* x_lp_dev) {
    LpPlanData* pd = nullptr;
    gs_status s = lp_entry(c, type, dir, inverse, prec, &pd);
    if (s != GS_OK) return s;
    if (!x_dev || !x_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    const int g = grid_for(pd->n, 256, c->num_sms * 8);
    if (prec == GS_BF16)
        k_lp_pack<__nv_bfloat16><<<g, 256, 0, c->stream>>>((const double2*)x_dev, x_lp_dev, pd->n);
    else
        k_lp_pack<float><<<g, 256, 0, c->stream>>>((const double2*)x_dev, x_lp_dev, pd->n);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status gs_lowp_unpack(gs_ctx* c, int type, int dir, int inverse, int prec,
                         const void* x_lp_dev, void* x_dev) {
    LpPlanData* pd = nullptr;
    gs_status s = lp_entry(c, type, dir, inverse, prec, &pd);
    if (s != GS_OK) return s;
    if (!x_dev || !x_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    const int g = grid_for(pd->n, 256, c->num_sms * 8);
    if (prec == GS_BF16)
        k_lp_unpack<__nv_bfloat16><<<g, 256, 0, c->stream>>>(x_lp_dev, (double2*)x_dev, pd->n);
    else
        k_lp_unpack<float><<<g, 256, 0, c->stream>>>(x_lp_dev, (double2*)x_dev, pd->n);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status wilson_apply_lowp(gs_ctx* c, int type, int dir, int inverse, int prec,
                            const void* x_lp_dev, void* y_lp_dev) {
    LpPlanData* pd = nullptr;
    gs_status s = lp_entry(c, type, dir, inverse, prec, &pd);
    if (s != GS_OK) return s;
    if (!x_lp_dev || !y_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    LpArgs a;
    memset(&a, 0, sizeof a);
    a.out = y_lp_dev;
    a.in = x_lp_dev;
    a.links = pd->links;
    a.nbr = pd->nbr_r;
    a.n = pd->n;
    a.diag = (float)(c->m0 + 4.0);
    a.epi = EPI_NONE;
    long long launches = 0;
    s = (prec == GS_BF16) ? launch_lp_stencil<__nv_bfloat16>(c, a, pd->hops, pd->variant, &launches)
                          : launch_lp_stencil<float>(c, a, pd->hops, pd->variant, &launches);
    c->launches += launches;
    c->stencil_sites += pd->n;
    return s;
}

}  // extern "C"
