// Device code of the low-precision (FP32 / BF16 storage, FP32 arithmetic)
// Wilson stencil and its reductions, shared by the mixed inner solver
// (mixed.cu) and the persistent solver kernels (persistent.cu).
#pragma once

#include <cuda_bf16.h>
#include <math.h>

#include "gs_internal.cuh"

namespace gs {

struct LpState;

// The whole lattice in site order (x0 fastest), whose neighbours follow from
// the site index: the stencil then reads no neighbour table.  k / L uses the
// multiply-high method for division by an invariant integer (Granlund and
// Montgomery, PLDI 1994): with l = ceil(log2 L) and
// m = floor(2^32 (2^l - L) / L) + 1, k / L = (umulhi(k, m) + k) >> l for every
// k < 2^31 (site indices are below 2^31 / 12).
struct LexDims {
    int on;         // 0: use the table
    int L[4];
    unsigned mag[3];
    int sh[3];
};

// Arguments of the low-precision stencil launches (FP32 arithmetic).
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
    LexDims lex;         // on: the set is the whole lattice in site order
};

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
    // CG: read through L2 only (coherent within a persistent kernel)
    template <bool CG = false>
    __device__ __forceinline__ static void load_spinor(const void* base, int64_t n, int64_t k,
                                                       float (&f)[24]) {
        const float4* b = (const float4*)base;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float4 v = CG ? __ldcg(b + c * n + k) : __ldg(b + c * n + k);
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
    template <bool CG = false>
    __device__ __forceinline__ static void load_spinor(const void* base, int64_t n, int64_t k,
                                                       float (&f)[24]) {
        const uint4* b = (const uint4*)base;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint4 v = CG ? __ldcg(b + c * n + k) : __ldg(b + c * n + k);
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

__device__ __forceinline__ unsigned lex_div(unsigned k, unsigned m, int l) {
    return (__umulhi(k, m) + k) >> l;
}

// forward and backward neighbours of site k in direction mu, periodic
__device__ __forceinline__ void lex_coords(const LexDims& d, int64_t k, int (&x)[4]) {
    const unsigned s = (unsigned)k;
    const unsigned q0 = lex_div(s, d.mag[0], d.sh[0]);
    const unsigned q1 = lex_div(q0, d.mag[1], d.sh[1]);
    const unsigned q2 = lex_div(q1, d.mag[2], d.sh[2]);
    x[0] = (int)(s - q0 * (unsigned)d.L[0]);
    x[1] = (int)(q0 - q1 * (unsigned)d.L[1]);
    x[2] = (int)(q1 - q2 * (unsigned)d.L[2]);
    x[3] = (int)q2;
}

template <int MU>
__device__ __forceinline__ int2 lex_hop(const LexDims& d, int64_t k, const int (&x)[4]) {
    int st = 1;
#pragma unroll
    for (int nu = 0; nu < MU; ++nu) st *= d.L[nu];
    const int s = (int)k, L = d.L[MU];
    return make_int2(x[MU] + 1 < L ? s + st : s - (L - 1) * st, x[MU] > 0 ? s - st : s + (L - 1) * st);
}

// the eight neighbours of site k: (f0, b0, f1, b1) and (f2, b2, f3, b3)
__device__ __forceinline__ void site_nbrs(const LpArgs& a, int64_t k, int4& n01, int4& n23) {
    if (a.lex.on) {
        int x[4];
        lex_coords(a.lex, k, x);
        const int2 h0 = lex_hop<0>(a.lex, k, x), h1 = lex_hop<1>(a.lex, k, x);
        const int2 h2 = lex_hop<2>(a.lex, k, x), h3 = lex_hop<3>(a.lex, k, x);
        n01 = make_int4(h0.x, h0.y, h1.x, h1.y);
        n23 = make_int4(h2.x, h2.y, h3.x, h3.y);
    } else {
        n01 = __ldg((const int4*)(a.nbr + k * 4));
        n23 = __ldg((const int4*)(a.nbr + k * 4) + 1);
    }
}

template <int MU>
__device__ __forceinline__ int2 dir_nbr(const LpArgs& a, int64_t k) {
    if (a.lex.on) {
        int x[4];
        lex_coords(a.lex, k, x);
        return lex_hop<MU>(a.lex, k, x);
    }
    return __ldg(a.nbr + k * 4 + MU);
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
    const int2 nb = valid ? dir_nbr<MU>(a, k) : make_int2(-1, -1);
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
template <class S, int MU, bool CG = false>
__device__ __forceinline__ void site_dir(const LpArgs& a, int64_t k, int2 nb, float (&acc)[24]) {
    const bool hf = nb.x >= 0, hb = nb.y >= 0;
    const int64_t jf = hf ? nb.x : k, jb = hb ? nb.y : k;
    float pf[24], pb[24], lf[12], lb[12];
    Store<S>::template load_spinor<CG>(a.in, a.n, jf, pf);
    Store<S>::template load_spinor<CG>(a.in, a.n, jb, pb);
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

// Raw (still packed) operands of one direction of one site: the two
// neighbour spinors and the two links, as loaded; unpacked only when used.
template <class S>
struct Raw;
template <>
struct Raw<float> {
    float4 pf[6], pb[6], lf[3], lb[3];
    __device__ __forceinline__ void load(const LpArgs& a, int mu, int64_t jf, int64_t jb, int64_t k) {
        const float4* in = (const float4*)a.in;
        const float4* L = (const float4*)a.links + (int64_t)mu * 3 * a.n;
#pragma unroll
        for (int c = 0; c < 6; ++c) pf[c] = __ldg(in + c * a.n + jf);
#pragma unroll
        for (int c = 0; c < 6; ++c) pb[c] = __ldg(in + c * a.n + jb);
#pragma unroll
        for (int c = 0; c < 3; ++c) lf[c] = __ldg(L + c * a.n + k);
#pragma unroll
        for (int c = 0; c < 3; ++c) lb[c] = __ldg(L + c * a.n + jb);
    }
    __device__ __forceinline__ static void spinor(const float4 (&v)[6], float (&f)[24]) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            f[4 * c] = v[c].x; f[4 * c + 1] = v[c].y; f[4 * c + 2] = v[c].z; f[4 * c + 3] = v[c].w;
        }
    }
    __device__ __forceinline__ static void link(const float4 (&v)[3], float (&f)[12]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            f[4 * c] = v[c].x; f[4 * c + 1] = v[c].y; f[4 * c + 2] = v[c].z; f[4 * c + 3] = v[c].w;
        }
    }
    __device__ __forceinline__ void unpack(float (&f)[24], float (&b)[24], float (&u)[12], float (&w)[12]) const {
        spinor(pf, f);
        spinor(pb, b);
        link(lf, u);
        link(lb, w);
    }
};
template <>
struct Raw<__nv_bfloat16> {
    uint4 pf[3], pb[3];
    uint2 lf[3], lb[3];
    __device__ __forceinline__ void load(const LpArgs& a, int mu, int64_t jf, int64_t jb, int64_t k) {
        const uint4* in = (const uint4*)a.in;
        const uint2* L = (const uint2*)a.links + (int64_t)mu * 3 * a.n;
#pragma unroll
        for (int c = 0; c < 3; ++c) pf[c] = __ldg(in + c * a.n + jf);
#pragma unroll
        for (int c = 0; c < 3; ++c) pb[c] = __ldg(in + c * a.n + jb);
#pragma unroll
        for (int c = 0; c < 3; ++c) lf[c] = __ldg(L + c * a.n + k);
#pragma unroll
        for (int c = 0; c < 3; ++c) lb[c] = __ldg(L + c * a.n + jb);
    }
    __device__ __forceinline__ static void spinor(const uint4 (&v)[3], float (&f)[24]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 t;
            t = unpack_bf2(v[c].x); f[8 * c + 0] = t.x; f[8 * c + 1] = t.y;
            t = unpack_bf2(v[c].y); f[8 * c + 2] = t.x; f[8 * c + 3] = t.y;
            t = unpack_bf2(v[c].z); f[8 * c + 4] = t.x; f[8 * c + 5] = t.y;
            t = unpack_bf2(v[c].w); f[8 * c + 6] = t.x; f[8 * c + 7] = t.y;
        }
    }
    __device__ __forceinline__ static void link(const uint2 (&v)[3], float (&f)[12]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 t;
            t = unpack_bf2(v[c].x); f[4 * c + 0] = t.x; f[4 * c + 1] = t.y;
            t = unpack_bf2(v[c].y); f[4 * c + 2] = t.x; f[4 * c + 3] = t.y;
        }
    }
    __device__ __forceinline__ void unpack(float (&f)[24], float (&b)[24], float (&u)[12], float (&w)[12]) const {
        spinor(pf, f);
        spinor(pb, b);
        link(lf, u);
        link(lb, w);
    }
};

// the two hops of direction MU from raw operands (masked hops contribute 0)
template <class S, int MU>
__device__ __forceinline__ void raw_dir(const Raw<S>& r, bool hf, bool hb, float (&acc)[24]) {
    float pf[24], pb[24], lf[12], lb[12];
    r.unpack(pf, pb, lf, lb);
    if (hf) {
        cf h[2][3], u[3][3], g[2][3];
        project<MU, true>(pf, h);
        rebuild(lf, u);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                cf t = cmul(u[q][0], h[s][0]);
                cfma_(t, u[q][1], h[s][1]);
                cfma_(t, u[q][2], h[s][2]);
                g[s][q] = t;
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
            for (int q = 0; q < 3; ++q) {
                cf t = cf{0.f, 0.f};
                ccfma_(t, u[0][q], h[s][0]);
                ccfma_(t, u[1][q], h[s][1]);
                ccfma_(t, u[2][q], h[s][2]);
                g[s][q] = t;
            }
        accumulate<MU, +1>(acc, g);
    }
}

template <class S, int EPI>
__device__ __forceinline__ void lp_finish(const LpArgs& a, LpState* st, float (&tot)[3]);

// Variant "pipelined site": one thread per site, like "site", but the loads of
// direction mu + 1 are issued before direction mu is computed (two operand
// buffers in registers, kept packed until used), so each thread waits for
// memory about twice per site instead of five times; fewer blocks fit per SM.
template <class S, int EPI, int MINB>
__global__ void __launch_bounds__(128, MINB) k_dslash_lp_pipe(LpArgs a) {
    const bool skip = a.st != nullptr && a.st->done;
    if (a.ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.ran = skip ? 0 : 1;
    if (skip) return;
    float e[3] = {0.f, 0.f, 0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int4 n01, n23;
        site_nbrs(a, k, n01, n23);
        // out-of-set neighbours (-1) read the site itself and are masked
        const bool h0f = n01.x >= 0, h0b = n01.y >= 0, h1f = n01.z >= 0, h1b = n01.w >= 0;
        const bool h2f = n23.x >= 0, h2b = n23.y >= 0, h3f = n23.z >= 0, h3b = n23.w >= 0;
        Raw<S> r0, r1;
        r0.load(a, 0, h0f ? n01.x : k, h0b ? n01.y : k, k);
        r1.load(a, 1, h1f ? n01.z : k, h1b ? n01.w : k, k);
        float acc[24];
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[q] = 0.f;
        raw_dir<S, 0>(r0, h0f, h0b, acc);
        r0.load(a, 2, h2f ? n23.x : k, h2b ? n23.y : k, k);
        raw_dir<S, 1>(r1, h1f, h1b, acc);
        r1.load(a, 3, h3f ? n23.z : k, h3b ? n23.w : k, k);
        raw_dir<S, 2>(r0, h2f, h2b, acc);
        float self[24];
        Store<S>::load_spinor(a.in, a.n, k, self);
        raw_dir<S, 3>(r1, h3f, h3b, acc);
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

template <class S, int EPI, int MINB>
__global__ void __launch_bounds__(128, MINB) k_dslash_lp_site(LpArgs a) {
    const bool skip = a.st != nullptr && a.st->done;
    if (a.ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.ran = skip ? 0 : 1;
    if (skip) return;
    float e[3] = {0.f, 0.f, 0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int4 n01, n23;
        site_nbrs(a, k, n01, n23);
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


}  // namespace
}  // namespace gs
