// The C -> C layer of the learned preconditioner (C = 24) on the fifth-generation
// tensor cores: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in
// tensor memory), weights moved by the bulk-copy engine, neighbour
// activations gathered by cp.async and transported by the CTA's threads.
//
// The layer  out(x)[R, a] = sum_d sum_k W_d[R, k] (U_d(x) in(x + d))[k, a]
// is a real GEMM over rows p = 3 x + a (site, colour):
//   A[p, k'] = Re / Im of T_d(x)[k, a],  T_d(x) = U_d(x) in(x + d)
//   B[n', k'] = the real form of W_d:  out_re = W_re T_re - W_im T_im,
//               out_im = W_im T_re + W_re T_im
// with n' = 2 R + (re, im), k' = (d, quarter, 2 kk + (re, im)), k = 24 quarter + kk.
// M = 256 rows per tile (two 128-lane accumulators), N = 192, K = 9 x 192,
// taken in 36 chunks of 48 (one transport, 24 input rows).  Operands are in
// the no-swizzle K-major core-matrix layout: an 8-row x 16-byte core matrix
// is 128 contiguous bytes, core matrices adjacent in K are 128 bytes apart
// (leading byte offset), 8-row groups 768 bytes apart (stride byte offset).
// The input activations are BF16 ([V][96][3] complex as bf16x2).
//
// Warp roles.  Warps 0-14 gather and transport: at chunk j they gather the
// raw neighbour rows of chunk j + 2 by cp.async (three raw buffers; the links
// of a transport once, two link buffers by transport parity), transport
// chunk j into the A stage (two stages, reused once the tensor core has
// committed the chunk two back) and arrive on the stage's full barrier; one
// named barrier per chunk among these warps orders the raw buffers.  Warp 15
// moves B_j by a bulk copy and issues the chunk's six MMAs as soon as the
// stage is full, then commits them to the stage's done barrier, so the MMAs
// never wait for a block barrier.  Every wait is bounded (the context's wait
// limit, GS_OPT_WAIT_LIMIT_US, 1 s by default); on a timeout the kernel
// stops, waits (bounded) for the MMAs it committed, frees its tensor memory
// and raises err.
#include <cuda_bf16.h>
#include <stdint.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kRows = 256;                       // GEMM rows per tile
constexpr int kRC = 96;                          // 4 C, C = 24
constexpr int kN = 192;                          // real output columns
constexpr int kQ = 24;                           // input rows per chunk
constexpr int kKC = 2 * kQ;                      // real K per chunk
constexpr int kChunks = 36;                      // 9 transports x 4 quarters
constexpr int kSites = 88;                       // site slots of a tile (at most 86 used)
constexpr uint32_t kSBO = (kKC / 8) * 128;       // 768
constexpr uint32_t kABytes = kRows * kKC * 2;    // 24576
constexpr uint32_t kBBytes = kN * kKC * 2;       // 18432
constexpr uint32_t kPStride = kQ * 3 * 4 + 16;   // 304: raw rows of one site (+16 against bank conflicts)
constexpr uint32_t kPBytes = kSites * kPStride;  // 26752
constexpr uint32_t kUBytes = kSites * 9 * 8;     // 6336
// dynamic shared memory map (offsets from a 128-byte aligned base): A and B
// stages x 2, raw rows x 3, links x 2, neighbour table
constexpr uint32_t kOffA = 0, kOffB = 2 * kABytes, kOffP = kOffB + 2 * kBBytes, kOffU = kOffP + 3 * kPBytes,
                   kOffY = kOffU + 2 * kUBytes, kSmemUsed = kOffY + 9 * kSites * 4;
constexpr size_t kSmem = kSmemUsed + 128;
constexpr int kThreads = 512;
constexpr int kStageWarps = 15;                  // gather + transport; warp 15 issues B and the MMAs
constexpr int kStageThreads = kStageWarps * 32;
constexpr int kHalfItems = 11 * 3 * 2;           // (8 site slots) x (8 rows) x (first / second row of a lane)
static_assert(kSmem <= 227 * 1024, "shared memory");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t core_off(int r, int k) {
    return (uint32_t)((r >> 3) * kSBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(kSBO >> 4) << 32) | ((uint64_t)1 << 46);
}
// D f32, A and B bf16, both K-major, N = 192, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: true when the phase of the given parity has completed, false
// after wait_ns of global time (the context's wait limit) or 2^30 polls
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long wait_ns) {
    const uint64_t t0 = gtime();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u && gtime() - t0 > wait_ns) return false;
    }
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // conj(a) b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// raw rows of chunk j of the tile into raw buffer j % 3, and with the first
// quarter of a transport its links into link buffer (transport & 1); issued
// by the transport warps, one commit group per chunk
__device__ __forceinline__ void gather(unsigned char* base, int j, const __nv_bfloat162* __restrict__ in,
                                       const float2* __restrict__ U32, int64_t xs0, int nsite) {
    const int d = j >> 2, qt = j & 3;
    const int* Y = (const int*)(base + kOffY) + d * kSites;
    const uint32_t P = su32(base + kOffP + (j % 3) * kPBytes);
    for (int i = threadIdx.x; i < nsite * 18; i += kStageThreads) {
        const int sl = i / 18, pc = i - sl * 18;
        const unsigned char* src = (const unsigned char*)(in + ((int64_t)Y[sl] * kRC + kQ * qt) * 3) + pc * 16;
        cp_async16(P + sl * kPStride + pc * 16, src);
    }
    if (d > 0 && qt == 0) {  // links of transport d, kept for its four quarters
        const int mu = (d - 1) & 3;
        const uint32_t Ub = su32(base + kOffU + (d & 1) * kUBytes);
        for (int i = threadIdx.x; i < nsite * 9; i += kStageThreads) {
            const int sl = i / 9, e = i - sl * 9;
            const int64_t ls = d <= 4 ? xs0 + sl : (int64_t)Y[sl];
            cp_async8(Ub + (sl * 9 + e) * 8, U32 + (ls * 4 + mu) * 9 + e);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Transport one chunk (24 input rows) of the raw rows in shared memory into
// the A stage.  MODE 0: identity, 1: U_mu(x) p (forward hop), 2: U^dag p
// (backward hop; the link is the neighbour's).  Half-items = (8 site slots)
// x (8 input rows) x (first or second row of a lane): lane = (site j, row q)
// handles row q or q + 4 of its site; the 66 half-items go in contiguous runs
// of four or five to the 15 transport warps, so a warp loads a site's link at
// most twice.  The bf16x2 stores of a warp land in 32 distinct banks (bank =
// 4 (row mod 8) + q).  Each output colour is one FMA chain per real
// component; the row bounds are checked only on the tile's edge items.
__device__ __forceinline__ uint32_t core_row(int r) { return (uint32_t)((r >> 3) * kSBO + (r & 7) * 16); }

// t = sum_c m_c p_c  (m_c = U[a][c]: forward) or sum_c conj(m_c) p_c (backward)
template <bool CONJ>
__device__ __forceinline__ float2 row3(float2 m0, float2 m1, float2 m2, float2 p0, float2 p1, float2 p2) {
    const float s = CONJ ? -1.f : 1.f;
    float re = m0.x * p0.x;
    re = fmaf(-s * m0.y, p0.y, re);
    re = fmaf(m1.x, p1.x, re);
    re = fmaf(-s * m1.y, p1.y, re);
    re = fmaf(m2.x, p2.x, re);
    re = fmaf(-s * m2.y, p2.y, re);
    float im = m0.x * p0.y;
    im = fmaf(s * m0.y, p0.x, im);
    im = fmaf(m1.x, p1.y, im);
    im = fmaf(s * m1.y, p1.x, im);
    im = fmaf(m2.x, p2.y, im);
    im = fmaf(s * m2.y, p2.x, im);
    return make_float2(re, im);
}

template <int MODE>
__device__ __forceinline__ void stage_chunk(const unsigned char* P, const float2* Ub, unsigned char* a_s, int warp,
                                            int sj, int kq, int off, int nsite) {
    const int h0 = warp * kHalfItems / kStageWarps, h1 = (warp + 1) * kHalfItems / kStageWarps;
    int cached = -1;
    float2 u[9];
    for (int hi = h0; hi < h1; ++hi) {
        const int sg = hi / 6, rem = hi - 6 * sg, kg = rem >> 1, h2 = rem & 1;
        const int sl = 8 * sg + sj;
        const int r0 = 3 * sl - off;
        if (r0 >= kRows) continue;
        const bool have = sl < nsite;
        if (MODE != 0 && have && sg != cached) {
#pragma unroll
            for (int e = 0; e < 9; ++e) u[e] = Ub[sl * 9 + e];
            cached = sg;
        }
        const int kk = 8 * kg + 4 * h2 + kq;
        // core matrix column of k' = 2 kk: (2 kk / 8) * 128 + (2 kk % 8) * 2
        const uint32_t ok = (uint32_t)((2 * kg + h2) * 128 + 4 * kq);
        float2 t0 = make_float2(0.f, 0.f), t1 = t0, t2 = t0;
        if (have) {
            const __nv_bfloat162* pr = (const __nv_bfloat162*)(P + sl * kPStride) + kk * 3;
            const float2 p0 = __bfloat1622float2(pr[0]), p1 = __bfloat1622float2(pr[1]),
                         p2 = __bfloat1622float2(pr[2]);
            if (MODE == 0) {
                t0 = p0;
                t1 = p1;
                t2 = p2;
            } else if (MODE == 1) {
                t0 = row3<false>(u[0], u[1], u[2], p0, p1, p2);
                t1 = row3<false>(u[3], u[4], u[5], p0, p1, p2);
                t2 = row3<false>(u[6], u[7], u[8], p0, p1, p2);
            } else {
                t0 = row3<true>(u[0], u[3], u[6], p0, p1, p2);
                t1 = row3<true>(u[1], u[4], u[7], p0, p1, p2);
                t2 = row3<true>(u[2], u[5], u[8], p0, p1, p2);
            }
        }
        if (r0 >= 0 && r0 + 2 < kRows) {
            *(__nv_bfloat162*)(a_s + core_row(r0) + ok) = __floats2bfloat162_rn(t0.x, t0.y);
            *(__nv_bfloat162*)(a_s + core_row(r0 + 1) + ok) = __floats2bfloat162_rn(t1.x, t1.y);
            *(__nv_bfloat162*)(a_s + core_row(r0 + 2) + ok) = __floats2bfloat162_rn(t2.x, t2.y);
        } else {
            if (r0 >= 0) *(__nv_bfloat162*)(a_s + core_row(r0) + ok) = __floats2bfloat162_rn(t0.x, t0.y);
            if (r0 + 1 >= 0 && r0 + 1 < kRows)
                *(__nv_bfloat162*)(a_s + core_row(r0 + 1) + ok) = __floats2bfloat162_rn(t1.x, t1.y);
            if (r0 + 2 < kRows) *(__nv_bfloat162*)(a_s + core_row(r0 + 2) + ok) = __floats2bfloat162_rn(t2.x, t2.y);
        }
    }
}

// named barrier of the transport warps with an OR of v over them
__device__ __forceinline__ bool stage_sync_or(int v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(v), "n"(kStageThreads)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_net_conv_tc(const __nv_bfloat162* __restrict__ in, float2* __restrict__ out,
                  const __nv_bfloat16* __restrict__ Bw, const float2* __restrict__ U32,
                  const int2* __restrict__ nbr, int64_t V, int* err, unsigned long long wait_ns) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    // afull: the transport warps filled A stage s; bfull: B_j landed in B stage
    // s; mdone: the MMAs of the stage's chunk completed (tcgen05.commit)
    __shared__ __align__(8) uint64_t afull[2], bfull[2], mdone[2];
    __shared__ uint32_t tslot;
    __shared__ uint32_t committed;   // chunks whose MMAs warp 15 has committed
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&afull[s])), "r"(kStageWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bfull[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mdone[s])));
        }
        committed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;

    const int64_t rows = 3 * V;
    const int64_t ntiles = (rows + kRows - 1) / kRows;
    uint32_t g = 0;  // chunks of the tiles before this one (stage = g & 1, use = g >> 1)
    int bad = 0;
    const int kq = lane & 3, sj = lane >> 2;
    for (int64_t tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x) {
        const int64_t row0 = tile * kRows;
        const int64_t xs0 = row0 / 3;
        const int off = (int)(row0 - 3 * xs0);
        int64_t xl = (row0 + kRows - 1) / 3;
        if (xl > V - 1) xl = V - 1;
        const int nsite = (int)(xl - xs0 + 1);
        // neighbour site of every (transport, site) of the tile
        int* Y = (int*)(base + kOffY);
        for (int i = tid; i < 9 * kSites; i += kThreads) {
            const int d = i / kSites, sl = i - d * kSites;
            if (sl < nsite) {
                const int64_t x = xs0 + sl;
                Y[i] = d == 0 ? (int)x : (d <= 4 ? __ldg(&nbr[x * 4 + d - 1].x) : __ldg(&nbr[x * 4 + d - 5].y));
            }
        }
        __syncthreads();
        if (warp < kStageWarps) {
            gather(base, 0, in, U32, xs0, nsite);
            gather(base, 1, in, U32, xs0, nsite);
            for (int j = 0; j < kChunks; ++j) {
                const uint32_t gj = g + (uint32_t)j, s = gj & 1u, u = gj >> 1;
                if (j + 1 < kChunks) asm volatile("cp.async.wait_group 1;" ::: "memory");
                else asm volatile("cp.async.wait_group 0;" ::: "memory");
                // the MMAs of chunk gj - 2 read this A stage: one thread waits
                // for their commit, the named barrier passes the news on (and
                // that every transport warp is done with chunk j - 1's raw rows)
                if (tid == 0 && gj >= 2 && !mbar_wait(su32(&mdone[s]), (u - 1) & 1u, wait_ns)) bad = 1;
                if (stage_sync_or(bad)) {
                    bad = 1;
                    break;
                }
                if (j + 2 < kChunks) gather(base, j + 2, in, U32, xs0, nsite);
                const int d = j >> 2;
                const unsigned char* P = base + kOffP + (j % 3) * kPBytes;
                const float2* Ub = (const float2*)(base + kOffU + (d & 1) * kUBytes);
                unsigned char* a_s = base + kOffA + s * kABytes;
                if (d == 0) stage_chunk<0>(P, Ub, a_s, warp, sj, kq, off, nsite);
                else if (d <= 4) stage_chunk<1>(P, Ub, a_s, warp, sj, kq, off, nsite);
                else stage_chunk<2>(P, Ub, a_s, warp, sj, kq, off, nsite);
                // the tensor core reads the stage through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&afull[s])) : "memory");
            }
        } else if (lane == 0) {
            // warp 15: B_j by bulk copy, then the chunk's MMAs once A and B are in
            for (int j = 0; j < kChunks; ++j) {
                const uint32_t gj = g + (uint32_t)j, s = gj & 1u, u = gj >> 1;
                if (gj >= 2 && !mbar_wait(su32(&mdone[s]), (u - 1) & 1u, wait_ns)) {  // B stage s free
                    bad = 1;
                    break;
                }
                const uint32_t bar = su32(&bfull[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBBytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        su32(base + kOffB + s * kBBytes)),
                    "l"(Bw + (size_t)j * (kBBytes / 2)), "r"(kBBytes), "r"(bar)
                    : "memory");
                if (!mbar_wait(su32(&afull[s]), u & 1u, wait_ns) || !mbar_wait(bar, u & 1u, wait_ns)) {
                    bad = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a0 = su32(base + kOffA + s * kABytes), b0 = su32(base + kOffB + s * kBBytes);
#pragma unroll
                for (int q = 0; q < 2; ++q)
#pragma unroll
                    for (int ks = 0; ks < kKC / 16; ++ks) {
                        const uint64_t ad = sdesc(a0 + q * 16 * kSBO + ks * 256);
                        const uint64_t bd = sdesc(b0 + ks * 256);
                        const uint32_t acc = (j > 0 || ks > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                tmem + (uint32_t)(q * kN)),
                            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                            : "memory");
                    }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        su32(&mdone[s]))
                    : "memory");
                committed = gj + 1;
            }
        }
        __syncwarp();
        // epilogue: the last chunk's commit covers every MMA of the tile
        if (tid == 0 && !bad) {
            const uint32_t gl = g + kChunks - 1;
            if (!mbar_wait(su32(&mdone[gl & 1u]), (gl >> 1) & 1u, wait_ns)) bad = 1;
        }
        g += kChunks;
        if (__syncthreads_or(bad)) bad = 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!bad) {
            // warp w reads lanes 32 (w % 4) .. + 31 of accumulator (w / 4) % 2, columns half w / 8
            const int q = (warp >> 2) & 1, wq = warp & 3, ch = warp >> 3;
            const int r = 128 * q + 32 * wq + lane;
            const int64_t p = row0 + r;
            const int64_t x = p / 3;
            const int a = (int)(p - 3 * x);
            for (int c = ch * (kN / 2); c < (ch + 1) * (kN / 2); c += 32) {
                uint32_t v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                      "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                      "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(q * kN + c)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (p < rows) {
                    float2* dst = out + (x * kRC + c / 2) * 3 + a;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        dst[3 * i] = make_float2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        if (__syncthreads_or(bad)) bad = 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (bad && tid == 0) atomicExch(err, 1);
    // every committed MMA has been waited for on the normal path; after a
    // timeout give the in-flight ones a bounded time before freeing
    __syncthreads();
    if (bad && tid == 0 && committed > 0) {
        const uint32_t gl = committed - 1;
        mbar_wait(su32(&mdone[gl & 1u]), (gl >> 1) & 1u, wait_ns);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// B chunks from the FP32 master weights WT[d][k][R] (complex, transposed)
__global__ void k_net_tc_pack(const float2* __restrict__ WT, __nv_bfloat16* __restrict__ Bw) {
    const int64_t n = (int64_t)kChunks * kN * kKC;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int chunk = (int)(e / (kN * kKC));
        const int rem = (int)(e - (int64_t)chunk * kN * kKC);
        const int np = rem / kKC, kp = rem - np * kKC;
        const int d = chunk >> 2, qt = chunk & 3;
        const int o = np >> 1, cout = np & 1, kk = kp >> 1, cin = kp & 1;
        const int k = kQ * qt + kk;
        const float2 w = WT[((int64_t)d * kRC + k) * kRC + o];
        const float v = cout == 0 ? (cin == 0 ? w.x : -w.y) : (cin == 0 ? w.y : w.x);
        Bw[(int64_t)chunk * (kBBytes / 2) + core_off(np, kp) / 2] = __float2bfloat16_rn(v);
    }
}

// ---------------------------------------------------------------------------
// The C -> 1 layer, weights first, on the tensor cores:
//   Phi[y][d][R][b] = sum_k W_d[R, k] in(y)[k, b]
// a real GEMM over rows p = 3 y + b with K = 2 x 96 (k' = 2 k + (re, im)) and
// N = 72 real outputs n' = 2 (4 d + R) + (re, im), padded to 80.  No
// transport: the A rows are the site's own activations (FP32, contiguous),
// converted to BF16 into the core-matrix layout.  128 rows per tile, one
// 80-column accumulator; 78 KB of shared memory and 128 TMEM columns, so two
// CTAs share an SM and overlap one's staging with the other's MMA/epilogue.
// ---------------------------------------------------------------------------
constexpr int kPhiRows = 128;
constexpr int kPhiK = 192;
constexpr int kPhiN = 80;
constexpr int kPhiOut = 72;
constexpr uint32_t kPhiSBO = (kPhiK / 8) * 128;          // 3072
constexpr uint32_t kPhiABytes = kPhiRows * kPhiK * 2;    // 49152
constexpr uint32_t kPhiBBytes = kPhiN * kPhiK * 2;       // 30720
constexpr size_t kPhiSmem = kPhiABytes + kPhiBBytes + 128;
constexpr int kPhiThreads = 256;
constexpr uint32_t kPhiIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kPhiN >> 3) << 17) |
                               ((uint32_t)(kPhiRows >> 4) << 24);

__device__ __forceinline__ uint32_t phi_off(int r, int k) {
    return (uint32_t)((r >> 3) * kPhiSBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint64_t phi_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(kPhiSBO >> 4) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(kPhiThreads, 2)
    k_net_phi_tc(const float2* __restrict__ in, float2* __restrict__ phi, const __nv_bfloat16* __restrict__ Bw,
                 int64_t V, int* err, unsigned long long wait_ns) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    unsigned char* sA = base;
    unsigned char* sB = base + kPhiABytes;
    __shared__ __align__(8) uint64_t bfull, mdone;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bfull)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mdone)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(su32(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&bfull)), "r"(kPhiBBytes)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         su32(sB)),
                     "l"(Bw), "r"(kPhiBBytes), "r"(su32(&bfull))
                     : "memory");
    }
    const int64_t rows = 3 * V;
    const int64_t ntiles = (rows + kPhiRows - 1) / kPhiRows;
    int bad = 0;
    uint32_t used = 0;  // tiles whose MMAs this CTA committed
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * kPhiRows;
        const int64_t y0 = row0 / 3;
        int64_t yl = (row0 + kPhiRows - 1) / 3;
        if (yl > V - 1) yl = V - 1;
        const int nsite = (int)(yl - y0 + 1);
        const int off = (int)(row0 - 3 * y0);
        // A: the tile's sites' activations, contiguous in memory ([y][k][b])
        // thread = (site, k): the three colours are three rows of the tile
        for (int e = tid; e < nsite * kRC; e += kPhiThreads) {
            const int sl = e / kRC, k = e - sl * kRC;
            const float2* src = in + ((y0 + sl) * kRC + k) * 3;
            const float2 v0 = __ldg(src), v1 = __ldg(src + 1), v2 = __ldg(src + 2);
            const int r = 3 * sl - off;
            if (r >= 0 && r < kPhiRows)
                *(__nv_bfloat162*)(sA + phi_off(r, 2 * k)) = __floats2bfloat162_rn(v0.x, v0.y);
            if (r + 1 >= 0 && r + 1 < kPhiRows)
                *(__nv_bfloat162*)(sA + phi_off(r + 1, 2 * k)) = __floats2bfloat162_rn(v1.x, v1.y);
            if (r + 2 < kPhiRows)
                *(__nv_bfloat162*)(sA + phi_off(r + 2, 2 * k)) = __floats2bfloat162_rn(v2.x, v2.y);
        }
        // rows past the last site (the last tile only) are zero
        for (int e = tid; e < kPhiRows * kRC; e += kPhiThreads) {
            const int r = e / kRC, k = e - r * kRC;
            if (row0 + r >= rows)
                *(__nv_bfloat162*)(sA + phi_off(r, 2 * k)) = __floats2bfloat162_rn(0.f, 0.f);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if ((used == 0 && !mbar_wait(su32(&bfull), 0u, wait_ns))) {
                bad = 1;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int ks = 0; ks < kPhiK / 16; ++ks) {
                    const uint64_t ad = phi_desc(su32(sA) + ks * 256);
                    const uint64_t bd = phi_desc(su32(sB) + ks * 256);
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(kPhiIdesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&mdone))
                             : "memory");
            }
        }
        if (__syncthreads_or(bad)) {
            bad = 1;
            break;
        }
        ++used;
        if (!mbar_wait(su32(&mdone), (used - 1) & 1u, wait_ns)) bad = 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!__syncthreads_or(bad)) {
            // warp w: lanes 32 (w % 4) .. + 31, columns 40 (w / 4) .. + 39
            const int wq = warp & 3, ch = warp >> 2;
            const int r = 32 * wq + lane;
            const int64_t p = row0 + r;
            const int64_t y = p / 3;
            const int b = (int)(p - 3 * y);
#pragma unroll
            for (int c8 = 0; c8 < 5; ++c8) {
                const int c = 40 * ch + 8 * c8;
                uint32_t v[8];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                               "=r"(v[6]), "=r"(v[7])
                             : "r"(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (p < rows) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int dR = c / 2 + i;
                        if (dR < kPhiOut / 2)
                            phi[(y * (kPhiOut / 2) + dR) * 3 + b] =
                                make_float2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
                    }
                }
            }
        } else {
            bad = 1;
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        if (__syncthreads_or(bad)) {
            bad = 1;
            break;
        }
    }
    if (bad && tid == 0) atomicExch(err, 1);
    // the weight copy must have landed before the CTA exits
    if (tid == 0 && used == 0) mbar_wait(su32(&bfull), 0u, wait_ns);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// B of the C -> 1 layer from its FP32 master weights WT[d][k][R] (R < 4)
__global__ void k_net_phi_pack(const float2* __restrict__ WT, __nv_bfloat16* __restrict__ Bw) {
    const int n = kPhiN * kPhiK;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int np = e / kPhiK, kp = e - np * kPhiK;
        float v = 0.f;
        if (np < kPhiOut) {
            const int o = np >> 1, cout = np & 1, k = kp >> 1, cin = kp & 1;
            const int d = o >> 2, R = o & 3;
            const float2 w = WT[((int64_t)d * kRC + k) * 4 + R];
            v = cout == 0 ? (cin == 0 ? w.x : -w.y) : (cin == 0 ? w.y : w.x);
        }
        Bw[phi_off(np, kp) / 2] = __float2bfloat16_rn(v);
    }
}

// ---------------------------------------------------------------------------
// The 1 -> C layer on the tensor cores: rows p = 3 x + a, K = 9 transports x
// 4 spins x (re, im) = 72 (padded to 80, the padding columns of A zero once),
// N = 192 (96 outputs x (re, im)); the threads stage U_d(x) in(x + d) for the
// 4 input rows (FP32 links and activations through L1); BF16 output in the
// layout the C -> C layer reads ([V][96][3] bf16x2).  128 rows per tile,
// weights resident (30 KB), 192 TMEM columns, two CTAs per SM.
// ---------------------------------------------------------------------------
constexpr int kL1Rows = 128;
constexpr int kL1K = 80;
constexpr uint32_t kL1SBO = (kL1K / 8) * 128;          // 1280
constexpr uint32_t kL1ABytes = kL1Rows * kL1K * 2;     // 20480
constexpr uint32_t kL1BBytes = kN * kL1K * 2;          // 30720
constexpr size_t kL1Smem = kL1ABytes + kL1BBytes + 128;
constexpr int kL1Threads = 256;
constexpr uint32_t kL1Idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                              ((uint32_t)(kL1Rows >> 4) << 24);

__device__ __forceinline__ uint32_t l1_off(int r, int k) {
    return (uint32_t)((r >> 3) * kL1SBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint64_t l1_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(kL1SBO >> 4) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(kL1Threads, 2)
    k_net_l1_tc(const float2* __restrict__ in, __nv_bfloat162* __restrict__ out, const __nv_bfloat16* __restrict__ Bw,
                const float2* __restrict__ U32, const int2* __restrict__ nbr, int64_t V, int* err,
                unsigned long long wait_ns) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    unsigned char* sA = base;
    unsigned char* sB = base + kL1ABytes;
    __shared__ __align__(8) uint64_t bfull, mdone;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bfull)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mdone)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // the padding columns 72..79 of A stay zero
    for (int r = tid; r < kL1Rows; r += kL1Threads) {
        *(uint4*)(sA + l1_off(r, 72)) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&bfull)), "r"(kL1BBytes)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         su32(sB)),
                     "l"(Bw), "r"(kL1BBytes), "r"(su32(&bfull))
                     : "memory");
    }
    const int64_t rows = 3 * V;
    const int64_t ntiles = (rows + kL1Rows - 1) / kL1Rows;
    int bad = 0;
    uint32_t used = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * kL1Rows;
        const int64_t x0 = row0 / 3;
        int64_t xl = (row0 + kL1Rows - 1) / 3;
        if (xl > V - 1) xl = V - 1;
        const int nsite = (int)(xl - x0 + 1);
        const int off = (int)(row0 - 3 * x0);
        // A: item = (site, transport): 4 input rows x 3 colours
        for (int e = tid; e < nsite * 9; e += kL1Threads) {
            const int sl = e / 9, d = e - sl * 9;
            const int64_t x = x0 + sl;
            int64_t y = x;
            const float2* uu = nullptr;
            bool dag = false;
            if (d >= 1 && d <= 4) {
                y = __ldg(&nbr[x * 4 + d - 1].x);
                uu = U32 + (x * 4 + d - 1) * 9;
            } else if (d >= 5) {
                y = __ldg(&nbr[x * 4 + d - 5].y);
                uu = U32 + (y * 4 + d - 5) * 9;
                dag = true;
            }
            float2 u[9];
            if (uu) {
#pragma unroll
                for (int i = 0; i < 9; ++i) u[i] = __ldg(uu + i);
            }
            const float2* src = in + y * 12;
            const int r0 = 3 * sl - off;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 p0 = __ldg(src + 3 * k), p1 = __ldg(src + 3 * k + 1), p2 = __ldg(src + 3 * k + 2);
                float2 t[3];
                if (!uu) {
                    t[0] = p0;
                    t[1] = p1;
                    t[2] = p2;
                } else if (!dag) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float2 q0 = cmul(u[3 * a], p0), q1 = cmul(u[3 * a + 1], p1), q2 = cmul(u[3 * a + 2], p2);
                        t[a] = make_float2(q0.x + q1.x + q2.x, q0.y + q1.y + q2.y);
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float2 q0 = cmulc(u[a], p0), q1 = cmulc(u[3 + a], p1), q2 = cmulc(u[6 + a], p2);
                        t[a] = make_float2(q0.x + q1.x + q2.x, q0.y + q1.y + q2.y);
                    }
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int r = r0 + a;
                    if (r >= 0 && r < kL1Rows)
                        *(__nv_bfloat162*)(sA + l1_off(r, 2 * (4 * d + k))) = __floats2bfloat162_rn(t[a].x, t[a].y);
                }
            }
        }
        // rows past the last site (the last tile only) are zero
        for (int e = tid; e < kL1Rows * 36; e += kL1Threads) {
            const int r = e / 36, q = e - r * 36;
            if (row0 + r >= rows) *(__nv_bfloat162*)(sA + l1_off(r, 2 * q)) = __floats2bfloat162_rn(0.f, 0.f);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if (used == 0 && !mbar_wait(su32(&bfull), 0u, wait_ns)) {
                bad = 1;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int ks = 0; ks < kL1K / 16; ++ks) {
                    const uint64_t ad = l1_desc(su32(sA) + ks * 256);
                    const uint64_t bd = l1_desc(su32(sB) + ks * 256);
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(kL1Idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&mdone))
                             : "memory");
            }
        }
        if (__syncthreads_or(bad)) {
            bad = 1;
            break;
        }
        ++used;
        if (!mbar_wait(su32(&mdone), (used - 1) & 1u, wait_ns)) bad = 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!__syncthreads_or(bad)) {
            // warp w: lanes 32 (w % 4) .. + 31, columns 96 (w / 4) .. + 95
            const int wq = warp & 3, ch = warp >> 2;
            const int r = 32 * wq + lane;
            const int64_t p = row0 + r;
            const int64_t x = p / 3;
            const int a = (int)(p - 3 * x);
            for (int c = 96 * ch; c < 96 * ch + 96; c += 32) {
                uint32_t v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                      "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                      "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (p < rows) {
                    __nv_bfloat162* dst = out + (x * kRC + c / 2) * 3 + a;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        dst[3 * i] = __floats2bfloat162_rn(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
                }
            }
        } else {
            bad = 1;
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        if (__syncthreads_or(bad)) {
            bad = 1;
            break;
        }
    }
    if (bad && tid == 0) atomicExch(err, 1);
    if (tid == 0 && used == 0) mbar_wait(su32(&bfull), 0u, wait_ns);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// B of the 1 -> C layer from its FP32 master weights WT[d][k][R] (k < 4)
__global__ void k_net_l1_pack(const float2* __restrict__ WT, __nv_bfloat16* __restrict__ Bw) {
    const int n = kN * kL1K;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int np = e / kL1K, kp = e - np * kL1K;
        float v = 0.f;
        if (kp < 72) {
            const int o = np >> 1, cout = np & 1, q = kp >> 1, cin = kp & 1;
            const int d = q >> 2, k = q & 3;
            const float2 w = WT[((int64_t)d * 4 + k) * kRC + o];
            v = cout == 0 ? (cin == 0 ? w.x : -w.y) : (cin == 0 ? w.y : w.x);
        }
        Bw[l1_off(np, kp) / 2] = __float2bfloat16_rn(v);
    }
}

// Failure-detection self-test: one thread waits, through the same bounded
// mbar_wait as the kernels above, on an mbarrier that nothing ever arrives
// at; the wait runs out after wait_ns and the kernel records GS_TIMEOUT.
__global__ void k_selftest_mbar_timeout(int* err, unsigned long long wait_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        if (!mbar_wait(su32(&bar), 0u, wait_ns)) atomicExch(err, (int)GS_TIMEOUT);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(su32(&bar)));
    }
}

}  // namespace

size_t net_tc_weight_elems() { return (size_t)kChunks * kN * kKC; }

gs_status net_tc_pack(gs_ctx* c, const float2* WT, __nv_bfloat16* Bw) {
    k_net_tc_pack<<<grid_for((int64_t)net_tc_weight_elems(), 256, c->num_sms * 4), 256, 0, c->stream>>>(WT, Bw);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

size_t net_phi_weight_elems() { return (size_t)kPhiN * kPhiK; }
size_t net_l1_weight_elems() { return (size_t)kN * kL1K; }

gs_status net_l1_pack(gs_ctx* c, const float2* WT, __nv_bfloat16* Bw) {
    k_net_l1_pack<<<grid_for(kN * kL1K, 256, 64), 256, 0, c->stream>>>(WT, Bw);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status net_l1_tc(gs_ctx* c, const float2* in, __nv_bfloat162* out, const __nv_bfloat16* Bw, const float2* U32,
                    const int2* nbr, int64_t V, int* err) {
    GS_CUDA(c, cudaFuncSetAttribute(k_net_l1_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kL1Smem));
    const int64_t ntiles = (3 * V + kL1Rows - 1) / kL1Rows;
    const int64_t cap = 2LL * c->num_sms;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    k_net_l1_tc<<<grid, kL1Threads, kL1Smem, c->stream>>>(in, out, Bw, U32, nbr, V, err, c->wait_ns);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status net_phi_pack(gs_ctx* c, const float2* WT, __nv_bfloat16* Bw) {
    k_net_phi_pack<<<grid_for(kPhiN * kPhiK, 256, 64), 256, 0, c->stream>>>(WT, Bw);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status net_phi_tc(gs_ctx* c, const float2* in, float2* phi, const __nv_bfloat16* Bw, int64_t V, int* err) {
    GS_CUDA(c, cudaFuncSetAttribute(k_net_phi_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPhiSmem));
    const int64_t ntiles = (3 * V + kPhiRows - 1) / kPhiRows;
    const int64_t cap = 2LL * c->num_sms;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    k_net_phi_tc<<<grid, kPhiThreads, kPhiSmem, c->stream>>>(in, phi, Bw, V, err, c->wait_ns);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status net_conv_tc(gs_ctx* c, const __nv_bfloat162* in, float2* out, const __nv_bfloat16* Bw, const float2* U32,
                      const int2* nbr, int64_t V, int* err) {
    GS_CUDA(c, cudaFuncSetAttribute(k_net_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    const int64_t ntiles = (3 * V + kRows - 1) / kRows;
    const int grid = (int)(ntiles < c->num_sms ? ntiles : c->num_sms);
    k_net_conv_tc<<<grid, kThreads, kSmem, c->stream>>>(in, out, Bw, U32, nbr, V, err, c->wait_ns);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// Runs k_selftest_mbar_timeout; *err_dev receives GS_TIMEOUT when the wait ran out.
gs_status selftest_mbar_timeout(gs_ctx* c, int* err_dev) {
    k_selftest_mbar_timeout<<<1, 32, 0, c->stream>>>(err_dev, c->wait_ns);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

}  // namespace gs
