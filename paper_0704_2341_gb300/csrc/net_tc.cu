// The C -> C layer of the learned preconditioner (C = 24) on the fifth-generation
// tensor cores: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in
// tensor memory), weights moved by the bulk-copy engine, transported
// activations staged into shared memory by the CTA's threads.
//
// The layer  out(x)[R, a] = sum_d sum_k W_d[R, k] (U_d(x) in(x + d))[k, a]
// is a real GEMM over rows p = 3 x + a (site, colour):
//   A[p, k'] = Re / Im of T_d(x)[k, a],  T_d(x) = U_d(x) in(x + d)
//   B[n', k'] = the real form of W_d:  out_re = W_re T_re - W_im T_im,
//               out_im = W_im T_re + W_re T_im
// with n' = 2 R + (re, im), k' = (d, half, 2 kk + (re, im)), k = 48 half + kk.
// M = 256 rows per tile (two 128-lane accumulators), N = 192, K = 9 x 192,
// taken in 18 chunks of 96 (one transport, 48 input rows).  Operands are in
// the no-swizzle K-major core-matrix layout: an 8-row x 16-byte core matrix
// is 128 contiguous bytes, core matrices adjacent in K are 128 bytes apart
// (leading byte offset), 8-row groups 1536 bytes apart (stride byte offset).
//
// Pipeline (two stages): for chunk j the threads build A_j while the tensor
// core runs chunk j - 1; one thread starts the bulk copy of B_j and, after
// the block barrier, issues the 12 MMAs of the chunk and commits them to the
// stage's mbarrier.  Every wait is bounded (1 s of global time); on a
// timeout the kernel stops, frees its tensor memory and raises err.
#include <cuda_bf16.h>
#include <stdint.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kRows = 256;                       // GEMM rows per tile
constexpr int kRC = 96;                          // 4 C, C = 24
constexpr int kN = 192;                          // real output columns
constexpr int kKC = 96;                          // real K per chunk
constexpr int kChunks = 18;                      // 9 transports x 2 halves
constexpr uint32_t kSBO = (kKC / 8) * 128;       // 1536
constexpr uint32_t kABytes = kRows * kKC * 2;    // 49152
constexpr uint32_t kBBytes = kN * kKC * 2;       // 36864
constexpr int kThreads = 256;
constexpr size_t kSmem = 2 * (size_t)(kABytes + kBBytes) + 256;

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
// bounded wait: true when the phase of the given parity has completed
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = gtime();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u && gtime() - t0 > 1000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // conj(a) b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_net_conv_tc(const float2* __restrict__ in, float2* __restrict__ out, const __nv_bfloat16* __restrict__ Bw,
                  const float2* __restrict__ U32, const int2* __restrict__ nbr, int64_t V, int* err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    // stage s: A at base + s kABytes, B at base + 2 kABytes + s kBBytes
    __shared__ __align__(8) uint64_t bfull[2], mdone[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bfull[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mdone[s])));
        }
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
    uint32_t g = 0;      // chunks issued so far (stage = g & 1, use = g >> 1)
    int bad = 0;
    const int kq = lane & 3, sj = lane >> 2;
    for (int64_t tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x) {
        const int64_t row0 = tile * kRows;
        const int64_t xs0 = row0 / 3;
        for (int j = 0; j < kChunks; ++j, ++g) {
            const uint32_t s = g & 1u, u = g >> 1;
            if (g >= 2 && !mbar_wait(su32(&mdone[s]), (u - 1) & 1u)) bad = 1;
            const int d = j >> 1, h = j & 1;
            if (tid == 0 && !bad) {
                const uint32_t bar = su32(&bfull[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBBytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        su32(base + 2 * kABytes + s * kBBytes)),
                    "l"(Bw + (size_t)j * (kBBytes / 2)), "r"(kBBytes), "r"(bar)
                    : "memory");
            }
            // A chunk: warp items = (group of 8 sites) x (group of 4 input rows)
            unsigned char* a_s = base + s * kABytes;
            for (int wi = warp; wi < 11 * 12; wi += kThreads / 32) {
                const int sg = wi / 12, kg = wi - sg * 12;
                const int64_t x = xs0 + 8 * sg + sj;
                const int64_t r0 = 3 * x - row0;
                if (r0 >= kRows) continue;
                const int kk = 4 * kg + kq, k = 48 * h + kk;
                float2 t[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                if (x < V) {
                    int64_t y = x;
                    const float2* uu = nullptr;
                    bool dag = false;
                    if (d >= 1 && d <= 4) {
                        y = __ldg(&nbr[x * 4 + (d - 1)].x);
                        uu = U32 + (x * 4 + (d - 1)) * 9;
                    } else if (d >= 5) {
                        y = __ldg(&nbr[x * 4 + (d - 5)].y);
                        uu = U32 + (y * 4 + (d - 5)) * 9;
                        dag = true;
                    }
                    const float2* src = in + (y * kRC + k) * 3;
                    const float2 p0 = __ldg(src), p1 = __ldg(src + 1), p2 = __ldg(src + 2);
                    if (!uu) {
                        t[0] = p0;
                        t[1] = p1;
                        t[2] = p2;
                    } else if (!dag) {
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float2 q0 = cmul(__ldg(uu + 3 * a), p0), q1 = cmul(__ldg(uu + 3 * a + 1), p1),
                                         q2 = cmul(__ldg(uu + 3 * a + 2), p2);
                            t[a] = make_float2(q0.x + q1.x + q2.x, q0.y + q1.y + q2.y);
                        }
                    } else {
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float2 q0 = cmulc(__ldg(uu + a), p0), q1 = cmulc(__ldg(uu + 3 + a), p1),
                                         q2 = cmulc(__ldg(uu + 6 + a), p2);
                            t[a] = make_float2(q0.x + q1.x + q2.x, q0.y + q1.y + q2.y);
                        }
                    }
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int64_t r = r0 + a;
                    if (r >= 0 && r < kRows)
                        *(__nv_bfloat162*)(a_s + core_off((int)r, 2 * kk)) = __floats2bfloat162_rn(t[a].x, t[a].y);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (__syncthreads_or(bad)) {
                bad = 1;
                break;
            }
            if (tid == 0) {
                if (!mbar_wait(su32(&bfull[s]), u & 1u)) {
                    bad = 1;
                } else {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t a0 = su32(base + s * kABytes), b0 = su32(base + 2 * kABytes + s * kBBytes);
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
                }
            }
        }
        if (bad) break;
        // epilogue: the last chunk's commit covers every MMA of the tile
        {
            const uint32_t gl = g - 1, s = gl & 1u, u = gl >> 1;
            if (!mbar_wait(su32(&mdone[s]), u & 1u)) bad = 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!bad) {
            const int q = warp >> 2, wq = warp & 3;
            const int r = 128 * q + 32 * wq + lane;
            const int64_t p = row0 + r;
            const int64_t x = p / 3;
            const int a = (int)(p - 3 * x);
            for (int c = 0; c < kN; c += 32) {
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
    if (bad && tid == 0) atomicExch(err, 1);
    // every committed MMA has been waited for on the normal path; after a
    // timeout give the in-flight ones a bounded time before freeing
    if (bad && tid == 0 && g > 0) {
        const uint32_t gl = g - 1;
        mbar_wait(su32(&mdone[gl & 1u]), (gl >> 1) & 1u);
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
        const int d = chunk >> 1, h = chunk & 1;
        const int o = np >> 1, cout = np & 1, kk = kp >> 1, cin = kp & 1;
        const int k = 48 * h + kk;
        const float2 w = WT[((int64_t)d * kRC + k) * kRC + o];
        const float v = cout == 0 ? (cin == 0 ? w.x : -w.y) : (cin == 0 ? w.y : w.x);
        Bw[(int64_t)chunk * (kBBytes / 2) + core_off(np, kp) / 2] = __float2bfloat16_rn(v);
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

gs_status net_conv_tc(gs_ctx* c, const float2* in, float2* out, const __nv_bfloat16* Bw, const float2* U32,
                      const int2* nbr, int64_t V, int* err) {
    GS_CUDA(c, cudaFuncSetAttribute(k_net_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    const int64_t ntiles = (3 * V + kRows - 1) / kRows;
    const int grid = (int)(ntiles < c->num_sms ? ntiles : c->num_sms);
    k_net_conv_tc<<<grid, kThreads, kSmem, c->stream>>>(in, out, Bw, U32, nbr, V, err);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

}  // namespace gs
