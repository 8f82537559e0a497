// Gauge-equivariant linear convolutional network: the learned preconditioner
// M ~ D_rr^-1 of the inner solve (forward, backward, Adam training step,
// inference) and flexible GMRES with M as right preconditioner.
//
// Layer (C_in -> C_out channels, activations [site][channel][spin][colour]):
//   out(x)[R, a] = sum_{d=0..8} sum_k W_d[R, k] (U_d(x) in(x + d))[k, a]
// with k = (channel, spin) of the input, R = (channel, spin) of the output and
// the nine parallel transports d = 0 (identity), 1 + mu (U_mu(x) in(x+mu)),
// 5 + mu (U_mu(x-mu)^dag in(x-mu)).  The network is 1 -> C -> C -> 1; its
// input is the rest-set vector embedded in the lattice (zero on the coarse
// sites), its output is read on the rest set.
//
// GB300 mapping: a block computes one tile of 8 sites x 3 colours (24 GEMM
// columns) for all output rows: the transported neighbour activations of the
// tile go to shared memory, each thread owns one output row and streams the
// weight column W_d[R, :] (stored transposed, [d][k][R], so a warp reads
// consecutive rows), accumulating 24 complex outputs in FP32 registers.
// Weights are kept in FP32 (training master) and BF16 (inference).
// Backward: the input gradient is the same convolution with W'_d =
// (W_{reverse(d)})^H; the weight gradient g_W_d = sum_{x,a} g_out(x) T_d(x)^H
// is accumulated per (site chunk, d) block and reduced over chunks in a fixed
// order (deterministic).
#include <cuda_bf16.h>
#include <math.h>

#include <complex>
#include <vector>

#include "gs_internal.cuh"

struct gs_net {
    int C = 0;
    float2* W[3] = {};       // FP32 master, transposed [9][K][R]
    __nv_bfloat162* Wb[3] = {};  // BF16 copy
    float2* G[3] = {};       // gradients (same layout)
    float2* Wp = nullptr;    // transformed weights of the backward input conv (max size)
    float* m[3] = {};        // Adam moments (as floats)
    float* v[3] = {};
    int64_t nel[3] = {};     // complex entries per layer
    long long step = 0;
    // scratch sized for a lattice
    int64_t capV = 0;
    float2* act[4] = {};     // act0 [V][4][3], act1/2 [V][4C][3], act3 [V][4][3]
    float2* gact[2] = {};    // gradient buffers [V][4C][3]
    float2* partial = nullptr;  // [chunks][9][K][R]
    float2* U32 = nullptr;      // FP32 links [V][4][9] (site order) of the last context
    const void* U32_src = nullptr;
    float* red = nullptr;       // small reduction scratch
    unsigned int* counter = nullptr;
    float* host_red = nullptr;
    __nv_bfloat16* Btc = nullptr;   // C -> C weights packed for the tensor cores (C = 24)
    __nv_bfloat16* Bphi = nullptr;  // C -> 1 weights packed for the tensor cores (C = 24)
    __nv_bfloat16* Bl1 = nullptr;   // 1 -> C weights packed for the tensor cores (C = 24)
    bool tc_dirty = true;           // Btc out of date with W[1]
    int* tc_err = nullptr;          // mapped host word raised by the tensor-core kernel
    int* tc_err_dev = nullptr;
};

namespace gs {
namespace {

constexpr int kTS = 8;           // sites per tile
constexpr int kNCol = kTS * 3;   // GEMM columns per tile
constexpr int kChunks = 32;      // site chunks of the weight gradient

__device__ __forceinline__ float2 cm(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cfma2(float2& acc, float2 a, float2 b) {  // acc += a b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmaconj(float2& acc, float2 a, float2 b) {  // acc += a conj(b)
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.y, b.x, acc.y);
    acc.y = fmaf(-a.x, b.y, acc.y);
}

__device__ __forceinline__ float2 loadw(const float2* W, int64_t i) { return __ldg(W + i); }
__device__ __forceinline__ float2 loadw(const __nv_bfloat162* W, int64_t i) {
    return __bfloat1622float2(W[i]);
}

// transported activations of one tile for transport d:
// T[k][s*3 + a] = (U_d(x_s) in(x_s + d))[k, a]; threads stride over (s, k)
template <int K>
__device__ __forceinline__ void stage_tile(const float2* __restrict__ in, const float2* __restrict__ U32,
                                           const int2* __restrict__ nbr, int64_t base, int64_t V, int d,
                                           float2 (*T)[kNCol]) {
    for (int e = threadIdx.x; e < kTS * K; e += blockDim.x) {
        const int s = e / K, k = e - s * K;
        const int64_t x = base + s;
        float2 t0 = make_float2(0.f, 0.f), t1 = t0, t2 = t0;
        if (x < V) {
            int64_t y = x;
            const float2* u = nullptr;
            bool dag = false;
            if (d >= 1 && d <= 4) {
                const int mu = d - 1;
                y = __ldg(nbr + x * 4 + mu).x;
                u = U32 + (x * 4 + mu) * 9;
            } else if (d >= 5) {
                const int mu = d - 5;
                y = __ldg(nbr + x * 4 + mu).y;
                u = U32 + (y * 4 + mu) * 9;
                dag = true;
            }
            const float2* src = in + (y * K + k) * 3;
            const float2 p0 = src[0], p1 = src[1], p2 = src[2];
            if (!u) {
                t0 = p0;
                t1 = p1;
                t2 = p2;
            } else if (!dag) {
                float2 r[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cfma2(r[a], __ldg(u + 3 * a + 0), p0);
                    cfma2(r[a], __ldg(u + 3 * a + 1), p1);
                    cfma2(r[a], __ldg(u + 3 * a + 2), p2);
                }
                t0 = r[0];
                t1 = r[1];
                t2 = r[2];
            } else {  // U^dag: row a = conj of column a
                float2 r[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float2 c0 = __ldg(u + 0 + a), c1 = __ldg(u + 3 + a), c2 = __ldg(u + 6 + a);
                    cfma2(r[a], make_float2(c0.x, -c0.y), p0);
                    cfma2(r[a], make_float2(c1.x, -c1.y), p1);
                    cfma2(r[a], make_float2(c2.x, -c2.y), p2);
                }
                t0 = r[0];
                t1 = r[1];
                t2 = r[2];
            }
        }
        T[k][s * 3 + 0] = t0;
        T[k][s * 3 + 1] = t1;
        T[k][s * 3 + 2] = t2;
    }
}

// out[V][R4][3] = sum_d W_d T_d ; threads: one per output row (>= 32)
template <int CIN, int COUT, class WT>
__global__ void k_net_conv(const float2* __restrict__ in, float2* __restrict__ out, const WT* __restrict__ W,
                           const float2* __restrict__ U32, const int2* __restrict__ nbr, int64_t V) {
    constexpr int K = 4 * CIN, R4 = 4 * COUT;
    __shared__ float2 T[K][kNCol];
    const int R = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * kTS; base < V; base += (int64_t)gridDim.x * kTS) {
        float2 acc[kNCol];
#pragma unroll
        for (int q = 0; q < kNCol; ++q) acc[q] = make_float2(0.f, 0.f);
        for (int d = 0; d < 9; ++d) {
            stage_tile<K>(in, U32, nbr, base, V, d, T);
            __syncthreads();
            if (R < R4) {
                const WT* wd = W + (int64_t)d * K * R4 + R;
                for (int k = 0; k < K; ++k) {
                    const float2 w = loadw(wd, (int64_t)k * R4);
#pragma unroll
                    for (int q = 0; q < kNCol; ++q) cfma2(acc[q], w, T[k][q]);
                }
            }
            __syncthreads();
        }
        if (R < R4) {
#pragma unroll
            for (int s = 0; s < kTS; ++s) {
                const int64_t x = base + s;
                if (x < V) {
                    float2* dst = out + (x * R4 + R) * 3;
                    dst[0] = acc[s * 3 + 0];
                    dst[1] = acc[s * 3 + 1];
                    dst[2] = acc[s * 3 + 2];
                }
            }
        }
    }
}

// The C -> 1 layer weights first: W_d acts on (channel, spin) and U_d on
// colour, so  out(x) = sum_d U_d(x) Phi_d(x + d)  with  Phi_d(y) = W_d in(y);
// Phi comes from the tensor-core kernel k_net_phi_tc (net_tc.cu).
// out(x)[R, a] = sum_d (U_d(x) Phi_d(x + d)[R])[a]; one thread per (site, R)
__global__ void k_net_phi_gather(const float2* __restrict__ phi, float2* __restrict__ out,
                                 const float2* __restrict__ U32, const int2* __restrict__ nbr, int64_t V) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V * 4; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i >> 2;
        const int R = (int)(i & 3);
        const float2* p0 = phi + ((x * 9) * 4 + R) * 3;
        float2 acc[3] = {p0[0], p0[1], p0[2]};
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int2 nb = __ldg(nbr + x * 4 + mu);
            {   // +mu: U_mu(x) Phi_{1+mu}(x + mu)
                const float2* p = phi + (((int64_t)nb.x * 9 + 1 + mu) * 4 + R) * 3;
                const float2* u = U32 + (x * 4 + mu) * 9;
                const float2 q0 = p[0], q1 = p[1], q2 = p[2];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cfma2(acc[a], __ldg(u + 3 * a), q0);
                    cfma2(acc[a], __ldg(u + 3 * a + 1), q1);
                    cfma2(acc[a], __ldg(u + 3 * a + 2), q2);
                }
            }
            {   // -mu: U_mu(x - mu)^dag Phi_{5+mu}(x - mu)
                const float2* p = phi + (((int64_t)nb.y * 9 + 5 + mu) * 4 + R) * 3;
                const float2* u = U32 + ((int64_t)nb.y * 4 + mu) * 9;
                const float2 q0 = p[0], q1 = p[1], q2 = p[2];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float2 c0 = __ldg(u + a), c1 = __ldg(u + 3 + a), c2 = __ldg(u + 6 + a);
                    cfma2(acc[a], make_float2(c0.x, -c0.y), q0);
                    cfma2(acc[a], make_float2(c1.x, -c1.y), q1);
                    cfma2(acc[a], make_float2(c2.x, -c2.y), q2);
                }
            }
        }
        float2* dst = out + (x * 4 + R) * 3;
        dst[0] = acc[0];
        dst[1] = acc[1];
        dst[2] = acc[2];
    }
}

// partial[chunk][d][k][R] = sum over the chunk's sites and colours of
// g_out(x)[R, a] conj(T_d(x)[k, a]);  grid = (kChunks, 9)
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_net_gradw(const float2* __restrict__ in, const float2* __restrict__ gout,
                                                  float2* __restrict__ partial, const float2* __restrict__ U32,
                                                  const int2* __restrict__ nbr, int64_t V) {
    constexpr int K = 4 * CIN, R4 = 4 * COUT, NE = K * R4;
    constexpr int PER = (NE + 255) / 256;
    __shared__ float2 T[K][kNCol];
    __shared__ float2 Gs[R4][kNCol];
    const int chunk = blockIdx.x, d = blockIdx.y;
    const int64_t tiles = (V + kTS - 1) / kTS;
    const int64_t t0 = tiles * chunk / gridDim.x, t1 = tiles * (chunk + 1) / gridDim.x;
    float2 acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t base = tile * kTS;
        stage_tile<K>(in, U32, nbr, base, V, d, T);
        for (int e = threadIdx.x; e < R4 * kNCol; e += blockDim.x) {
            const int R = e / kNCol, col = e - R * kNCol;
            const int s = col / 3, a = col - s * 3;
            const int64_t x = base + s;
            Gs[R][col] = (x < V) ? gout[(x * R4 + R) * 3 + a] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = threadIdx.x + q * 256;
            if (e < NE) {
                const int k = e / R4, R = e - k * R4;
                float2 s = acc[q];
#pragma unroll 8
                for (int col = 0; col < kNCol; ++col) cfmaconj(s, Gs[R][col], T[k][col]);
                acc[q] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = threadIdx.x + q * 256;
        if (e < NE) partial[((int64_t)chunk * 9 + d) * NE + e] = acc[q];
    }
}

// G (+)= sum over chunks of the partials (fixed order)
__global__ void k_net_reduce(const float2* __restrict__ partial, float2* __restrict__ G, int64_t nel,
                             int chunks, int accumulate) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nel;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 s = accumulate ? G[i] : make_float2(0.f, 0.f);
        for (int c = 0; c < chunks; ++c) {
            const float2 p = partial[(int64_t)c * nel + i];
            s.x += p.x;
            s.y += p.y;
        }
        G[i] = s;
    }
}

// W' of the backward input convolution: W'T[d'][R][k] = conj(WT[d][k][R]),
// d' the reversed transport (0 -> 0, +mu <-> -mu)
__global__ void k_net_wprime(const float2* __restrict__ W, float2* __restrict__ Wp, int K, int R4) {
    const int64_t n = 9LL * K * R4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(i / ((int64_t)K * R4));
        const int64_t rem = i - (int64_t)d * K * R4;
        const int k = (int)(rem / R4), R = (int)(rem - (int64_t)k * R4);
        const int dp = d == 0 ? 0 : (d <= 4 ? d + 4 : d - 4);
        const float2 w = W[i];
        Wp[((int64_t)dp * R4 + R) * K + k] = make_float2(w.x, -w.y);
    }
}

// rest vector (label order, complex128 or complex64) -> whole lattice (site order), zero on b
__global__ void k_net_embed64(const double2* __restrict__ t, const int32_t* __restrict__ perm, int64_t nb,
                              int64_t nr, float2* __restrict__ full) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 12;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 12;
        const int c = (int)(i - k * 12);
        const double2 v = t[i];
        full[(int64_t)perm[nb + k] * 12 + c] = make_float2((float)v.x, (float)v.y);
    }
}
__global__ void k_net_embed32(const float2* __restrict__ t, const int32_t* __restrict__ perm, int64_t nb,
                              int64_t nr, float2* __restrict__ full) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 12;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 12;
        const int c = (int)(i - k * 12);
        full[(int64_t)perm[nb + k] * 12 + c] = t[i];
    }
}
__global__ void k_net_restrict64(const float2* __restrict__ full, const int32_t* __restrict__ perm,
                                 int64_t nb, int64_t nr, double2* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 12;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 12;
        const int c = (int)(i - k * 12);
        const float2 v = full[(int64_t)perm[nb + k] * 12 + c];
        y[i] = make_double2((double)v.x, (double)v.y);
    }
}

// ---------------------------------------------------------------------------
// FP32 vectors of the flexible GMRES: the low-precision stencil's layout,
// [6][n_r] float4 (float4 c of site k holds complexes 2c and 2c + 1), seen
// by the BLAS below as n_r x 12 complex numbers in one consistent order.
// ---------------------------------------------------------------------------
constexpr int kFgBlas = 256;
constexpr int kFgChunk = 8;

// v = s r (FP64 AoS rest vector -> FP32 layout)
__global__ void k_fg_pack(const double2* __restrict__ r, float4* __restrict__ v, int64_t nr, double sc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 6;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / nr, k = i - c * nr;
        const double2 a = r[k * 12 + 2 * c], b = r[k * 12 + 2 * c + 1];
        v[i] = make_float4((float)(sc * a.x), (float)(sc * a.y), (float)(sc * b.x), (float)(sc * b.y));
    }
}
__global__ void k_fg_unpack(const float4* __restrict__ v, double2* __restrict__ r, int64_t nr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 6;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / nr, k = i - c * nr;
        const float4 a = v[i];
        r[k * 12 + 2 * c] = make_double2(a.x, a.y);
        r[k * 12 + 2 * c + 1] = make_double2(a.z, a.w);
    }
}
// rest vector in the FP32 layout -> whole lattice (site order), zero on b
__global__ void k_net_embed_lp(const float4* __restrict__ v, const int32_t* __restrict__ perm, int64_t nb,
                               int64_t nr, float2* __restrict__ full) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 6;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / nr, k = i - c * nr;
        const float4 a = v[i];
        float2* dst = full + (int64_t)perm[nb + k] * 12 + 2 * c;
        dst[0] = make_float2(a.x, a.y);
        dst[1] = make_float2(a.z, a.w);
    }
}
__global__ void k_net_restrict_lp(const float2* __restrict__ full, const int32_t* __restrict__ perm, int64_t nb,
                                  int64_t nr, float4* __restrict__ v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 6;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / nr, k = i - c * nr;
        const float2* src = full + (int64_t)perm[nb + k] * 12 + 2 * c;
        const float2 a = src[0], b = src[1];
        v[i] = make_float4(a.x, a.y, b.x, b.y);
    }
}
// out[k] = <X_k, y> (k < nvec), FP32 products summed per thread, FP64 across
// threads and blocks; block (bx, chunk) takes vectors 8 chunk .. + 7 against
// one load of y; the last block adds the per-block partials in block order
__global__ void k_fg_multidot(const float2* __restrict__ X, int64_t ld, const float2* __restrict__ y, int64_t n,
                              int nvec, double2* out, double* partial, unsigned int* counter) {
    __shared__ double sm[kFgBlas / 32][2 * kFgChunk];
    __shared__ bool am_last;
    const int k0 = blockIdx.y * kFgChunk;
    const int nk = nvec - k0 < kFgChunk ? nvec - k0 : kFgChunk;
    float a[2 * kFgChunk];
#pragma unroll
    for (int q = 0; q < 2 * kFgChunk; ++q) a[q] = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 w = y[i];
#pragma unroll
        for (int q = 0; q < kFgChunk; ++q) {
            if (q < nk) {
                const float2 u = X[(int64_t)(k0 + q) * ld + i];
                a[2 * q] = fmaf(u.x, w.x, fmaf(u.y, w.y, a[2 * q]));
                a[2 * q + 1] = fmaf(u.x, w.y, fmaf(-u.y, w.x, a[2 * q + 1]));
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < 2 * kFgChunk; ++q) {
        double v = (double)a[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) sm[warp][q] = v;
    }
    __syncthreads();
    const unsigned nblocks = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) {
        for (int q = 0; q < nk; ++q) {
            double s0 = 0.0, s1 = 0.0;
            for (int w = 0; w < nw; ++w) {
                s0 += sm[w][2 * q];
                s1 += sm[w][2 * q + 1];
            }
            double* part = partial + ((int64_t)(k0 + q) * gridDim.x + blockIdx.x) * 2;
            part[0] = s0;
            part[1] = s1;
        }
        __threadfence();
        am_last = atomicAdd(counter, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int kk = threadIdx.x; kk < nvec; kk += blockDim.x) {
        double s0 = 0.0, s1 = 0.0;
        const double* part = partial + (int64_t)kk * gridDim.x * 2;
#pragma unroll 8
        for (unsigned b = 0; b < gridDim.x; ++b) {
            s0 += __ldcg(part + 2 * b);
            s1 += __ldcg(part + 2 * b + 1);
        }
        out[kk] = make_double2(s0, s1);
    }
    if (threadIdx.x == 0) *counter = 0u;
}
// y += sign sum_k coef[k] X_k (coefficients FP64 on the device)
__global__ void k_fg_multiaxpy(const float2* __restrict__ X, int64_t ld, int nvec, const double2* __restrict__ coef,
                               float2* __restrict__ y, int64_t n, float sign) {
    __shared__ float2 cf[kMaxRestart + 1];
    for (int k = threadIdx.x; k < nvec; k += blockDim.x) {
        const double2 c = coef[k];
        cf[k] = make_float2(sign * (float)c.x, sign * (float)c.y);
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 acc = y[i];
        for (int k = 0; k < nvec; ++k) {
            const float2 c = cf[k], u = X[(int64_t)k * ld + i];
            acc.x = fmaf(c.x, u.x, fmaf(-c.y, u.y, acc.x));
            acc.y = fmaf(c.x, u.y, fmaf(c.y, u.x, acc.y));
        }
        y[i] = acc;
    }
}
__global__ void k_fg_scale(const float2* __restrict__ x, float2* __restrict__ y, int64_t n, float a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = x[i];
        y[i] = make_float2(a * v.x, a * v.y);
    }
}

// loss of one sample: sums ||y_r - z||^2 and ||z||^2 into red[0..1]
// (last-block pattern), then g_y = coef (y - z) on r, 0 on b
__global__ void k_net_loss(const float2* __restrict__ yfull, const float2* __restrict__ z,
                           const int32_t* __restrict__ perm, int64_t nb, int64_t nr, float* red,
                           unsigned int* counter) {
    __shared__ float sm[2][32];
    __shared__ bool last;
    float a = 0.f, b = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 12;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 12;
        const int c = (int)(i - k * 12);
        const float2 y = yfull[(int64_t)perm[nb + k] * 12 + c], zz = z[i];
        const float dx = y.x - zz.x, dy = y.y - zz.y;
        a = fmaf(dx, dx, fmaf(dy, dy, a));
        b = fmaf(zz.x, zz.x, fmaf(zz.y, zz.y, b));
    }
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        sm[0][warp] = a;
        sm[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float s0 = 0.f, s1 = 0.f;
        for (int w = 0; w < nw; ++w) {
            s0 += sm[0][w];
            s1 += sm[1][w];
        }
        red[2 + 2 * blockIdx.x] = s0;
        red[3 + 2 * blockIdx.x] = s1;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        float s0 = 0.f, s1 = 0.f;
        // L2 loads (written before the counter reached gridDim.x), in flight together
#pragma unroll 8
        for (unsigned bl = 0; bl < gridDim.x; ++bl) {
            s0 += __ldcg(red + 2 + 2 * bl);
            s1 += __ldcg(red + 3 + 2 * bl);
        }
        red[0] = s0;
        red[1] = s1;
        *counter = 0u;
    }
}

__global__ void k_net_lossgrad(const float2* __restrict__ yfull, const float2* __restrict__ z,
                               const int32_t* __restrict__ perm, int64_t nb, int64_t nr,
                               const float* __restrict__ red, float scale, float2* __restrict__ gfull) {
    const float coef = 2.f * scale / red[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 12;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 12;
        const int c = (int)(i - k * 12);
        const int64_t f = (int64_t)perm[nb + k] * 12 + c;
        const float2 y = yfull[f], zz = z[i];
        gfull[f] = make_float2(coef * (y.x - zz.x), coef * (y.y - zz.y));
    }
}

// Adam on the real and imaginary parts; refreshes the BF16 copy
__global__ void k_net_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, __nv_bfloat16* __restrict__ wb, int64_t n, float lr,
                           float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void k_net_tobf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(w[i]);
}

__global__ void k_links32(const double2* __restrict__ U, float2* __restrict__ U32, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        U32[i] = make_float2((float)U[i].x, (float)U[i].y);
}

// layer shapes: 0: 1 -> C, 1: C -> C, 2: C -> 1
inline void layer_dims(int C, int l, int* cin, int* cout) {
    *cin = (l == 0) ? 1 : C;
    *cout = (l == 2) ? 1 : C;
}

template <int C, class WT>
void conv_dispatch_t(int cin, int cout, const float2* in, float2* out, const WT* W, const float2* U32,
                     const int2* nbr, int64_t V, int blocks, cudaStream_t s) {
    if (cin == 1 && cout == C) k_net_conv<1, C, WT><<<blocks, 4 * C < 32 ? 32 : 4 * C, 0, s>>>(in, out, W, U32, nbr, V);
    else if (cin == C && cout == C) k_net_conv<C, C, WT><<<blocks, 4 * C < 32 ? 32 : 4 * C, 0, s>>>(in, out, W, U32, nbr, V);
    else if (cin == C && cout == 1) k_net_conv<C, 1, WT><<<blocks, 32, 0, s>>>(in, out, W, U32, nbr, V);
    else if (cin == 1 && cout == 1) k_net_conv<1, 1, WT><<<blocks, 32, 0, s>>>(in, out, W, U32, nbr, V);
}

template <int C>
void gradw_dispatch_t(int cin, int cout, const float2* in, const float2* gout, float2* partial,
                      const float2* U32, const int2* nbr, int64_t V, cudaStream_t s) {
    dim3 g(kChunks, 9);
    if (cin == 1 && cout == C) k_net_gradw<1, C><<<g, 256, 0, s>>>(in, gout, partial, U32, nbr, V);
    else if (cin == C && cout == C) k_net_gradw<C, C><<<g, 256, 0, s>>>(in, gout, partial, U32, nbr, V);
    else if (cin == C && cout == 1) k_net_gradw<C, 1><<<g, 256, 0, s>>>(in, gout, partial, U32, nbr, V);
}

}  // namespace

static bool net_channels_ok(int C) { return C == 2 || C == 4 || C == 8 || C == 24; }

template <class WT>
static void conv_dispatch(int C, int cin, int cout, const float2* in, float2* out, const WT* W,
                          const float2* U32, const int2* nbr, int64_t V, int blocks, cudaStream_t s) {
    switch (C) {
        case 2: conv_dispatch_t<2, WT>(cin, cout, in, out, W, U32, nbr, V, blocks, s); break;
        case 4: conv_dispatch_t<4, WT>(cin, cout, in, out, W, U32, nbr, V, blocks, s); break;
        case 8: conv_dispatch_t<8, WT>(cin, cout, in, out, W, U32, nbr, V, blocks, s); break;
        default: conv_dispatch_t<24, WT>(cin, cout, in, out, W, U32, nbr, V, blocks, s); break;
    }
}

static void gradw_dispatch(int C, int cin, int cout, const float2* in, const float2* gout,
                           float2* partial, const float2* U32, const int2* nbr, int64_t V,
                           cudaStream_t s) {
    switch (C) {
        case 2: gradw_dispatch_t<2>(cin, cout, in, gout, partial, U32, nbr, V, s); break;
        case 4: gradw_dispatch_t<4>(cin, cout, in, gout, partial, U32, nbr, V, s); break;
        case 8: gradw_dispatch_t<8>(cin, cout, in, gout, partial, U32, nbr, V, s); break;
        default: gradw_dispatch_t<24>(cin, cout, in, gout, partial, U32, nbr, V, s); break;
    }
}

// scratch of a network for a lattice of V sites; FP32 links of the context
static gs_status net_prepare(gs_ctx* c, gs_net* nt) {
    const int64_t V = c->V;
    if (nt->capV < V) {
        for (auto& a : nt->act) cudaFree(a);
        for (auto& a : nt->gact) cudaFree(a);
        cudaFree(nt->U32);
        nt->U32 = nullptr;
        nt->U32_src = nullptr;
        const size_t big = (size_t)V * 4 * nt->C * 3 * sizeof(float2);
        const size_t sm = (size_t)V * 12 * sizeof(float2);
        if (cudaMalloc(&nt->act[0], sm) != cudaSuccess || cudaMalloc(&nt->act[1], big) != cudaSuccess ||
            cudaMalloc(&nt->act[2], big) != cudaSuccess || cudaMalloc(&nt->act[3], sm) != cudaSuccess ||
            cudaMalloc(&nt->gact[0], big) != cudaSuccess || cudaMalloc(&nt->gact[1], big) != cudaSuccess ||
            cudaMalloc(&nt->U32, (size_t)V * 36 * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            nt->capV = 0;
            return set_err(c, GS_ENOMEM, "allocating network activations failed");
        }
        nt->capV = V;
    }
    if (nt->U32_src != (const void*)c || !c->net_links_fresh) {
        k_links32<<<grid_for(V * 36, 256, c->num_sms * 8), 256, 0, c->stream>>>(c->U_abi, nt->U32, V * 36);
        c->launches++;
        GS_CHECK_LAUNCH(c);
        nt->U32_src = c;
        c->net_links_fresh = true;
    }
    return GS_OK;
}

// y_full = M(x_full) with BF16 (infer) or FP32 weights; acts kept in nt->act
static gs_status net_forward(gs_ctx* c, gs_net* nt, bool bf16) {
    const Plan* id = c->plans[0];
    const int64_t V = c->V;
    const int blocks = (int)((V + kTS - 1) / kTS);
    for (int l = 0; l < 3; ++l) {
        int cin, cout;
        layer_dims(nt->C, l, &cin, &cout);
        const bool tc = bf16 && nt->Btc && c->opt_net_kernel == 0;
        if (tc && nt->tc_dirty) {
            gs_status s;
            if ((s = net_l1_pack(c, nt->W[0], nt->Bl1)) != GS_OK) return s;
            if ((s = net_tc_pack(c, nt->W[1], nt->Btc)) != GS_OK) return s;
            if ((s = net_phi_pack(c, nt->W[2], nt->Bphi)) != GS_OK) return s;
            nt->tc_dirty = false;
        }
        if (tc && l == 0) {
            // 1 -> C on the tensor cores; its BF16 output (the C -> C layer's
            // input) is kept in act[1]'s memory
            gs_status s = net_l1_tc(c, nt->act[0], (__nv_bfloat162*)nt->act[1], nt->Bl1, nt->U32, id->nbr, V,
                                    nt->tc_err_dev);
            if (s != GS_OK) return s;
            continue;
        }
        if (tc && l == 1) {
            gs_status s;
            if ((s = net_conv_tc(c, (const __nv_bfloat162*)nt->act[1], nt->act[2], nt->Btc, nt->U32, id->nbr, V,
                                 nt->tc_err_dev)) != GS_OK)
                return s;
            continue;
        }
        if (tc && l == 2) {
            // weights first; Phi ([V][9][4][3]) in the training gradient buffer
            gs_status s = net_phi_tc(c, nt->act[2], nt->gact[0], nt->Bphi, V, nt->tc_err_dev);
            if (s != GS_OK) return s;
            k_net_phi_gather<<<grid_for(V * 4, 256, c->num_sms * 8), 256, 0, c->stream>>>(nt->gact[0], nt->act[3],
                                                                                      nt->U32, id->nbr, V);
            c->launches += 1;
            GS_CHECK_LAUNCH(c);
            continue;
        }
        if (bf16)
            conv_dispatch<__nv_bfloat162>(nt->C, cin, cout, nt->act[l], nt->act[l + 1], nt->Wb[l],
                                          nt->U32, id->nbr, V, blocks, c->stream);
        else
            conv_dispatch<float2>(nt->C, cin, cout, nt->act[l], nt->act[l + 1], nt->W[l], nt->U32,
                                  id->nbr, V, blocks, c->stream);
        c->launches++;
        GS_CHECK_LAUNCH(c);
    }
    return GS_OK;
}

// y = M(t) for a rest vector (FP64 in and out), BF16 weights
gs_status net_apply_rest(gs_ctx* c, gs_net* nt, const Plan* p, const double2* t, double2* y) {
    gs_status s = net_prepare(c, nt);
    if (s != GS_OK) return s;
    const int64_t V = c->V, nb = p->nb, nr = V - nb;
    GS_CUDA(c, cudaMemsetAsync(nt->act[0], 0, (size_t)V * 12 * sizeof(float2), c->stream));
    const int g = grid_for(nr * 12, 256, c->num_sms * 8);
    k_net_embed64<<<g, 256, 0, c->stream>>>(t, p->perm, nb, nr, nt->act[0]);
    c->launches++;
    if ((s = net_forward(c, nt, true)) != GS_OK) return s;
    k_net_restrict64<<<g, 256, 0, c->stream>>>(nt->act[3], p->perm, nb, nr, y);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}


// host launchers of the FP32 FGMRES BLAS
static gs_status fg_multidot(gs_ctx* c, const float2* X, int64_t ld, int nvec, const float2* y, int64_t n,
                             double2* out) {
    const int nchunks = (nvec + kFgChunk - 1) / kFgChunk;
    int64_t cap = (int64_t)c->num_sms * 8 / nchunks;
    if (cap < 64) cap = 64;
    if (cap > kRedScratchDoubles / (2 * nvec)) cap = kRedScratchDoubles / (2 * nvec);
    dim3 g(grid_for(n, kFgBlas, (int)cap), nchunks);
    k_fg_multidot<<<g, kFgBlas, 0, c->stream>>>(X, ld, y, n, nvec, out, c->fg_red.partial, c->fg_red.counter);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}
static gs_status fg_multiaxpy(gs_ctx* c, const float2* X, int64_t ld, int nvec, const double2* coef, float2* y,
                              int64_t n, float sign) {
    k_fg_multiaxpy<<<grid_for(n, kFgBlas, c->num_sms * 16), kFgBlas, 0, c->stream>>>(X, ld, nvec, coef, y, n, sign);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// z = M(v) for rest vectors in the FP32 layout (BF16 weights)
static gs_status net_apply_lp(gs_ctx* c, gs_net* nt, const Plan* p, const float4* v, float4* z) {
    gs_status s = net_prepare(c, nt);
    if (s != GS_OK) return s;
    const int64_t V = c->V, nb = p->nb, nr = V - nb;
    GS_CUDA(c, cudaMemsetAsync(nt->act[0], 0, (size_t)V * 12 * sizeof(float2), c->stream));
    const int g = grid_for(nr * 6, 256, c->num_sms * 8);
    k_net_embed_lp<<<g, 256, 0, c->stream>>>(v, p->perm, nb, nr, nt->act[0]);
    c->launches++;
    if ((s = net_forward(c, nt, true)) != GS_OK) return s;
    k_net_restrict_lp<<<g, 256, 0, c->stream>>>(nt->act[3], p->perm, nb, nr, z);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// after a synchronisation: did a tensor-core layer give up on a wait?
static gs_status net_check(gs_ctx* c, gs_net* nt) {
    if (nt->tc_err && *(volatile int*)nt->tc_err) {
        *(volatile int*)nt->tc_err = 0;
        return set_err(c, GS_TIMEOUT, "tensor-core network layer: a wait timed out");
    }
    return GS_OK;
}

// Flexible GMRES(m) for D_rr e = r with the network as right preconditioner,
// in FP32: it is one cycle of the FP64 defect correction, which only asks it
// to reduce the residual by the cycle tolerance and recomputes the true
// residual in FP64 afterwards.  Vectors in the low-precision stencil's FP32
// layout: v_0 = r / ||r||; z_j = M(v_j), w = D_rr z_j (FP32 stencil), CGS2
// with FP32 products and FP64 sums, Givens rotations on the host;
// e = sum_j z_j y_j (returned in FP64).  Stops at the estimate
// ||r - D_rr e|| <= tol ||r||.
gs_status inner_fgmres_net(gs_ctx* c, const Plan* p, const double2* r, double2* e, double tol,
                           int m, int* iters_out) {
    gs_net* nt = c->net;
    if (!nt) return set_err(c, GS_EINVAL, "no network attached (gs_set_net)");
    const int64_t nb = p->nb, nr = c->V - nb, n = nr * kSiteC;
    const size_t vb = (size_t)n * sizeof(float2);
    if (m < 1) m = 1;
    if (m > kMaxRestart) m = kMaxRestart;
    if (c->fg_cap < nr || c->fg_m < m) {
        cudaFree(c->fg_V);
        cudaFree(c->fg_Z);
        cudaFree(c->fg_w);
        c->fg_V = c->fg_Z = c->fg_w = nullptr;
        if (cudaMalloc(&c->fg_V, vb * (m + 1)) != cudaSuccess || cudaMalloc(&c->fg_Z, vb * m) != cudaSuccess ||
            cudaMalloc(&c->fg_w, vb) != cudaSuccess) {
            cudaGetLastError();
            c->fg_cap = 0;
            return set_err(c, GS_ENOMEM, "allocating FGMRES vectors failed");
        }
        c->fg_cap = nr;
        c->fg_m = m;
    }
    if (!c->fg_h) {
        const size_t hb = (2 * (kMaxRestart + 2) + 1) * sizeof(double2);
        if (cudaMalloc(&c->fg_h, hb) != cudaSuccess || cudaHostAlloc(&c->fg_h_host, hb, 0) != cudaSuccess ||
            cudaMalloc(&c->fg_y, (kMaxRestart + 1) * sizeof(double2)) != cudaSuccess ||
            cudaHostAlloc(&c->fg_y_host, (kMaxRestart + 1) * sizeof(double2), 0) != cudaSuccess ||
            cudaMalloc(&c->fg_red.partial, kRedScratchDoubles * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&c->fg_red.counter, sizeof(unsigned int)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GS_ENOMEM, "allocating FGMRES scratch failed");
        }
        GS_CUDA(c, cudaMemsetAsync(c->fg_red.counter, 0, sizeof(unsigned int), c->stream));
    }
    gs_status s;
    float2* V = c->fg_V;
    float2* Z = c->fg_Z;
    float2* w = c->fg_w;
    double2* hbuf = (double2*)c->fg_h;
    double2* hbuf_host = (double2*)c->fg_h_host;
    // beta = ||r|| (FP64), v_0 = r / beta
    if ((s = launch_norm2(c, c->fg_red, r, n, c->scal_dev)) != GS_OK) return s;
    GS_CUDA(c, cudaMemcpyAsync(c->scal_host, c->scal_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    const double beta = sqrt(c->scal_host[0]);
    *iters_out = 0;
    if (!(beta > 0.0)) {
        GS_CUDA(c, cudaMemsetAsync(e, 0, (size_t)n * sizeof(double2), c->stream));
        return isfinite(beta) ? GS_OK : set_err(c, GS_NONFINITE, "non-finite FGMRES rhs");
    }
    const int g6 = grid_for(nr * 6, 256, c->num_sms * 8);
    k_fg_pack<<<g6, 256, 0, c->stream>>>(r, (float4*)V, nr, 1.0 / beta);
    c->launches++;
    using cplx = std::complex<double>;
    std::vector<cplx> H((size_t)(m + 1) * m), gv(m + 1, 0.0), cs(m), sn(m);
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
        float2* Vj = V + (size_t)j * n;
        float2* Zj = Z + (size_t)j * n;
        if ((s = net_apply_lp(c, nt, p, (const float4*)Vj, (float4*)Zj)) != GS_OK) return s;
        if ((s = lp_rr_apply_f32(c, p, Zj, w)) != GS_OK) return s;
        double2* h = hbuf;
        double2* h2 = hbuf + (m + 2);
        double2* hn2 = hbuf + 2 * (m + 2);
        if ((s = fg_multidot(c, V, n, j + 1, w, n, h)) != GS_OK) return s;
        if ((s = fg_multiaxpy(c, V, n, j + 1, h, w, n, -1.f)) != GS_OK) return s;
        if ((s = fg_multidot(c, V, n, j + 1, w, n, h2)) != GS_OK) return s;
        if ((s = fg_multiaxpy(c, V, n, j + 1, h2, w, n, -1.f)) != GS_OK) return s;
        if ((s = fg_multidot(c, w, n, 1, w, n, hn2)) != GS_OK) return s;
        GS_CUDA(c, cudaMemcpyAsync(hbuf_host, hbuf, (2 * (m + 2) + 1) * sizeof(double2), cudaMemcpyDeviceToHost,
                                   c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        if ((s = net_check(c, nt)) != GS_OK) return s;
        const double hn = sqrt(hbuf_host[2 * (m + 2)].x);
        if (!isfinite(hn)) return set_err(c, GS_NONFINITE, "non-finite FGMRES norm");
        for (int i = 0; i <= j; ++i)
            H[(size_t)i * m + j] = cplx(hbuf_host[i].x + hbuf_host[m + 2 + i].x, hbuf_host[i].y + hbuf_host[m + 2 + i].y);
        H[(size_t)(j + 1) * m + j] = hn;
        if (hn > 0.0) {
            k_fg_scale<<<grid_for(n, kFgBlas, c->num_sms * 16), kFgBlas, 0, c->stream>>>(w, V + (size_t)(j + 1) * n, n,
                                                                                       (float)(1.0 / hn));
            c->launches++;
        }
        for (int i = 0; i < j; ++i) {
            const cplx h0 = H[(size_t)i * m + j], h1 = H[(size_t)(i + 1) * m + j];
            H[(size_t)i * m + j] = std::conj(cs[i]) * h0 + std::conj(sn[i]) * h1;
            H[(size_t)(i + 1) * m + j] = -sn[i] * h0 + cs[i] * h1;
        }
        const cplx aa = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
        const double hh = sqrt(std::norm(aa) + std::norm(bb));
        cs[j] = hh > 0.0 ? aa / hh : cplx(1.0);
        sn[j] = hh > 0.0 ? bb / hh : cplx(0.0);
        H[(size_t)j * m + j] = hh;
        H[(size_t)(j + 1) * m + j] = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = std::conj(cs[j]) * gv[j];
        k = j + 1;
        if (std::abs(gv[j + 1]) <= tol * beta || hn == 0.0) break;
    }
    std::vector<cplx> y(k);
    for (int i = k - 1; i >= 0; --i) {
        cplx acc = gv[i];
        for (int l = i + 1; l < k; ++l) acc -= H[(size_t)i * m + l] * y[l];
        y[i] = acc / H[(size_t)i * m + i];
    }
    double2* yh = (double2*)c->fg_y_host;
    for (int i = 0; i < k; ++i) yh[i] = make_double2(y[i].real(), y[i].imag());
    GS_CUDA(c, cudaMemcpyAsync(c->fg_y, yh, k * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    // e = sum_j z_j y_j, accumulated in w (FP32), returned in FP64
    GS_CUDA(c, cudaMemsetAsync(w, 0, vb, c->stream));
    if ((s = fg_multiaxpy(c, Z, n, k, (const double2*)c->fg_y, w, n, 1.f)) != GS_OK) return s;
    k_fg_unpack<<<g6, 256, 0, c->stream>>>((const float4*)w, e, nr);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    *iters_out = k;
    return GS_OK;
}

void free_net_ctx(gs_ctx* c) {
    cudaFree(c->fg_V);
    cudaFree(c->fg_Z);
    cudaFree(c->fg_w);
    cudaFree(c->fg_h);
    cudaFree(c->fg_y);
    cudaFree(c->fg_red.partial);
    cudaFree(c->fg_red.counter);
    if (c->fg_h_host) cudaFreeHost(c->fg_h_host);
    if (c->fg_y_host) cudaFreeHost(c->fg_y_host);
    c->fg_V = c->fg_Z = c->fg_w = nullptr;
    c->fg_h = c->fg_y = nullptr;
    c->fg_h_host = c->fg_y_host = nullptr;
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_net_create(gs_net** out, int channels) {
    if (!out || !net_channels_ok(channels)) return GS_EINVAL;
    gs_net* nt = new gs_net();
    nt->C = channels;
    bool ok = true;
    for (int l = 0; l < 3; ++l) {
        int cin, cout;
        layer_dims(channels, l, &cin, &cout);
        nt->nel[l] = 9LL * 4 * cin * 4 * cout;
        const size_t b = (size_t)nt->nel[l] * sizeof(float2);
        ok = ok && cudaMalloc(&nt->W[l], b) == cudaSuccess && cudaMalloc(&nt->G[l], b) == cudaSuccess &&
             cudaMalloc(&nt->Wb[l], (size_t)nt->nel[l] * sizeof(__nv_bfloat162)) == cudaSuccess &&
             cudaMalloc(&nt->m[l], b) == cudaSuccess && cudaMalloc(&nt->v[l], b) == cudaSuccess;
        if (ok) {
            cudaMemset(nt->W[l], 0, b);
            cudaMemset(nt->m[l], 0, b);
            cudaMemset(nt->v[l], 0, b);
            cudaMemset(nt->Wb[l], 0, (size_t)nt->nel[l] * sizeof(__nv_bfloat162));
        }
    }
    const int64_t big = 9LL * 4 * channels * 4 * channels;
    ok = ok && cudaMalloc(&nt->Wp, big * sizeof(float2)) == cudaSuccess &&
         cudaMalloc(&nt->partial, (size_t)kChunks * big * sizeof(float2)) == cudaSuccess &&
         cudaMalloc(&nt->red, 4096 * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&nt->counter, sizeof(unsigned int)) == cudaSuccess &&
         cudaHostAlloc(&nt->host_red, 4 * sizeof(float), 0) == cudaSuccess &&
         cudaHostAlloc(&nt->tc_err, sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
         cudaHostGetDevicePointer(&nt->tc_err_dev, nt->tc_err, 0) == cudaSuccess;
    if (ok) *nt->tc_err = 0;
    if (ok && channels == 24)
        ok = cudaMalloc(&nt->Btc, net_tc_weight_elems() * sizeof(__nv_bfloat16)) == cudaSuccess &&
             cudaMalloc(&nt->Bphi, net_phi_weight_elems() * sizeof(__nv_bfloat16)) == cudaSuccess &&
             cudaMalloc(&nt->Bl1, net_l1_weight_elems() * sizeof(__nv_bfloat16)) == cudaSuccess;
    if (ok) ok = cudaMemset(nt->counter, 0, sizeof(unsigned int)) == cudaSuccess &&
                 cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        gs_net_destroy(nt);
        return GS_ENOMEM;
    }
    *out = nt;
    return GS_OK;
}

gs_status gs_net_destroy(gs_net* nt) {
    if (!nt) return GS_OK;
    cudaDeviceSynchronize();
    for (int l = 0; l < 3; ++l) {
        cudaFree(nt->W[l]);
        cudaFree(nt->Wb[l]);
        cudaFree(nt->G[l]);
        cudaFree(nt->m[l]);
        cudaFree(nt->v[l]);
    }
    for (auto& a : nt->act) cudaFree(a);
    for (auto& a : nt->gact) cudaFree(a);
    cudaFree(nt->Wp);
    cudaFree(nt->partial);
    cudaFree(nt->U32);
    cudaFree(nt->red);
    cudaFree(nt->counter);
    if (nt->host_red) cudaFreeHost(nt->host_red);
    if (nt->tc_err) cudaFreeHost(nt->tc_err);
    cudaFree(nt->Btc);
    cudaFree(nt->Bphi);
    cudaFree(nt->Bl1);
    cudaGetLastError();
    delete nt;
    return GS_OK;
}

// w_host: complex64 [9][4 C_out][4 C_in] (W_d[R][k]); stored transposed
gs_status gs_net_set_weights(gs_net* nt, int layer, const void* w_host) {
    if (!nt || layer < 0 || layer > 2 || !w_host) return GS_EINVAL;
    int cin, cout;
    layer_dims(nt->C, layer, &cin, &cout);
    const int K = 4 * cin, R4 = 4 * cout;
    const float2* src = (const float2*)w_host;
    std::vector<float2> t((size_t)nt->nel[layer]);
    for (int d = 0; d < 9; ++d)
        for (int R = 0; R < R4; ++R)
            for (int k = 0; k < K; ++k)
                t[((size_t)d * K + k) * R4 + R] = src[((size_t)d * R4 + R) * K + k];
    if (cudaMemcpy(nt->W[layer], t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return GS_ECUDA;
    k_net_tobf16<<<grid_for(2 * nt->nel[layer], 256, 1024), 256>>>((const float*)nt->W[layer],
                                                                   (__nv_bfloat16*)nt->Wb[layer],
                                                                   2 * nt->nel[layer]);
    const size_t b = (size_t)nt->nel[layer] * sizeof(float2);
    cudaMemset(nt->m[layer], 0, b);
    cudaMemset(nt->v[layer], 0, b);
    nt->step = 0;
    nt->tc_dirty = true;
    return cudaDeviceSynchronize() == cudaSuccess ? GS_OK : GS_ECUDA;
}

// what: 0 = FP32 weights, 1 = gradients of the last training step; layout as set
gs_status gs_net_get(gs_net* nt, int what, int layer, void* host_out) {
    if (!nt || layer < 0 || layer > 2 || !host_out || (what != 0 && what != 1)) return GS_EINVAL;
    int cin, cout;
    layer_dims(nt->C, layer, &cin, &cout);
    const int K = 4 * cin, R4 = 4 * cout;
    std::vector<float2> t((size_t)nt->nel[layer]);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(t.data(), what == 0 ? nt->W[layer] : nt->G[layer], t.size() * sizeof(float2),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return GS_ECUDA;
    float2* dst = (float2*)host_out;
    for (int d = 0; d < 9; ++d)
        for (int R = 0; R < R4; ++R)
            for (int k = 0; k < K; ++k)
                dst[((size_t)d * R4 + R) * K + k] = t[((size_t)d * K + k) * R4 + R];
    return GS_OK;
}

gs_status gs_net_apply(gs_ctx* c, gs_net* nt, int type, int dir, int inverse, const void* t_dev,
                       void* y_dev) {
    if (!c || !nt) return GS_EINVAL;
    if (!t_dev || !y_dev) return set_err(c, GS_EINVAL, "null vector");
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    if ((s = net_apply_rest(c, nt, p, (const double2*)t_dev, (double2*)y_dev)) != GS_OK) return s;
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return net_check(c, nt);
}

// One training step on `batch` pairs of the rest set of (type, dir, inverse):
// t_dev, z_dev complex64 [batch][n_r][12] (z = D_rr^-1 t).  Loss = mean over
// the batch of ||M(t)|_r - z||^2 / ||z||^2 (returned in *loss_out); the
// gradients are left in the network; if update != 0 an Adam step with
// learning rate lr follows (beta1 0.9, beta2 0.999, eps 1e-8).
gs_status gs_net_train_step(gs_ctx* c, gs_net* nt, int type, int dir, int inverse, int batch,
                            const void* t_dev, const void* z_dev, float lr, int update, float* loss_out) {
    if (!c || !nt) return GS_EINVAL;
    if (batch < 1 || !t_dev || !z_dev) return set_err(c, GS_EINVAL, "bad batch");
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    if ((s = net_prepare(c, nt)) != GS_OK) return s;
    const Plan* id = c->plans[0];
    const int64_t V = c->V, nb = p->nb, nr = V - nb;
    const int g = grid_for(nr * 12, 256, 1024);
    const int blocks = (int)((V + kTS - 1) / kTS);
    const float2* T = (const float2*)t_dev;
    const float2* Z = (const float2*)z_dev;
    double loss = 0.0;
    for (int b = 0; b < batch; ++b) {
        const float2* tb = T + (size_t)b * nr * 12;
        const float2* zb = Z + (size_t)b * nr * 12;
        GS_CUDA(c, cudaMemsetAsync(nt->act[0], 0, (size_t)V * 12 * sizeof(float2), c->stream));
        k_net_embed32<<<g, 256, 0, c->stream>>>(tb, p->perm, nb, nr, nt->act[0]);
        c->launches++;
        if ((s = net_forward(c, nt, false)) != GS_OK) return s;
        k_net_loss<<<g, 256, 0, c->stream>>>(nt->act[3], zb, p->perm, nb, nr, nt->red, nt->counter);
        // gradient of the last activation into gact[0] (only 12 per site used)
        GS_CUDA(c, cudaMemsetAsync(nt->gact[0], 0, (size_t)V * 12 * sizeof(float2), c->stream));
        k_net_lossgrad<<<g, 256, 0, c->stream>>>(nt->act[3], zb, p->perm, nb, nr, nt->red,
                                                 1.0f / batch, nt->gact[0]);
        c->launches += 2;
        GS_CUDA(c, cudaMemcpyAsync(nt->host_red, nt->red, 2 * sizeof(float), cudaMemcpyDeviceToHost,
                                   c->stream));
        // backward through the three layers
        float2* gout = nt->gact[0];
        float2* gin = nt->gact[1];
        for (int l = 2; l >= 0; --l) {
            int cin, cout;
            layer_dims(nt->C, l, &cin, &cout);
            gradw_dispatch(nt->C, cin, cout, nt->act[l], gout, nt->partial, nt->U32, id->nbr, V, c->stream);
            k_net_reduce<<<grid_for(nt->nel[l], 256, 1024), 256, 0, c->stream>>>(nt->partial, nt->G[l],
                                                                                 nt->nel[l], kChunks, b > 0);
            c->launches += 2;
            if (l > 0) {
                k_net_wprime<<<grid_for(nt->nel[l], 256, 1024), 256, 0, c->stream>>>(nt->W[l], nt->Wp,
                                                                                    4 * cin, 4 * cout);
                conv_dispatch<float2>(nt->C, cout, cin, gout, gin, nt->Wp, nt->U32, id->nbr, V, blocks,
                                      c->stream);
                c->launches += 2;
                float2* tmp = gout;
                gout = gin;
                gin = tmp;
            }
            GS_CHECK_LAUNCH(c);
        }
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        loss += (double)nt->host_red[0] / (double)nt->host_red[1];
    }
    if (loss_out) *loss_out = (float)(loss / batch);
    if (update) {
        nt->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)nt->step), c2 = 1.f - powf(b2, (float)nt->step);
        for (int l = 0; l < 3; ++l) {
            k_net_adam<<<grid_for(2 * nt->nel[l], 256, 1024), 256, 0, c->stream>>>(
                (float*)nt->W[l], (const float*)nt->G[l], nt->m[l], nt->v[l], (__nv_bfloat16*)nt->Wb[l],
                2 * nt->nel[l], lr, b1, b2, 1e-8f, c1, c2);
            c->launches++;
        }
        nt->tc_dirty = true;
        GS_CHECK_LAUNCH(c);
    }
    return GS_OK;
}

gs_status gs_set_net(gs_ctx* c, gs_net* nt) {
    if (!c) return GS_EINVAL;
    c->net = nt;
    return GS_OK;
}

}  // extern "C"
