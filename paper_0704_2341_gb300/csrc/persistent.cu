// Persistent BiCGStab on D_rr: the whole inner solve in one cooperative launch.
//
// On the lattices of the benchmark (8^4: 3840 rest sites) a BiCGStab
// iteration is latency bound: five kernel launches, each ending in a
// reduction tail, cost more than the arithmetic.  Here every block of one
// co-resident grid runs all iterations; the four phases of an iteration are
// separated by a grid barrier, and each reduction is finished by every block
// summing the per-block partials in the same fixed order, so all blocks hold
// bit-identical scalars without another barrier.
//
// Grid barrier: one release add per block on an arrival counter that grows
// through the launch, acquire polls until the barrier's last arrival (see
// gridsync.cuh).  Every wait is bounded: after kSpinLimit polls or the
// context's wait limit of global time the waiting block records GS_TIMEOUT in
// the error word, the other blocks leave when they see it, and the host reads
// the status.  The
// grid is sized with the occupancy calculator and launched with
// cudaLaunchCooperativeKernel, which refuses grids that cannot be
// co-resident.
//
// Vectors written inside the kernel are read with L2-only loads (__ldcg):
// the read-only cache path is not coherent with writes of other blocks of
// the same kernel.
#include "dslash_f64.cuh"
#include "gridsync.cuh"
#include "lowp.cuh"

namespace gs {
namespace {

constexpr int kPThreads = 128;
constexpr int kPart = 8;   // values per block in one slot of the partial sums

// Sum NV values over the block (fixed tree); thread 0 gets the result.
template <int NV, class T>
__device__ void block_sum(T (&v)[NV], T (&out)[NV]) {
    __shared__ T sm[kPThreads / 32][kPart];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        T x = v[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) sm[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) out[q] = (sm[0][q] + sm[1][q]) + (sm[2][q] + sm[3][q]);
    }
    __syncthreads();
}

// Every block adds the partials of all blocks in the same order (warp w
// takes blocks w*32 + lane, w*32 + lane + 128, ...; then a fixed tree), so
// all blocks hold bit-identical totals; the totals land in every thread.
template <int NV, class T>
__device__ void grid_total(const T* partial, T (&tot)[NV]) {
    __shared__ T sh[kPThreads / 32][kPart];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = T(0);
    // L2 loads (written by other blocks before the grid barrier); not
    // volatile, so the loads of all iterations can be in flight at once
#pragma unroll 2
    for (int b = warp * 32 + lane; b < (int)gridDim.x; b += kPThreads) {
        const T* p = partial + (int64_t)b * kPart;
#pragma unroll
        for (int q = 0; q < NV; ++q) s[q] += __ldcg(p + q);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[warp][q] = s[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = (sh[0][q] + sh[1][q]) + (sh[2][q] + sh[3][q]);
    __syncthreads();
}

template <int NV, class T>
__device__ __forceinline__ void put_partial(T* partial, const T (&v)[NV]) {
    T b[NV];
    T vv[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) vv[q] = v[q];
    block_sum<NV, T>(vv, b);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partial[(int64_t)blockIdx.x * kPart + q] = b[q];
    }
}

// complex helpers on double2 scalars
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double inv = 1.0 / (b.x * b.x + b.y * b.y);
    return make_double2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}

struct PArgs64 {
    StencilArgs A;  // v = D_rr p with <rhat, v>
    StencilArgs C;  // t = D_rr s with <t, s>, <t, t>, <rhat, t>
    const double2* b;
    double2 *x, *r, *rhat, *p, *v, *s, *t;
    int64_t n;        // complex entries (12 per site)
    int ts;           // sites per stencil tile (<= 32)
    double tol;
    int maxit;
    double* partial;  // [6 slots][gridDim][kPart]
    GridSync sync;
    BicgState* st;
    unsigned long long* phases;  // [16] or null: cycles per phase (block 0)
};

// phase clock of block 0 (profiling only)
struct PhaseClock {
    unsigned long long acc[15];
    long long t;
    bool on;
    __device__ void start(bool enable) {
        on = enable && blockIdx.x == 0 && threadIdx.x == 0;
#pragma unroll
        for (int i = 0; i < 15; ++i) acc[i] = 0;
        t = on ? clock64() : 0;
    }
    __device__ __forceinline__ void mark(int i) {
        if (on) {
            const long long now = clock64();
            acc[i] += (unsigned long long)(now - t);
            t = now;
        }
    }
    __device__ void flush(unsigned long long* out) {
        if (on)
#pragma unroll
            for (int i = 0; i < 15; ++i) atomicAdd(out + i, acc[i]);
    }
};

// van der Vorst's BiCGStab with four grid barriers per iteration:
//   A: v = D p, <rhat, v>                      | alpha = rho / <rhat, v>
//   B: s = r - alpha v, ||s||^2, <rhat, s>     | stop early if ||s|| small
//   C: t = D s, <t, s>, <t, t>, <rhat, t>      | omega = <t, s> / <t, t>,
//                                              | rho' = <rhat, s> - omega <rhat, t>
//   D: x += alpha p + omega s, r = s - omega t,
//      p = r + beta (p - omega v), ||r||^2     | converged?
// rho' = <rhat, r'> = <rhat, s - omega t> by linearity, so the x, r and p
// updates share one phase and the reduction that decides beta comes with t's
// stencil.  (<rhat, s> vanishes in exact arithmetic, but not in rounding:
// dropping it stalls the iteration once rhat and r are nearly orthogonal.)
__global__ void __launch_bounds__(kPThreads) k_bicg_persistent_f64(PArgs64 P) {
    __shared__ double red[4][24][kSitesPerBlock];
    __shared__ double2 sc[5];   // alpha, omega, beta, rho, <rhat, s>
    __shared__ int s_flag;       // 0, or 10 + a failure status
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t slot = (int64_t)gridDim.x * kPart;
    const int ts = P.ts;
    double* part = P.partial;
    bool ok = true;
    int iter = 0;
    double rr = 0.0, bb = 0.0, tol2 = 0.0;
    int status = GS_OK;
    bool conv = false, early = false;

    // x = 0, r = rhat = p = b, ||b||^2
    {
        double v[1] = {0.0};
        for (int64_t i = tid; i < P.n; i += nth) {
            const double2 bi = __ldcg(P.b + i);
            P.x[i] = make_double2(0.0, 0.0);
            P.r[i] = bi;
            P.rhat[i] = bi;
            P.p[i] = bi;
            v[0] = fma(bi.x, bi.x, fma(bi.y, bi.y, v[0]));
        }
        put_partial<1, double>(part, v);
        ok = grid_sync(P.sync);
        double tot[1];
        grid_total<1, double>(part, tot);
        bb = rr = tot[0];
        tol2 = P.tol * P.tol * bb;
        if (threadIdx.x == 0) sc[3] = make_double2(bb, 0.0);
        if (!(bb > 0.0)) {
            conv = (bb == 0.0);
            if (!conv) status = GS_NONFINITE;
        }
        __syncthreads();
    }
    PhaseClock pc;
    pc.start(P.phases != nullptr);
    while (ok && !conv && status == GS_OK && iter < P.maxit) {
        // A: v = D p, <rhat, v> -> alpha
        {
            double e[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            for (int64_t base = (int64_t)blockIdx.x * ts; base < P.A.n_out; base += (int64_t)gridDim.x * ts)
                f64_tile<EPI_DOT_RHAT_V, true>(P.A, base, ts, red, e);
            double v[2] = {e[0], e[1]};
            put_partial<2, double>(part + slot, v);
            pc.mark(0);
            if (!(ok = grid_sync(P.sync))) break;
            pc.mark(1);
            double tot[2];
            grid_total<2, double>(part + slot, tot);
            if (threadIdx.x == 0) {
                s_flag = 0;
                if (tot[0] == 0.0 && tot[1] == 0.0) s_flag = 10 + GS_BREAKDOWN;
                else {
                    sc[0] = zdiv(sc[3], make_double2(tot[0], tot[1]));
                    if (!isfinite(sc[0].x) || !isfinite(sc[0].y)) s_flag = 10 + GS_NONFINITE;
                }
            }
            __syncthreads();
            pc.mark(2);
            if (s_flag >= 10) {
                status = s_flag - 10;
                break;
            }
        }
        // B: s = r - alpha v ; ||s||^2, <rhat, s>
        {
            const double2 al = sc[0];
            double v[3] = {0.0, 0.0, 0.0};
            for (int64_t i = tid; i < P.n; i += nth) {
                const double2 vi = __ldcg(P.v + i), ri = __ldcg(P.r + i), hi = __ldcg(P.rhat + i);
                double2 si;
                si.x = ri.x - (al.x * vi.x - al.y * vi.y);
                si.y = ri.y - (al.x * vi.y + al.y * vi.x);
                P.s[i] = si;
                v[0] = fma(si.x, si.x, fma(si.y, si.y, v[0]));
                v[1] = fma(hi.x, si.x, fma(hi.y, si.y, v[1]));
                v[2] = fma(hi.x, si.y, fma(-hi.y, si.x, v[2]));
            }
            put_partial<3, double>(part + 2 * slot, v);
            pc.mark(3);
            if (!(ok = grid_sync(P.sync))) break;
            pc.mark(4);
            double tot[3];
            grid_total<3, double>(part + 2 * slot, tot);
            if (threadIdx.x == 0) sc[4] = make_double2(tot[1], tot[2]);
            pc.mark(5);
            if (!isfinite(tot[0])) {
                status = GS_NONFINITE;
                break;
            }
            if (tot[0] <= tol2) {   // x += alpha p below, after the loop
                rr = tot[0];
                ++iter;
                conv = early = true;
                break;
            }
        }
        // C: t = D s, <t, s>, <t, t>, <rhat, t> -> omega, rho', beta
        {
            double e[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            for (int64_t base = (int64_t)blockIdx.x * ts; base < P.C.n_out; base += (int64_t)gridDim.x * ts)
                f64_tile<EPI_DOT_TSR, true>(P.C, base, ts, red, e);
            put_partial<5, double>(part + 3 * slot, e);
            pc.mark(6);
            if (!(ok = grid_sync(P.sync))) break;
            pc.mark(7);
            double tot[5];
            grid_total<5, double>(part + 3 * slot, tot);
            if (threadIdx.x == 0) {
                const double inv = tot[2] > 0.0 ? 1.0 / tot[2] : 0.0;
                const double2 om = make_double2(tot[0] * inv, tot[1] * inv);
                const double2 rs = sc[4];
                const double2 rho_new = make_double2(rs.x - (om.x * tot[3] - om.y * tot[4]),
                                                     rs.y - (om.x * tot[4] + om.y * tot[3]));
                sc[1] = om;
                s_flag = (isfinite(om.x) && isfinite(om.y)) ? 0 : 10 + GS_NONFINITE;
                // beta = (rho' / rho) (alpha / omega); a zero omega or rho' is a
                // breakdown unless phase D's residual shows convergence
                if (s_flag == 0 && !(om.x == 0.0 && om.y == 0.0) && !(rho_new.x == 0.0 && rho_new.y == 0.0)) {
                    sc[2] = zmul(zdiv(rho_new, sc[3]), zdiv(sc[0], om));
                    sc[3] = rho_new;
                } else if (s_flag == 0) {
                    s_flag = 1;     // breakdown pending
                    sc[2] = make_double2(0.0, 0.0);
                }
            }
            __syncthreads();
            pc.mark(8);
            if (s_flag >= 10) {
                status = s_flag - 10;
                break;
            }
        }
        // D: x += alpha p + omega s ; r = s - omega t ; p = r + beta (p - omega v) ; ||r||^2
        {
            const double2 al = sc[0], om = sc[1], be = sc[2];
            const bool pending = s_flag == 1;
            double v[1] = {0.0};
            for (int64_t i = tid; i < P.n; i += nth) {
                const double2 si = __ldcg(P.s + i), ti = __ldcg(P.t + i), vi = __ldcg(P.v + i);
                double2 pi = __ldcg(P.p + i), xi = __ldcg(P.x + i);
                xi.x = fma(al.x, pi.x, fma(-al.y, pi.y, xi.x));
                xi.y = fma(al.x, pi.y, fma(al.y, pi.x, xi.y));
                xi.x = fma(om.x, si.x, fma(-om.y, si.y, xi.x));
                xi.y = fma(om.x, si.y, fma(om.y, si.x, xi.y));
                P.x[i] = xi;
                double2 ri;
                ri.x = si.x - (om.x * ti.x - om.y * ti.y);
                ri.y = si.y - (om.x * ti.y + om.y * ti.x);
                P.r[i] = ri;
                double2 q;
                q.x = pi.x - (om.x * vi.x - om.y * vi.y);
                q.y = pi.y - (om.x * vi.y + om.y * vi.x);
                pi.x = fma(be.x, q.x, fma(-be.y, q.y, ri.x));
                pi.y = fma(be.x, q.y, fma(be.y, q.x, ri.y));
                P.p[i] = pi;
                v[0] = fma(ri.x, ri.x, fma(ri.y, ri.y, v[0]));
            }
            put_partial<1, double>(part + 4 * slot, v);
            pc.mark(9);
            ++iter;
            if (!(ok = grid_sync(P.sync))) break;
            pc.mark(10);
            double tot[1];
            grid_total<1, double>(part + 4 * slot, tot);
            pc.mark(11);
            rr = tot[0];
            if (!isfinite(rr)) {
                status = GS_NONFINITE;
                break;
            }
            if (rr <= tol2) {
                conv = true;
                break;
            }
            if (pending) {
                status = GS_BREAKDOWN;
                break;
            }
        }
    }
    if (early) {
        // converged on s: x += alpha p (each thread its own entries; no
        // other block reads x again)
        const double2 al = sc[0];
        for (int64_t i = tid; i < P.n; i += nth) {
            const double2 pi = __ldcg(P.p + i);
            double2 xi = __ldcg(P.x + i);
            xi.x = fma(al.x, pi.x, fma(-al.y, pi.y, xi.x));
            xi.y = fma(al.x, pi.y, fma(al.y, pi.x, xi.y));
            P.x[i] = xi;
        }
    }
    pc.flush(P.phases);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        BicgState* st = P.st;
        st->iter = iter;
        st->rr = rr;
        st->bb = bb;
        st->status = ok ? status : (int)GS_TIMEOUT;
        st->done = (conv || !ok || status != GS_OK) ? 1 : 0;
        publish(st);
    }
}

// ---------------------------------------------------------------------------
// low-precision persistent BiCGStab (FP32 arithmetic; FP32 or BF16 storage)
// ---------------------------------------------------------------------------
struct PArgsLp {
    LpArgs A;  // in = p, out = v, epi_vec = rhat
    LpArgs C;  // in = s, out = t, epi_vec = s
    const double2* r64;   // FP64 right-hand side of the cycle (rest set, AoS)
    const double* rr64;   // its ||.||^2 (device)
    void *x, *r, *rhat, *p, *v, *s, *t;
    int64_t n;            // sites
    float tol;
    int maxit;
    float* partial;       // [6 slots][gridDim][kPart]
    GridSync sync;
    LpState* st;
};

template <class S, int EPI>
__device__ __forceinline__ void lp_site_stencil(const LpArgs& a, int64_t k, float (&e)[3]) {
    const int4 n01 = __ldg((const int4*)(a.nbr + k * 4));
    const int4 n23 = __ldg((const int4*)(a.nbr + k * 4) + 1);
    float acc[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) acc[q] = 0.f;
    site_dir<S, 0, true>(a, k, make_int2(n01.x, n01.y), acc);
    site_dir<S, 1, true>(a, k, make_int2(n01.z, n01.w), acc);
    site_dir<S, 2, true>(a, k, make_int2(n23.x, n23.y), acc);
    site_dir<S, 3, true>(a, k, make_int2(n23.z, n23.w), acc);
    float self[24];
    Store<S>::template load_spinor<true>(a.in, a.n, k, self);
#pragma unroll
    for (int q = 0; q < 24; ++q) acc[q] = fmaf(a.diag, self[q], acc[q]);
    Store<S>::store_spinor(a.out, a.n, k, acc);
    float w[24];
    Store<S>::template load_spinor<true>(a.epi_vec, a.n, k, w);
    if (EPI == EPI_DOT_RHAT_V) {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            e[0] = fmaf(w[2 * q], acc[2 * q], fmaf(w[2 * q + 1], acc[2 * q + 1], e[0]));
            e[1] = fmaf(w[2 * q], acc[2 * q + 1], fmaf(-w[2 * q + 1], acc[2 * q], e[1]));
        }
    } else {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float tr = acc[2 * q], ti = acc[2 * q + 1];
            e[0] = fmaf(tr, w[2 * q], fmaf(ti, w[2 * q + 1], e[0]));
            e[1] = fmaf(tr, w[2 * q + 1], fmaf(-ti, w[2 * q], e[1]));
            e[2] = fmaf(tr, tr, fmaf(ti, ti, e[2]));
        }
    }
}

__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 fdiv2(float2 a, float2 b) {
    const float inv = 1.0f / (b.x * b.x + b.y * b.y);
    return make_float2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}

// Register budget for four blocks per SM (128 registers; 24^3 x 48, FP32:
// 0.69 of measured HBM against 0.65 at the compiler's 164 and three per SM).
// In a batched call with low-precision inner solves these are the only
// cooperative blocks (the FP64 fallback runs one launch per phase there), so
// the call's block ledger still counts blocks of one size.
template <class S>
__global__ void __launch_bounds__(kPThreads, 4) k_bicg_persistent_lp(PArgsLp P) {
    __shared__ float2 sc[4];  // alpha, omega, beta, rho
    __shared__ int s_flag;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t slot = (int64_t)gridDim.x * kPart;
    float* part = P.partial;
    bool ok = true, conv = false;
    int iter = 0, status = GS_OK;
    float rr = 0.f, bb = 0.f, tol2 = 0.f;
    // r = rhat = p = r64 / ||r64||, x = 0
    {
        const double nrm2 = *P.rr64;
        const float scale = nrm2 > 0.0 ? (float)(1.0 / sqrt(nrm2)) : 0.f;
        float v[1] = {0.f};
        for (int64_t k = tid; k < P.n; k += nth) {
            float f[24], z[24];
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                const double2 w = __ldcg(P.r64 + k * 12 + q);
                f[2 * q] = (float)w.x * scale;
                f[2 * q + 1] = (float)w.y * scale;
                z[2 * q] = z[2 * q + 1] = 0.f;
            }
            Store<S>::store_spinor(P.r, P.n, k, f);
            Store<S>::store_spinor(P.rhat, P.n, k, f);
            Store<S>::store_spinor(P.p, P.n, k, f);
            Store<S>::store_spinor(P.x, P.n, k, z);
            Store<S>::template load_spinor<true>(P.r, P.n, k, f);
#pragma unroll
            for (int q = 0; q < 24; ++q) v[0] = fmaf(f[q], f[q], v[0]);
        }
        put_partial<1, float>(part, v);
        ok = grid_sync(P.sync);
        float tot[1];
        grid_total<1, float>(part, tot);
        bb = rr = tot[0];
        tol2 = P.tol * P.tol * bb;
        if (threadIdx.x == 0) sc[3] = make_float2(bb, 0.f);
        if (!(bb > 0.f)) {
            conv = (bb == 0.f);
            if (!conv) status = GS_NONFINITE;
        }
        __syncthreads();
    }
    while (ok && !conv && status == GS_OK && iter < P.maxit) {
        {  // A: v = D p, <rhat, v> -> alpha
            float e[3] = {0.f, 0.f, 0.f};
            for (int64_t k = tid; k < P.n; k += nth) lp_site_stencil<S, EPI_DOT_RHAT_V>(P.A, k, e);
            float v[2] = {e[0], e[1]};
            put_partial<2, float>(part + slot, v);
            if (!(ok = grid_sync(P.sync))) break;
            float tot[2];
            grid_total<2, float>(part + slot, tot);
            if (threadIdx.x == 0) {
                s_flag = 0;
                if (tot[0] == 0.f && tot[1] == 0.f) s_flag = 10 + GS_BREAKDOWN;
                else {
                    sc[0] = fdiv2(sc[3], make_float2(tot[0], tot[1]));
                    if (!isfinite(sc[0].x) || !isfinite(sc[0].y)) s_flag = 10 + GS_NONFINITE;
                }
            }
            __syncthreads();
            if (s_flag >= 10) {
                status = s_flag - 10;
                break;
            }
        }
        {  // B: s = r - alpha v ; x += alpha p ; ||s||^2
            const float2 al = sc[0];
            float v[1] = {0.f};
            for (int64_t k = tid; k < P.n; k += nth) {
                float fr[24], fv[24], fp[24], fx[24];
                Store<S>::template load_spinor<true>(P.r, P.n, k, fr);
                Store<S>::template load_spinor<true>(P.v, P.n, k, fv);
                Store<S>::template load_spinor<true>(P.p, P.n, k, fp);
                Store<S>::template load_spinor<true>(P.x, P.n, k, fx);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const float vr = fv[2 * q], vi = fv[2 * q + 1];
                    fr[2 * q] -= al.x * vr - al.y * vi;
                    fr[2 * q + 1] -= al.x * vi + al.y * vr;
                    const float pr = fp[2 * q], pi = fp[2 * q + 1];
                    fx[2 * q] = fmaf(al.x, pr, fmaf(-al.y, pi, fx[2 * q]));
                    fx[2 * q + 1] = fmaf(al.x, pi, fmaf(al.y, pr, fx[2 * q + 1]));
                }
                Store<S>::store_spinor(P.s, P.n, k, fr);
                Store<S>::store_spinor(P.x, P.n, k, fx);
#pragma unroll
                for (int q = 0; q < 24; ++q) v[0] = fmaf(fr[q], fr[q], v[0]);
            }
            put_partial<1, float>(part + 2 * slot, v);
            if (!(ok = grid_sync(P.sync))) break;
            float tot[1];
            grid_total<1, float>(part + 2 * slot, tot);
            if (!isfinite(tot[0])) {
                status = GS_NONFINITE;
                break;
            }
            if (tot[0] <= tol2) {
                rr = tot[0];
                ++iter;
                conv = true;
                break;
            }
        }
        {  // C: t = D s, <t, s>, <t, t> -> omega
            float e[3] = {0.f, 0.f, 0.f};
            for (int64_t k = tid; k < P.n; k += nth) lp_site_stencil<S, EPI_DOT_TS>(P.C, k, e);
            put_partial<3, float>(part + 3 * slot, e);
            if (!(ok = grid_sync(P.sync))) break;
            float tot[3];
            grid_total<3, float>(part + 3 * slot, tot);
            if (threadIdx.x == 0) {
                const float inv = tot[2] > 0.f ? 1.f / tot[2] : 0.f;
                sc[1] = make_float2(tot[0] * inv, tot[1] * inv);
                s_flag = (isfinite(sc[1].x) && isfinite(sc[1].y)) ? 0 : 10 + GS_NONFINITE;
            }
            __syncthreads();
            if (s_flag >= 10) {
                status = s_flag - 10;
                break;
            }
        }
        {  // D: x += omega s ; r = s - omega t ; <rhat, r>, ||r||^2 -> beta
            const float2 om = sc[1];
            float v[3] = {0.f, 0.f, 0.f};
            for (int64_t k = tid; k < P.n; k += nth) {
                float fs[24], ft[24], fh[24], fx[24];
                Store<S>::template load_spinor<true>(P.s, P.n, k, fs);
                Store<S>::template load_spinor<true>(P.t, P.n, k, ft);
                Store<S>::template load_spinor<true>(P.rhat, P.n, k, fh);
                Store<S>::template load_spinor<true>(P.x, P.n, k, fx);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const float sr = fs[2 * q], si = fs[2 * q + 1];
                    fx[2 * q] = fmaf(om.x, sr, fmaf(-om.y, si, fx[2 * q]));
                    fx[2 * q + 1] = fmaf(om.x, si, fmaf(om.y, sr, fx[2 * q + 1]));
                    const float tr = ft[2 * q], ti = ft[2 * q + 1];
                    const float r_ = sr - (om.x * tr - om.y * ti);
                    const float i_ = si - (om.x * ti + om.y * tr);
                    fs[2 * q] = r_;
                    fs[2 * q + 1] = i_;
                    v[0] = fmaf(fh[2 * q], r_, fmaf(fh[2 * q + 1], i_, v[0]));
                    v[1] = fmaf(fh[2 * q], i_, fmaf(-fh[2 * q + 1], r_, v[1]));
                    v[2] = fmaf(r_, r_, fmaf(i_, i_, v[2]));
                }
                Store<S>::store_spinor(P.x, P.n, k, fx);
                Store<S>::store_spinor(P.r, P.n, k, fs);
            }
            put_partial<3, float>(part + 4 * slot, v);
            if (!(ok = grid_sync(P.sync))) break;
            float tot[3];
            grid_total<3, float>(part + 4 * slot, tot);
            ++iter;
            rr = tot[2];
            if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
                status = GS_NONFINITE;
                break;
            }
            if (rr <= tol2) {
                conv = true;
                break;
            }
            if ((om.x == 0.f && om.y == 0.f) || (tot[0] == 0.f && tot[1] == 0.f)) {
                status = GS_BREAKDOWN;
                break;
            }
            if (threadIdx.x == 0) {
                const float2 rho_new = make_float2(tot[0], tot[1]);
                sc[2] = fmul2(fdiv2(rho_new, sc[3]), fdiv2(sc[0], om));
                sc[3] = rho_new;
            }
            __syncthreads();
        }
        {  // E: p = r + beta (p - omega v)
            const float2 be = sc[2], om = sc[1];
            for (int64_t k = tid; k < P.n; k += nth) {
                float fr[24], fv[24], fp[24];
                Store<S>::template load_spinor<true>(P.r, P.n, k, fr);
                Store<S>::template load_spinor<true>(P.v, P.n, k, fv);
                Store<S>::template load_spinor<true>(P.p, P.n, k, fp);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const float vr = fv[2 * q], vi = fv[2 * q + 1];
                    const float qr = fp[2 * q] - (om.x * vr - om.y * vi);
                    const float qi = fp[2 * q + 1] - (om.x * vi + om.y * vr);
                    fp[2 * q] = fmaf(be.x, qr, fmaf(-be.y, qi, fr[2 * q]));
                    fp[2 * q + 1] = fmaf(be.x, qi, fmaf(be.y, qr, fr[2 * q + 1]));
                }
                Store<S>::store_spinor(P.p, P.n, k, fp);
            }
            if (!(ok = grid_sync(P.sync))) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        LpState* st = P.st;
        st->iter = iter;
        st->rr = rr;
        st->bb = bb;
        st->status = ok ? status : (int)GS_TIMEOUT;
        st->done = 1;
        lp_publish(st);
    }
}

// Failure-detection self-test: block 0 never arrives at the grid barrier (it
// waits, bounded by the same limit, on a flag that nothing sets); every other
// block's grid_sync runs out of time and records GS_TIMEOUT in the error word.
__global__ void __launch_bounds__(kPThreads) k_selftest_grid_timeout(GridSync g, const int* never) {
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            const unsigned long long t0 = global_ns();
            while (vload(never) == 0 && global_ns() - t0 < g.wait_ns) {
            }
        }
        return;
    }
    grid_sync(g);
}

// co-resident grid for a cooperative launch on a set of rest_sites sites: at
// most `want` blocks.  Inside schur_solve_batched (no GS_OPT_COOP_BLOCKS) the
// grid comes from the call's block ledger: on a small rest set a kernel that
// passes `round` (the blocks for one pass over the set) asks for exactly
// that -- on 8^4 the four permutations' FP64 solves take 120 + 64 + 120 + 64
// of the 456 co-resident blocks, one tile round per stencil phase each
// (45.0 solves/s against 40.2 with 76 blocks each); otherwise it asks for its
// share of the GPU while n solves run (two blocks per SM on small sets, all
// co-resident blocks on large ones).
template <class K>
static int coop_grid(gs_ctx* c, K kernel, int64_t want, int64_t rest_sites, int64_t round = 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    const int64_t full = (int64_t)per_sm * c->num_sms;
    if (c->ledger && c->coop_block_cap == 0) {
        int64_t w = want < full ? want : full;
        if (w > kMaxRedBlocks) w = kMaxRedBlocks;
        if (w < 1) w = 1;
        const int n = c->ledger->running.load() > 1 ? c->ledger->running.load() : 1;
        const bool small = rest_sites <= kBatchMaxRestSites;
        const int64_t target = (small && round > 0) ? round
                               : (small && per_sm > 2 ? 2 : per_sm) * (int64_t)c->num_sms / n;
        return (int)ledger_grant(c, per_sm, w, target > 0 ? target : 1);
    }
    int64_t g = coop_blocks(c, per_sm, rest_sites);
    if (want < g) g = want;
    if (g < 1) g = 1;
    if (g > kMaxRedBlocks) g = kMaxRedBlocks;
    return (int)g;
}

}  // namespace

// scratch of the persistent kernels (partials and the barrier words)
struct PersistScratch {
    void* partial = nullptr;
    unsigned int* words = nullptr;  // count, gen, err
};

static gs_status persist_scratch(gs_ctx* c, PersistScratch** out) {
    if (!c->persist) {
        PersistScratch* p = new PersistScratch();
        if (cudaMalloc(&p->partial, 6 * (size_t)kMaxRedBlocks * kPart * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&p->words, 4 * sizeof(unsigned int)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(p->partial);
            delete p;
            return set_err(c, GS_ENOMEM, "allocating the persistent-solver scratch failed");
        }
        c->persist = p;
    }
    *out = (PersistScratch*)c->persist;
    return GS_OK;
}

void free_persist(gs_ctx* c) {
    PersistScratch* p = (PersistScratch*)c->persist;
    if (!p) return;
    cudaFree(p->partial);
    cudaFree(p->words);
    delete p;
    c->persist = nullptr;
}

gs_status persistent_bicg_f64(gs_ctx* c, const StencilArgs& A, const StencilArgs& C,
                              const double2* b, double2* x, InnerWork& w, int64_t n, double tol,
                              int maxit) {
    PersistScratch* ps = nullptr;
    gs_status s = persist_scratch(c, &ps);
    if (s != GS_OK) return s;
    const int64_t tiles = (A.n_out + kSitesPerBlock - 1) / kSitesPerBlock;
    const int64_t want = tiles > (int64_t)c->num_sms ? tiles : (int64_t)c->num_sms;
    const int g = coop_grid(c, k_bicg_persistent_f64, want, A.n_out, tiles);
    if (g < 1) return set_err(c, GS_ECUDA, "no co-resident grid for the persistent solver");
    // tiles of up to 32 sites, no more than the grid needs to cover the rest set
    // once (3840 sites on 152 blocks: 26 per tile, so every SM shares the work)
    int64_t ts = (A.n_out + g - 1) / g;
    if (ts > kSitesPerBlock) ts = kSitesPerBlock;
    if (ts < 1) ts = 1;
    GS_CUDA(c, cudaMemsetAsync(ps->words, 0, 4 * sizeof(unsigned int), c->stream));
    PArgs64 P;
    memset(&P, 0, sizeof P);
    P.A = A;
    P.C = C;
    P.C.epi_vec2 = w.rhat;   // <rhat, t> comes with t's stencil
    P.A.st = nullptr;
    P.C.st = nullptr;
    P.A.ran = P.C.ran = nullptr;
    P.b = b;
    P.x = x;
    P.r = w.r;
    P.rhat = w.rhat;
    P.p = w.p;
    P.v = w.v;
    P.s = w.s;
    P.t = w.t;
    P.n = n;
    P.ts = (int)ts;
    P.tol = tol;
    P.maxit = maxit;
    P.partial = (double*)ps->partial;
    P.sync.count = ps->words;
    P.sync.gen = ps->words + 1;
    P.sync.err = (int*)(ps->words + 2);
    P.sync.wait_ns = c->wait_ns;
    P.st = w.st;
    P.phases = c->prof.on ? c->prof.phases_dev : nullptr;
    void* args[] = {&P};
    GS_CUDA(c, cudaLaunchCooperativeKernel((const void*)k_bicg_persistent_f64, dim3(g),
                                           dim3(kPThreads), args, 0, c->stream));
    c->launches++;
    return GS_OK;
}

template <class S>
static gs_status persistent_bicg_lp_t(gs_ctx* c, const LpArgs& A, const LpArgs& C,
                                      const double2* r64, const double* rr64, void* const* vecs,
                                      LpState* st, int64_t n, float tol, int maxit) {
    PersistScratch* ps = nullptr;
    gs_status s = persist_scratch(c, &ps);
    if (s != GS_OK) return s;
    const int64_t blocks = (n + kPThreads - 1) / kPThreads;
    const int64_t want = blocks > (int64_t)c->num_sms ? blocks : (int64_t)c->num_sms;
    void (*kern)(PArgsLp) = k_bicg_persistent_lp<S>;
    // in a batched call on a small set: one pass with about 96 sites per block
    // (8^4, four FP32-inner solves at once: 87.1 solves/s with 40 + 24 + 40 +
    // 24 blocks, 84.9 with one full 128-site round, 75.8 with 76 blocks each)
    const int g = coop_grid(c, kern, want, n, (n + 95) / 96);
    if (g < 1) return set_err(c, GS_ECUDA, "no co-resident grid for the persistent solver");
    GS_CUDA(c, cudaMemsetAsync(ps->words, 0, 4 * sizeof(unsigned int), c->stream));
    PArgsLp P;
    memset(&P, 0, sizeof P);
    P.A = A;
    P.C = C;
    P.A.st = P.C.st = nullptr;
    P.A.ran = P.C.ran = nullptr;
    P.r64 = r64;
    P.rr64 = rr64;
    P.x = vecs[0];
    P.r = vecs[1];
    P.rhat = vecs[2];
    P.p = vecs[3];
    P.v = vecs[4];
    P.s = vecs[5];
    P.t = vecs[6];
    P.n = n;
    P.tol = tol;
    P.maxit = maxit;
    P.partial = (float*)ps->partial;
    P.sync.count = ps->words;
    P.sync.gen = ps->words + 1;
    P.sync.err = (int*)(ps->words + 2);
    P.sync.wait_ns = c->wait_ns;
    P.st = st;
    void* args[] = {&P};
    GS_CUDA(c, cudaLaunchCooperativeKernel((const void*)kern, dim3(g),
                                           dim3(kPThreads), args, 0, c->stream));
    c->launches++;
    return GS_OK;
}

gs_status persistent_bicg_lp(gs_ctx* c, int prec, const LpArgs& A, const LpArgs& C,
                             const double2* r64, const double* rr64, void* const* vecs, LpState* st,
                             int64_t n, float tol, int maxit) {
    if (prec == GS_BF16)
        return persistent_bicg_lp_t<__nv_bfloat16>(c, A, C, r64, rr64, vecs, st, n, tol, maxit);
    return persistent_bicg_lp_t<float>(c, A, C, r64, rr64, vecs, st, n, tol, maxit);
}

// Runs k_selftest_grid_timeout on a co-resident grid of two blocks with the
// persistent solvers' barrier words; returns the error word's status.
gs_status selftest_grid_timeout(gs_ctx* c, gs_status* result) {
    PersistScratch* ps = nullptr;
    gs_status s = persist_scratch(c, &ps);
    if (s != GS_OK) return s;
    GS_CUDA(c, cudaMemsetAsync(ps->words, 0, 4 * sizeof(unsigned int), c->stream));
    GridSync g;
    g.count = ps->words;
    g.gen = ps->words + 1;
    g.err = (int*)(ps->words + 2);
    g.wait_ns = c->wait_ns;
    const int* never = (const int*)(ps->words + 3);   // zeroed above, never written
    void* args[] = {&g, &never};
    GS_CUDA(c, cudaLaunchCooperativeKernel((const void*)k_selftest_grid_timeout, dim3(2),
                                           dim3(kPThreads), args, 0, c->stream));
    c->launches++;
    int h = 0;
    GS_CUDA(c, cudaMemcpyAsync(&h, ps->words + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    *result = (gs_status)h;
    return GS_OK;
}

}  // namespace gs
