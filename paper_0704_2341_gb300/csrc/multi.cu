// Several right-hand sides on one lattice, solved together.
//
// The low-precision vectors of N right-hand sides interleave the sources
// inside each site ([16-byte group][site][rhs]), so one thread per
// (site, rhs) reads its neighbours coalesced while the threads of the same
// site share the site's links through L1: the link bytes per site-source
// fall by a factor N (the stencil is HBM bound, so this is its gain; the
// SU(3) x (3 x N) products stay on the FP32 pipe, which is far from busy).
//
// The inner D_rr solves of all sources run in one persistent cooperative
// kernel with per-source BiCGStab scalars and convergence flags; the FP64
// defect correction and the outer GMRES(m) run the sources in lock step
// (one batched S_bb application per Arnoldi step).
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "gridsync.cuh"
#include "lowp.cuh"

namespace gs {

constexpr int kMaxRhs = 32;

namespace {

// thread block of the persistent multi-source kernel: N sources (fastest, x)
// by ceil(128 / N) sites (y), so every thread keeps one source
int multi_sites_per_block(int N) { return (128 + N - 1) / N; }
constexpr int kMultiMaxThreads = 256;

struct MArgs {
    const void* in;
    void* out;
    const void* links;   // [mu][3][n] (12-real links)
    const int2* nbr;     // [n][4]
    int64_t n;           // sites
    int N;               // sources
    float diag;
};

// one direction (both hops) for site k, source j; spinor index k*N + j
template <class S, int MU, bool CG>
__device__ __forceinline__ void mdir(const MArgs& a, int64_t k, int j, int2 nb, float (&acc)[24]) {
    const bool hf = nb.x >= 0, hb = nb.y >= 0;
    const int64_t nN = a.n * a.N;
    const int64_t jf = (hf ? nb.x : k) * a.N + j, jb = (hb ? nb.y : k) * a.N + j;
    const int64_t lb_site = hb ? nb.y : k;
    float pf[24], pb[24], lf[12], lb[12];
    Store<S>::template load_spinor<CG>(a.in, nN, jf, pf);
    Store<S>::template load_spinor<CG>(a.in, nN, jb, pb);
    Store<S>::load_link(a.links, a.n, MU, k, lf);
    Store<S>::load_link(a.links, a.n, MU, lb_site, lb);
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

// out(k, j) = diag in(k, j) + hops; returns the 24 output reals in acc
template <class S, bool CG>
__device__ __forceinline__ void mstencil(const MArgs& a, int64_t k, int j, float (&acc)[24]) {
    const int4 n01 = __ldg((const int4*)(a.nbr + k * 4));
    const int4 n23 = __ldg((const int4*)(a.nbr + k * 4) + 1);
#pragma unroll
    for (int q = 0; q < 24; ++q) acc[q] = 0.f;
    mdir<S, 0, CG>(a, k, j, make_int2(n01.x, n01.y), acc);
    mdir<S, 1, CG>(a, k, j, make_int2(n01.z, n01.w), acc);
    mdir<S, 2, CG>(a, k, j, make_int2(n23.x, n23.y), acc);
    mdir<S, 3, CG>(a, k, j, make_int2(n23.z, n23.w), acc);
    float self[24];
    const int64_t nN = a.n * a.N;
    Store<S>::template load_spinor<CG>(a.in, nN, k * a.N + j, self);
#pragma unroll
    for (int q = 0; q < 24; ++q) acc[q] = fmaf(a.diag, self[q], acc[q]);
}

template <class S>
__global__ void __launch_bounds__(128) k_dslash_multi(MArgs a) {
    const int64_t nN = a.n * a.N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nN;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / a.N;
        const int j = (int)(i - k * a.N);
        float acc[24];
        mstencil<S, false>(a, k, j, acc);
        Store<S>::store_spinor(a.out, nN, i, acc);
    }
}

// [N][n][12] complex128 <-> [group][n][N] low precision
template <class S>
__global__ void k_multi_pack(const double2* __restrict__ x, void* y, int64_t n, int N) {
    const int64_t nN = n * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nN;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / N;
        const int j = (int)(i - k * N);
        float f[24];
        const double2* src = x + ((int64_t)j * n + k) * 12;
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const double2 v = src[q];
            f[2 * q] = (float)v.x;
            f[2 * q + 1] = (float)v.y;
        }
        Store<S>::store_spinor(y, nN, i, f);
    }
}

template <class S>
__global__ void k_multi_unpack(const void* x, double2* __restrict__ y, int64_t n, int N) {
    const int64_t nN = n * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nN;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / N;
        const int j = (int)(i - k * N);
        float f[24];
        Store<S>::load_spinor(x, nN, i, f);
        double2* dst = y + ((int64_t)j * n + k) * 12;
#pragma unroll
        for (int q = 0; q < 12; ++q) dst[q] = make_double2((double)f[2 * q], (double)f[2 * q + 1]);
    }
}

// ---------------------------------------------------------------------------
// persistent multi-source BiCGStab (FP32 arithmetic)
// ---------------------------------------------------------------------------
struct MState {
    int iter[kMaxRhs];
    int status[kMaxRhs];
    float rr[kMaxRhs];
    float bb[kMaxRhs];
    int lockstep_iters;
    int err;
};

struct PMArgs {
    MArgs D;                 // the operator (in/out set per phase)
    const double2* r64;      // [N][n][12] FP64 right-hand sides of the cycle
    const double* rr64;      // [N] their squared norms
    void *x, *r, *rhat, *p, *v, *s, *t;
    float tol;
    int maxit;
    float* partial;          // [6 slots][gridDim][N][4]
    GridSync sync;
    MState* st;
};

// Per-source block sums of NV values; thread t holds source t % N.  The
// partial of (block, source j, q) goes to part[(block * N + j) * 4 + q].
template <int NV>
__device__ void m_put_partial(float* part, const float (&v)[NV], int N, float* buf) {
    const int B = blockDim.x * blockDim.y;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;  // source = t % N
#pragma unroll
    for (int q = 0; q < NV; ++q) buf[q * B + t] = v[q];
    __syncthreads();
    if (t < N * NV) {
        const int j = t % N, q = t / N;
        float s = 0.f;
        for (int u = j; u < B; u += N) s += buf[q * B + u];
        part[((int64_t)blockIdx.x * N + j) * 4 + q] = s;
    }
    __syncthreads();
}

// every block: per-source totals in the same order; tot[q * kMaxRhs + j]
template <int NV>
__device__ void m_grid_total(const float* part, int N, float* tot) {
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if (t < N * NV) {
        const int j = t % N, q = t / N;
        float s = 0.f;
        // L2 loads (written before the grid barrier), pipelined; fixed order
#pragma unroll 8
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(part + ((int64_t)b * N + j) * 4 + q);
        tot[q * kMaxRhs + j] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ float2 fm2(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 fd2(float2 a, float2 b) {
    const float inv = 1.0f / (b.x * b.x + b.y * b.y);
    return make_float2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}

template <class S>
__global__ void __launch_bounds__(kMultiMaxThreads) k_bicg_persistent_multi(PMArgs P) {
    extern __shared__ float buf[];            // [3][blockDim]
    __shared__ float tot[3 * kMaxRhs];
    __shared__ float2 alpha[kMaxRhs], omega[kMaxRhs], beta[kMaxRhs], rho[kMaxRhs];
    __shared__ float tol2[kMaxRhs];
    __shared__ int active[kMaxRhs], status[kMaxRhs], iters[kMaxRhs];
    __shared__ float rrs[kMaxRhs], bbs[kMaxRhs];
    __shared__ int n_active;
    const int N = P.D.N;
    const int64_t n = P.D.n, nN = n * N;
    const int j = threadIdx.x;                       // this thread's source
    const int64_t site0 = blockIdx.x * (int64_t)blockDim.y + threadIdx.y;
    const int64_t sstride = (int64_t)gridDim.x * blockDim.y;
    const int tflat = threadIdx.y * blockDim.x + threadIdx.x;
    const int64_t slot = (int64_t)gridDim.x * N * 4;
    float* part = P.partial;
    bool ok = true;
    int it = 0;
    MArgs A = P.D;  // v = D p
    A.in = P.p;
    A.out = P.v;
    MArgs C = P.D;  // t = D s
    C.in = P.s;
    C.out = P.t;
    // init: r = rhat = p = r64_j / ||r64_j||, x = 0
    {
        float v[1] = {0.f};
        const double nrm2 = P.rr64[j];
        const float scale = nrm2 > 0.0 ? (float)(1.0 / sqrt(nrm2)) : 0.f;
        for (int64_t k = site0; k < n; k += sstride) {
            const int64_t i = k * N + j;
            float f[24], z[24];
            const double2* src = P.r64 + ((int64_t)j * n + k) * 12;
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                const double2 w = __ldcg(src + q);
                f[2 * q] = (float)w.x * scale;
                f[2 * q + 1] = (float)w.y * scale;
                z[2 * q] = z[2 * q + 1] = 0.f;
            }
            Store<S>::store_spinor(P.r, nN, i, f);
            Store<S>::store_spinor(P.rhat, nN, i, f);
            Store<S>::store_spinor(P.p, nN, i, f);
            Store<S>::store_spinor(P.x, nN, i, z);
            Store<S>::template load_spinor<true>(P.r, nN, i, f);
#pragma unroll
            for (int q = 0; q < 24; ++q) v[0] = fmaf(f[q], f[q], v[0]);
        }
        m_put_partial<1>(part, v, N, buf);
        ok = grid_sync(P.sync);
        m_grid_total<1>(part, N, tot);
        if (tflat < N) {
            const int q = tflat;
            const float b = tot[q];
            bbs[q] = rrs[q] = b;
            rho[q] = make_float2(b, 0.f);
            tol2[q] = P.tol * P.tol * b;
            iters[q] = 0;
            status[q] = isfinite(b) ? GS_OK : GS_NONFINITE;
            active[q] = (b > 0.f && isfinite(b)) ? 1 : 0;
        }
        __syncthreads();
        if (tflat == 0) {
            int a = 0;
            for (int q = 0; q < N; ++q) a += active[q];
            n_active = a;
        }
        __syncthreads();
    }
    while (ok && n_active > 0 && it < P.maxit) {
        // A: v = D p ; <rhat, v>_j -> alpha_j
        {
            float e[2] = {0.f, 0.f};
            if (active[j]) {
                for (int64_t k = site0; k < n; k += sstride) {
                    const int64_t i = k * N + j;
                    float acc[24], w[24];
                    mstencil<S, true>(A, k, j, acc);
                    Store<S>::store_spinor(P.v, nN, i, acc);
                    Store<S>::template load_spinor<true>(P.rhat, nN, i, w);
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        e[0] = fmaf(w[2 * q], acc[2 * q], fmaf(w[2 * q + 1], acc[2 * q + 1], e[0]));
                        e[1] = fmaf(w[2 * q], acc[2 * q + 1], fmaf(-w[2 * q + 1], acc[2 * q], e[1]));
                    }
                }
            }
            m_put_partial<2>(part + slot, e, N, buf);
            if (!(ok = grid_sync(P.sync))) break;
            m_grid_total<2>(part + slot, N, tot);
            if (tflat < N && active[tflat]) {
                const int q = tflat;
                const float2 den = make_float2(tot[q], tot[kMaxRhs + q]);
                if (den.x == 0.f && den.y == 0.f) {
                    status[q] = GS_BREAKDOWN;
                    active[q] = 0;
                } else {
                    alpha[q] = fd2(rho[q], den);
                    if (!isfinite(alpha[q].x) || !isfinite(alpha[q].y)) {
                        status[q] = GS_NONFINITE;
                        active[q] = 0;
                    }
                }
            }
            __syncthreads();
        }
        // B: s = r - alpha v ; x += alpha p ; ||s||^2
        {
            float e[1] = {0.f};
            if (active[j]) {
                const float2 al = alpha[j];
                for (int64_t k = site0; k < n; k += sstride) {
                    const int64_t i = k * N + j;
                    float fr[24], fv[24], fp[24], fx[24];
                    Store<S>::template load_spinor<true>(P.r, nN, i, fr);
                    Store<S>::template load_spinor<true>(P.v, nN, i, fv);
                    Store<S>::template load_spinor<true>(P.p, nN, i, fp);
                    Store<S>::template load_spinor<true>(P.x, nN, i, fx);
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        const float vr = fv[2 * q], vi = fv[2 * q + 1];
                        fr[2 * q] -= al.x * vr - al.y * vi;
                        fr[2 * q + 1] -= al.x * vi + al.y * vr;
                        const float pr = fp[2 * q], pi = fp[2 * q + 1];
                        fx[2 * q] = fmaf(al.x, pr, fmaf(-al.y, pi, fx[2 * q]));
                        fx[2 * q + 1] = fmaf(al.x, pi, fmaf(al.y, pr, fx[2 * q + 1]));
                    }
                    Store<S>::store_spinor(P.s, nN, i, fr);
                    Store<S>::store_spinor(P.x, nN, i, fx);
#pragma unroll
                    for (int q = 0; q < 24; ++q) e[0] = fmaf(fr[q], fr[q], e[0]);
                }
            }
            m_put_partial<1>(part + 2 * slot, e, N, buf);
            if (!(ok = grid_sync(P.sync))) break;
            m_grid_total<1>(part + 2 * slot, N, tot);
            if (tflat < N && active[tflat]) {
                const int q = tflat;
                if (!isfinite(tot[q])) {
                    status[q] = GS_NONFINITE;
                    active[q] = 0;
                } else if (tot[q] <= tol2[q]) {  // converged on s: x already updated
                    rrs[q] = tot[q];
                    iters[q] += 1;
                    active[q] = -1;              // finished this iteration
                }
            }
            __syncthreads();
        }
        // C: t = D s ; <t, s>_j, <t, t>_j -> omega_j
        {
            float e[3] = {0.f, 0.f, 0.f};
            if (active[j] > 0) {
                for (int64_t k = site0; k < n; k += sstride) {
                    const int64_t i = k * N + j;
                    float acc[24], w[24];
                    mstencil<S, true>(C, k, j, acc);
                    Store<S>::store_spinor(P.t, nN, i, acc);
                    Store<S>::template load_spinor<true>(P.s, nN, i, w);
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        const float tr = acc[2 * q], ti = acc[2 * q + 1];
                        e[0] = fmaf(tr, w[2 * q], fmaf(ti, w[2 * q + 1], e[0]));
                        e[1] = fmaf(tr, w[2 * q + 1], fmaf(-ti, w[2 * q], e[1]));
                        e[2] = fmaf(tr, tr, fmaf(ti, ti, e[2]));
                    }
                }
            }
            m_put_partial<3>(part + 3 * slot, e, N, buf);
            if (!(ok = grid_sync(P.sync))) break;
            m_grid_total<3>(part + 3 * slot, N, tot);
            if (tflat < N && active[tflat] > 0) {
                const int q = tflat;
                const float tt = tot[2 * kMaxRhs + q];
                const float inv = tt > 0.f ? 1.f / tt : 0.f;
                omega[q] = make_float2(tot[q] * inv, tot[kMaxRhs + q] * inv);
                if (!isfinite(omega[q].x) || !isfinite(omega[q].y)) {
                    status[q] = GS_NONFINITE;
                    active[q] = 0;
                }
            }
            __syncthreads();
        }
        // D: x += omega s ; r = s - omega t ; <rhat, r>_j, ||r_j||^2
        {
            float e[3] = {0.f, 0.f, 0.f};
            if (active[j] > 0) {
                const float2 om = omega[j];
                for (int64_t k = site0; k < n; k += sstride) {
                    const int64_t i = k * N + j;
                    float fs[24], ft[24], fh[24], fx[24];
                    Store<S>::template load_spinor<true>(P.s, nN, i, fs);
                    Store<S>::template load_spinor<true>(P.t, nN, i, ft);
                    Store<S>::template load_spinor<true>(P.rhat, nN, i, fh);
                    Store<S>::template load_spinor<true>(P.x, nN, i, fx);
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
                        e[0] = fmaf(fh[2 * q], r_, fmaf(fh[2 * q + 1], i_, e[0]));
                        e[1] = fmaf(fh[2 * q], i_, fmaf(-fh[2 * q + 1], r_, e[1]));
                        e[2] = fmaf(r_, r_, fmaf(i_, i_, e[2]));
                    }
                    Store<S>::store_spinor(P.x, nN, i, fx);
                    Store<S>::store_spinor(P.r, nN, i, fs);
                }
            }
            m_put_partial<3>(part + 4 * slot, e, N, buf);
            if (!(ok = grid_sync(P.sync))) break;
            m_grid_total<3>(part + 4 * slot, N, tot);
            if (tflat < N && active[tflat] > 0) {
                const int q = tflat;
                const float2 rho_new = make_float2(tot[q], tot[kMaxRhs + q]);
                const float rr = tot[2 * kMaxRhs + q];
                const float2 om = omega[q];
                rrs[q] = rr;
                iters[q] += 1;
                if (!isfinite(rho_new.x) || !isfinite(rho_new.y) || !isfinite(rr)) {
                    status[q] = GS_NONFINITE;
                    active[q] = 0;
                } else if (rr <= tol2[q]) {
                    active[q] = 0;
                } else if ((om.x == 0.f && om.y == 0.f) || (rho_new.x == 0.f && rho_new.y == 0.f)) {
                    status[q] = GS_BREAKDOWN;
                    active[q] = 0;
                } else {
                    beta[q] = fm2(fd2(rho_new, rho[q]), fd2(alpha[q], om));
                    rho[q] = rho_new;
                }
            }
            if (tflat < N && active[tflat] < 0) active[tflat] = 0;
            __syncthreads();
        }
        // E: p = r + beta (p - omega v)
        {
            if (active[j] > 0) {
                const float2 be = beta[j], om = omega[j];
                for (int64_t k = site0; k < n; k += sstride) {
                    const int64_t i = k * N + j;
                    float fr[24], fv[24], fp[24];
                    Store<S>::template load_spinor<true>(P.r, nN, i, fr);
                    Store<S>::template load_spinor<true>(P.v, nN, i, fv);
                    Store<S>::template load_spinor<true>(P.p, nN, i, fp);
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        const float vr = fv[2 * q], vi = fv[2 * q + 1];
                        const float qr = fp[2 * q] - (om.x * vr - om.y * vi);
                        const float qi = fp[2 * q + 1] - (om.x * vi + om.y * vr);
                        fp[2 * q] = fmaf(be.x, qr, fmaf(-be.y, qi, fr[2 * q]));
                        fp[2 * q + 1] = fmaf(be.x, qi, fmaf(be.y, qr, fr[2 * q + 1]));
                    }
                    Store<S>::store_spinor(P.p, nN, i, fp);
                }
            }
            if (tflat == 0) {
                int a = 0;
                for (int q = 0; q < N; ++q) a += active[q] > 0;
                n_active = a;
            }
            ++it;
            if (!(ok = grid_sync(P.sync))) break;
        }
    }
    if (blockIdx.x == 0) {
        if (tflat < N) {
            const int q = tflat;
            P.st->iter[q] = iters[q];
            P.st->status[q] = ok ? status[q] : (int)GS_TIMEOUT;
            P.st->rr[q] = rrs[q];
            P.st->bb[q] = bbs[q];
        }
        if (tflat == 0) {
            P.st->lockstep_iters = it;
            P.st->err = ok ? 0 : (int)GS_TIMEOUT;
        }
    }
}

// z_j += sqrt(rr64_j) e_j
template <class S>
__global__ void k_multi_accum(const void* e, const double* __restrict__ rr64, double2* z, int64_t n,
                              int N) {
    const int64_t nN = n * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nN;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / N;
        const int j = (int)(i - k * N);
        const double scale = sqrt(rr64[j]);
        float f[24];
        Store<S>::load_spinor(e, nN, i, f);
        double2* dst = z + ((int64_t)j * n + k) * 12;
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            double2 zz = dst[q];
            zz.x = fma(scale, (double)f[2 * q], zz.x);
            zz.y = fma(scale, (double)f[2 * q + 1], zz.y);
            dst[q] = zz;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct MultiWork {
    int prec = -1;
    size_t cap = 0;             // bytes per low-precision vector
    void* lp[7] = {};           // x, r, rhat, p, v, s, t
    size_t cap64 = 0;           // bytes of one FP64 multi-source rest vector
    double2* r64 = nullptr;     // [N][n][12]
    double* rr64 = nullptr;     // [kMaxRhs]
    double* rr64_host = nullptr;
    float* partial = nullptr;   // 6 slots x kMaxRedBlocks x kMaxRhs x 4
    unsigned int* words = nullptr;
    MState* st = nullptr;
    MState* st_host = nullptr;
    // S_bb / solve workspaces
    size_t capb = 0, capr = 0, capz = 0, capv = 0, capF = 0, capZ = 0, capX = 0, capWB = 0;
    double2 *t64 = nullptr, *z64 = nullptr;     // rest vectors [N][nr][12]
    double2 *F = nullptr, *Z = nullptr, *X = nullptr;  // full vectors [N][V][12]
    double2 *wb = nullptr, *basis = nullptr, *w = nullptr, *xb = nullptr;
    int cap_m = 0;
    double2* hbuf = nullptr;
    double2* hbuf_host = nullptr;
    double2* y = nullptr;
    double2* y_host = nullptr;
    RedScratch red;
};

static MultiWork* multi_of(gs_ctx* c) {
    if (!c->multi) c->multi = new MultiWork();
    return (MultiWork*)c->multi;
}

void free_multi(gs_ctx* c) {
    MultiWork* m = (MultiWork*)c->multi;
    if (!m) return;
    for (void* p : m->lp) cudaFree(p);
    void* d[] = {m->r64, m->rr64, m->partial, m->words, m->st, m->t64, m->z64, m->F, m->Z, m->X,
                 m->wb, m->basis, m->w, m->xb, m->hbuf, m->y, m->red.partial, m->red.counter};
    for (void* p : d) cudaFree(p);
    if (m->rr64_host) cudaFreeHost(m->rr64_host);
    if (m->st_host) cudaFreeHost(m->st_host);
    if (m->hbuf_host) cudaFreeHost(m->hbuf_host);
    if (m->y_host) cudaFreeHost(m->y_host);
    delete m;
    c->multi = nullptr;
}

static gs_status grow(gs_ctx* c, void** p, size_t* cap, size_t need) {
    if (*cap >= need && *p) return GS_OK;
    cudaFree(*p);
    *p = nullptr;
    if (cudaMalloc(p, need) != cudaSuccess) {
        cudaGetLastError();
        *cap = 0;
        return set_err(c, GS_ENOMEM, "allocating %zu bytes for the multi-source solve failed", need);
    }
    *cap = need;
    return GS_OK;
}

static gs_status multi_fixed(gs_ctx* c, MultiWork* m) {
    if (m->st) return GS_OK;
    if (cudaMalloc(&m->rr64, kMaxRhs * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->partial, 6 * (size_t)kMaxRedBlocks * kMaxRhs * 4 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->words, 4 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&m->st, sizeof(MState)) != cudaSuccess ||
        cudaMalloc(&m->hbuf, (size_t)kMaxRhs * (2 * (kMaxRestart + 2) + 1) * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&m->y, (size_t)kMaxRhs * (kMaxRestart + 1) * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&m->red.partial, kRedScratchDoubles * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->red.counter, sizeof(unsigned int)) != cudaSuccess ||
        cudaHostAlloc(&m->rr64_host, kMaxRhs * sizeof(double), 0) != cudaSuccess ||
        cudaHostAlloc(&m->st_host, sizeof(MState), 0) != cudaSuccess ||
        cudaHostAlloc(&m->hbuf_host, (size_t)kMaxRhs * (2 * (kMaxRestart + 2) + 1) * sizeof(double2), 0) != cudaSuccess ||
        cudaHostAlloc(&m->y_host, (size_t)kMaxRhs * (kMaxRestart + 1) * sizeof(double2), 0) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, GS_ENOMEM, "allocating the multi-source state failed");
    }
    GS_CUDA(c, cudaMemsetAsync(m->red.counter, 0, sizeof(unsigned int), c->stream));
    return GS_OK;
}

static size_t lp_spinor_bytes(int prec) { return prec == GS_BF16 ? 48 : 96; }

// norms of N FP64 rest vectors -> m->rr64 (device) and m->rr64_host
static gs_status multi_norms(gs_ctx* c, MultiWork* m, const double2* v, int64_t n, int N) {
    for (int j = 0; j < N; ++j) {
        gs_status s = launch_norm2(c, m->red, v + (size_t)j * n * kSiteC, n * kSiteC, m->rr64 + j);
        if (s != GS_OK) return s;
    }
    GS_CUDA(c, cudaMemcpyAsync(m->rr64_host, m->rr64, N * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

// z_j = D_rr^-1 t_j for N sources (rest vectors [N][nr][12]); FP64 defect
// correction around the persistent multi-source low-precision BiCGStab.
static gs_status inner_solve_multi(gs_ctx* c, const Plan* p, int N, const double2* t, double2* z,
                                   const gs_solve_opts& o, gs_solve_stats& st) {
    const int prec = (o.inner_prec == GS_BF16) ? GS_BF16 : GS_F32;
    MultiWork* m = multi_of(c);
    gs_status s = multi_fixed(c, m);
    if (s != GS_OK) return s;
    LowpTables tb;
    if ((s = lowp_tables(c, p, prec, &tb)) != GS_OK) return s;
    const int64_t n = tb.n;
    const size_t lpb = (size_t)n * N * lp_spinor_bytes(prec);
    if (m->prec != prec || m->cap < lpb) {
        for (void*& q : m->lp) {
            cudaFree(q);
            q = nullptr;
        }
        m->cap = 0;
        for (void*& q : m->lp)
            if (cudaMalloc(&q, lpb) != cudaSuccess) {
                cudaGetLastError();
                return set_err(c, GS_ENOMEM, "allocating multi-source vectors failed");
            }
        m->cap = lpb;
        m->prec = prec;
    }
    const size_t vb = (size_t)N * n * kSiteC * sizeof(double2);
    if ((s = grow(c, (void**)&m->r64, &m->cap64, vb)) != GS_OK) return s;
    GS_CUDA(c, cudaMemsetAsync(z, 0, vb, c->stream));
    GS_CUDA(c, cudaMemcpyAsync(m->r64, t, vb, cudaMemcpyDeviceToDevice, c->stream));
    if ((s = multi_norms(c, m, m->r64, n, N)) != GS_OK) return s;
    std::vector<double> tt(N), target(N);
    bool all = true;
    for (int j = 0; j < N; ++j) {
        tt[j] = m->rr64_host[j];
        if (!isfinite(tt[j])) return set_err(c, GS_NONFINITE, "non-finite right-hand side");
        target[j] = o.inner_tol * o.inner_tol * tt[j];
        all = all && (tt[j] <= target[j]);
    }
    st.inner_solves += N;
    if (all) return GS_OK;
    const float lo_tol = (float)(o.lowp_tol > 0.0 ? o.lowp_tol : (prec == GS_BF16 ? 3e-2 : 1e-5));
    const int SB = multi_sites_per_block(N);
    const int B = N * SB;
    int per_sm = 0;
    const size_t dsm = 3 * (size_t)B * sizeof(float);
    auto kern = (prec == GS_BF16) ? k_bicg_persistent_multi<__nv_bfloat16>
                                  : k_bicg_persistent_multi<float>;
    GS_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, dsm));
    if (per_sm < 1) return set_err(c, GS_ECUDA, "multi-source kernel does not fit on an SM");
    int64_t g = coop_blocks(c, per_sm, n);
    const int64_t want = (n + SB - 1) / SB;
    if (g > want) g = want < c->num_sms ? (want < 1 ? 1 : want) : want;
    if (g > (int64_t)per_sm * c->num_sms) g = (int64_t)per_sm * c->num_sms;
    if (g > kMaxRedBlocks) g = kMaxRedBlocks;
    StencilArgs ra;
    memset(&ra, 0, sizeof ra);
    ra.o0 = p->nb;
    ra.n_out = n;
    ra.a0 = p->nb;
    ra.a1 = c->V;
    ra.b1 = c->V;
    ra.diag = c->m0 + 4.0;
    ra.negate = 1;
    ra.plan = p;
    ra.nbr = p->nbr;
    ra.links = p->links;
    std::vector<double> rr(tt);
    std::vector<int> stalls(N, 0);
    long long lp_iters = 0;
    int cycles = 0;
    for (; cycles < 100; ++cycles) {
        bool pending = false;
        for (int j = 0; j < N; ++j) pending = pending || (rr[j] > target[j] && stalls[j] < 3);
        if (!pending) break;
        // sources already converged get a zero right-hand side (they stay put)
        for (int j = 0; j < N; ++j)
            if (!(rr[j] > target[j]) || stalls[j] >= 3) {
                GS_CUDA(c, cudaMemsetAsync(m->r64 + (size_t)j * n * kSiteC, 0,
                                           (size_t)n * kSiteC * sizeof(double2), c->stream));
                m->rr64_host[j] = 0.0;
            }
        GS_CUDA(c, cudaMemcpyAsync(m->rr64, m->rr64_host, N * sizeof(double), cudaMemcpyHostToDevice,
                                   c->stream));
        GS_CUDA(c, cudaMemsetAsync(m->words, 0, 4 * sizeof(unsigned int), c->stream));
        PMArgs P;
        memset(&P, 0, sizeof P);
        P.D.links = tb.links;
        P.D.nbr = tb.nbr;
        P.D.n = n;
        P.D.N = N;
        P.D.diag = (float)(c->m0 + 4.0);
        P.r64 = m->r64;
        P.rr64 = m->rr64;
        P.x = m->lp[0];
        P.r = m->lp[1];
        P.rhat = m->lp[2];
        P.p = m->lp[3];
        P.v = m->lp[4];
        P.s = m->lp[5];
        P.t = m->lp[6];
        P.tol = lo_tol;
        P.maxit = o.inner_max_iter;
        P.partial = m->partial;
        P.sync.count = m->words;
        P.sync.gen = m->words + 1;
        P.sync.err = (int*)(m->words + 2);
        P.sync.wait_ns = c->wait_ns;
        P.st = m->st;
        void* args[] = {&P};
        GS_CUDA(c, cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)g), dim3(N, SB), args,
                                               dsm, c->stream));
        c->launches++;
        GS_CUDA(c, cudaMemcpyAsync(m->st_host, m->st, sizeof(MState), cudaMemcpyDeviceToHost,
                                   c->stream));
        // z_j += ||r_j|| e_j ; r = t - D_rr z ; norms
        const int ga = grid_for(n * N, 256, c->num_sms * 8);
        if (prec == GS_BF16)
            k_multi_accum<__nv_bfloat16><<<ga, 256, 0, c->stream>>>(m->lp[0], m->rr64, z, n, N);
        else
            k_multi_accum<float><<<ga, 256, 0, c->stream>>>(m->lp[0], m->rr64, z, n, N);
        c->launches++;
        GS_CHECK_LAUNCH(c);
        for (int j = 0; j < N; ++j) {
            ra.out = m->r64 + (size_t)j * n * kSiteC;
            ra.inA = z + (size_t)j * n * kSiteC;
            ra.addend = t + (size_t)j * n * kSiteC;
            if ((s = launch_stencil_f64(c, ra)) != GS_OK) return s;
        }
        if ((s = multi_norms(c, m, m->r64, n, N)) != GS_OK) return s;
        if (m->st_host->err) return set_err(c, GS_TIMEOUT, "multi-source inner solve: barrier timeout");
        lp_iters += m->st_host->lockstep_iters;
        for (int j = 0; j < N; ++j) {
            const double nr2 = m->rr64_host[j];
            if (!isfinite(nr2)) return set_err(c, GS_NONFINITE, "non-finite multi-source residual");
            if (rr[j] > target[j]) stalls[j] = (nr2 > 0.25 * rr[j]) ? stalls[j] + 1 : 0;
            rr[j] = nr2;
        }
    }
    st.inner_iters += lp_iters;
    st.lowp_cycles += cycles;
    if (lp_iters > st.inner_max_seen) st.inner_max_seen = (int)lp_iters;
    gs_status res = GS_OK;
    for (int j = 0; j < N; ++j) {
        const double rel = tt[j] > 0.0 ? sqrt(rr[j] / tt[j]) : 0.0;
        if (rel > st.inner_residual) st.inner_residual = rel;
        if (rr[j] > target[j]) res = GS_MAXITER;
    }
    if (res != GS_OK)
        return set_err(c, res, "multi-source inner solve stalled (residual %.3e)", st.inner_residual);
    return GS_OK;
}

// y_j = S_bb x_j for N coarse vectors ([N][nb][12])
static gs_status schur_apply_multi(gs_ctx* c, const Plan* p, int N, const double2* xb, double2* yb,
                                   const gs_solve_opts& o, gs_solve_stats& st) {
    MultiWork* m = multi_of(c);
    const int64_t nb = p->nb, V = c->V, nr = V - nb;
    const size_t rb = (size_t)N * nr * kSiteC * sizeof(double2);
    gs_status s;
    if ((s = grow(c, (void**)&m->t64, &m->capr, rb)) != GS_OK) return s;
    if ((s = grow(c, (void**)&m->z64, &m->capz, rb)) != GS_OK) return s;
    StencilArgs a;
    memset(&a, 0, sizeof a);
    a.diag = c->m0 + 4.0;
    a.plan = p;
    a.nbr = p->nbr;
    a.links = p->links;
    for (int j = 0; j < N; ++j) {  // t_j = -D_rb x_j
        a.out = m->t64 + (size_t)j * nr * kSiteC;
        a.o0 = nb;
        a.n_out = nr;
        a.inA = xb + (size_t)j * nb * kSiteC;
        a.a0 = 0;
        a.a1 = nb;
        a.b1 = nb;
        a.negate = 1;
        if ((s = launch_stencil_f64(c, a)) != GS_OK) return s;
    }
    gs_status si = inner_solve_multi(c, p, N, m->t64, m->z64, o, st);
    if (si != GS_OK && si != GS_MAXITER) return si;
    for (int j = 0; j < N; ++j) {  // y_j = D_bb x_j + D_br z_j
        a.out = yb + (size_t)j * nb * kSiteC;
        a.o0 = 0;
        a.n_out = nb;
        a.inA = xb + (size_t)j * nb * kSiteC;
        a.a0 = 0;
        a.a1 = nb;
        a.inB = m->z64 + (size_t)j * nr * kSiteC;
        a.b1 = V;
        a.negate = 0;
        if ((s = launch_stencil_f64(c, a)) != GS_OK) return s;
    }
    return si;
}

// Lock-step restarted GMRES(m) for N systems S_bb x_j = w_j.
static gs_status outer_gmres_multi(gs_ctx* c, const Plan* p, int N, const double2* wb, double2* xb,
                                   const gs_solve_opts& o, gs_solve_stats& st) {
    using cplx = std::complex<double>;
    MultiWork* m = multi_of(c);
    const int64_t nbs = p->nb, n = nbs * kSiteC;
    const int M = o.restart;
    gs_status s;
    const size_t vb = (size_t)n * sizeof(double2);
    if ((s = grow(c, (void**)&m->basis, &m->capv, vb * N * (M + 1))) != GS_OK) return s;
    if (!m->w) {
        if (cudaMalloc(&m->w, vb * N) != cudaSuccess || cudaMalloc(&m->xb, vb * N) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GS_ENOMEM, "allocating GMRES vectors failed");
        }
        m->capb = vb * N;
    } else if (m->capb < vb * N) {
        cudaFree(m->w);
        cudaFree(m->xb);
        m->w = m->xb = nullptr;
        if (cudaMalloc(&m->w, vb * N) != cudaSuccess || cudaMalloc(&m->xb, vb * N) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GS_ENOMEM, "allocating GMRES vectors failed");
        }
        m->capb = vb * N;
    }
    auto Vj = [&](int j, int i) { return m->basis + ((size_t)j * (M + 1) + i) * n; };
    GS_CUDA(c, cudaMemsetAsync(xb, 0, vb * N, c->stream));
    std::vector<double> bnorm(N);
    if ((s = multi_norms(c, m, wb, nbs, N)) != GS_OK) return s;
    std::vector<char> done(N, 0);
    for (int j = 0; j < N; ++j) {
        bnorm[j] = sqrt(m->rr64_host[j]);
        if (!isfinite(bnorm[j])) return set_err(c, GS_NONFINITE, "non-finite right-hand side");
        if (bnorm[j] == 0.0) done[j] = 1;
    }
    std::vector<cplx> H((size_t)N * (M + 1) * M), g((size_t)N * (M + 1)), cs((size_t)N * M),
        sn((size_t)N * M);
    std::vector<int> kk(N, 0);
    std::vector<char> frozen(N, 0);
    int total = 0;
    bool first = true;
    gs_status inner_flag = GS_OK;
    double worst = 0.0;
    while (true) {
        // residuals r_j = w_j - S x_j (tight), except on the first cycle (x = 0)
        if (first) {
            for (int j = 0; j < N; ++j)
                GS_CUDA(c, cudaMemcpyAsync(Vj(j, 0), wb + (size_t)j * n, vb, cudaMemcpyDeviceToDevice,
                                           c->stream));
        } else {
            s = schur_apply_multi(c, p, N, xb, m->w, o, st);
            if (s == GS_MAXITER) inner_flag = s;
            else if (s != GS_OK) return s;
            for (int j = 0; j < N; ++j) {
                if ((s = launch_scale_copy(c, wb + (size_t)j * n, Vj(j, 0), n, 1.0)) != GS_OK) return s;
                if ((s = launch_axpby(c, make_double2(-1.0, 0.0), m->w + (size_t)j * n,
                                      make_double2(1.0, 0.0), Vj(j, 0), n)) != GS_OK)
                    return s;
            }
        }
        // norms of the N residuals (gather them into the w buffer layout)
        for (int j = 0; j < N; ++j)
            if ((s = launch_norm2(c, m->red, Vj(j, 0), n, m->rr64 + j)) != GS_OK) return s;
        GS_CUDA(c, cudaMemcpyAsync(m->rr64_host, m->rr64, N * sizeof(double), cudaMemcpyDeviceToHost,
                                   c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        first = false;
        bool all = true;
        worst = 0.0;
        for (int j = 0; j < N; ++j) {
            if (bnorm[j] == 0.0) continue;
            const double beta = sqrt(m->rr64_host[j]);
            if (!isfinite(beta)) return set_err(c, GS_NONFINITE, "non-finite outer residual");
            worst = std::max(worst, beta / bnorm[j]);
            done[j] = beta <= o.tol * bnorm[j];
            all = all && done[j];
            frozen[j] = done[j];
            kk[j] = 0;
            if (!done[j]) {
                if ((s = launch_scale_copy(c, Vj(j, 0), Vj(j, 0), n, 1.0 / beta)) != GS_OK) return s;
                for (int i = 0; i <= M; ++i) g[(size_t)j * (M + 1) + i] = 0.0;
                g[(size_t)j * (M + 1)] = beta;
            }
        }
        st.outer_residual = worst;
        if (all || total >= o.max_iter) break;
        for (int i = 0; i < M; ++i) {
            // batched S application on V_i of the unfrozen sources (zeros for the frozen)
            double eta = o.relax_cap;
            for (int j = 0; j < N; ++j) {
                double2* dst = m->w + (size_t)j * n;  // used as the batched input copy
                if (frozen[j]) {
                    GS_CUDA(c, cudaMemsetAsync(dst, 0, vb, c->stream));
                } else {
                    GS_CUDA(c, cudaMemcpyAsync(dst, Vj(j, i), vb, cudaMemcpyDeviceToDevice, c->stream));
                    const double rel = std::abs(g[(size_t)j * (M + 1) + i]) / bnorm[j];
                    double e = rel > 0.0 ? o.inner_tol / rel : o.relax_cap;
                    eta = std::min(eta, e);
                }
            }
            gs_solve_opts oj = o;
            if (o.inner_relax) oj.inner_tol = std::max(o.inner_tol, std::min(eta, o.relax_cap));
            // S applied to the batched copy in m->w, output in m->xb, then
            // moved to basis slot i+1 of each source to be orthogonalised there
            double2* tmp_out = m->xb;
            s = schur_apply_multi(c, p, N, m->w, tmp_out, oj, st);
            if (s == GS_MAXITER) inner_flag = s;
            else if (s != GS_OK) return s;
            for (int j = 0; j < N; ++j)
                GS_CUDA(c, cudaMemcpyAsync(Vj(j, i + 1), tmp_out + (size_t)j * n, vb,
                                           cudaMemcpyDeviceToDevice, c->stream));
            ++total;
            // CGS2 per unfrozen source; H column to the host
            const size_t hstride = 2 * (kMaxRestart + 2) + 1;
            for (int j = 0; j < N; ++j) {
                if (frozen[j]) continue;
                double2* h = m->hbuf + (size_t)j * hstride;
                double2* h2 = h + (M + 2);
                double2* wj = Vj(j, i + 1);
                if ((s = launch_multidot(c, m->red, Vj(j, 0), n, i + 1, wj, n, h, 0)) != GS_OK) return s;
                if ((s = launch_multiaxpy(c, Vj(j, 0), n, i + 1, h, wj, n, -1)) != GS_OK) return s;
                if ((s = launch_multidot(c, m->red, Vj(j, 0), n, i + 1, wj, n, h2, 0)) != GS_OK) return s;
                if ((s = launch_multiaxpy(c, Vj(j, 0), n, i + 1, h2, wj, n, -1)) != GS_OK) return s;
                if ((s = launch_norm2(c, m->red, wj, n, (double*)(h + 2 * (M + 2)))) != GS_OK) return s;
            }
            GS_CUDA(c, cudaMemcpyAsync(m->hbuf_host, m->hbuf, (size_t)N * hstride * sizeof(double2),
                                       cudaMemcpyDeviceToHost, c->stream));
            GS_CUDA(c, cudaStreamSynchronize(c->stream));
            bool any = false;
            for (int j = 0; j < N; ++j) {
                if (frozen[j]) continue;
                const double2* hh = m->hbuf_host + (size_t)j * hstride;
                cplx* Hj = H.data() + (size_t)j * (M + 1) * M;
                cplx* gj = g.data() + (size_t)j * (M + 1);
                cplx* cj = cs.data() + (size_t)j * M;
                cplx* sj = sn.data() + (size_t)j * M;
                const double hn = sqrt(hh[2 * (M + 2)].x);
                if (!isfinite(hn)) return set_err(c, GS_NONFINITE, "non-finite Arnoldi norm");
                for (int q = 0; q <= i; ++q)
                    Hj[(size_t)q * M + i] = cplx(hh[q].x + hh[M + 2 + q].x, hh[q].y + hh[M + 2 + q].y);
                Hj[(size_t)(i + 1) * M + i] = hn;
                if (hn > 0.0)
                    if ((s = launch_scale_copy(c, Vj(j, i + 1), Vj(j, i + 1), n, 1.0 / hn)) != GS_OK) return s;
                for (int q = 0; q < i; ++q) {
                    const cplx a0 = Hj[(size_t)q * M + i], a1 = Hj[(size_t)(q + 1) * M + i];
                    Hj[(size_t)q * M + i] = std::conj(cj[q]) * a0 + std::conj(sj[q]) * a1;
                    Hj[(size_t)(q + 1) * M + i] = -sj[q] * a0 + cj[q] * a1;
                }
                const cplx aa = Hj[(size_t)i * M + i], bb = Hj[(size_t)(i + 1) * M + i];
                const double hh2 = sqrt(std::norm(aa) + std::norm(bb));
                if (hh2 > 0.0) {
                    cj[i] = aa / hh2;
                    sj[i] = bb / hh2;
                } else {
                    cj[i] = 1.0;
                    sj[i] = 0.0;
                }
                Hj[(size_t)i * M + i] = hh2;
                Hj[(size_t)(i + 1) * M + i] = 0.0;
                gj[i + 1] = -sj[i] * gj[i];
                gj[i] = std::conj(cj[i]) * gj[i];
                kk[j] = i + 1;
                if (std::abs(gj[i + 1]) <= o.tol * bnorm[j] || hn == 0.0) frozen[j] = 1;
                any = any || !frozen[j];
            }
            if (!any || total >= o.max_iter) break;
        }
        // x_j += V_j y_j
        for (int j = 0; j < N; ++j) {
            const int k = kk[j];
            if (done[j] || k == 0) continue;
            const cplx* Hj = H.data() + (size_t)j * (M + 1) * M;
            const cplx* gj = g.data() + (size_t)j * (M + 1);
            std::vector<cplx> y(k);
            for (int q = k - 1; q >= 0; --q) {
                cplx acc = gj[q];
                for (int l = q + 1; l < k; ++l) acc -= Hj[(size_t)q * M + l] * y[l];
                y[q] = acc / Hj[(size_t)q * M + q];
            }
            double2* yh = m->y_host + (size_t)j * (kMaxRestart + 1);
            for (int q = 0; q < k; ++q) yh[q] = make_double2(y[q].real(), y[q].imag());
        }
        GS_CUDA(c, cudaMemcpyAsync(m->y, m->y_host, (size_t)N * (kMaxRestart + 1) * sizeof(double2),
                                   cudaMemcpyHostToDevice, c->stream));
        for (int j = 0; j < N; ++j) {
            const int k = kk[j];
            if (done[j] || k == 0) continue;
            if ((s = launch_multiaxpy(c, Vj(j, 0), n, k, m->y + (size_t)j * (kMaxRestart + 1),
                                      xb + (size_t)j * n, n, +1)) != GS_OK)
                return s;
        }
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int j = 0; j < N; ++j) frozen[j] = 0;
    }
    st.outer_iters = total;
    for (int j = 0; j < N; ++j)
        if (!done[j] && bnorm[j] > 0.0)
            return set_err(c, GS_MAXITER, "batched GMRES(%d) reached %d steps (worst residual %.3e)",
                           M, total, worst);
    return inner_flag;
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_lowp_pack_multi(gs_ctx* c, int type, int dir, int inverse, int prec, int nrhs,
                             const void* x_dev, void* x_lp_dev) {
    if (!c) return GS_EINVAL;
    if (nrhs < 1 || nrhs > kMaxRhs) return set_err(c, GS_EINVAL, "nrhs %d not in 1..%d", nrhs, kMaxRhs);
    if (prec != GS_F32 && prec != GS_BF16) return set_err(c, GS_EINVAL, "precision %d", prec);
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    if (!x_dev || !x_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    LowpTables tb;
    if ((s = lowp_tables(c, p, prec, &tb)) != GS_OK) return s;
    const int g = grid_for(tb.n * nrhs, 256, c->num_sms * 8);
    if (prec == GS_BF16)
        k_multi_pack<__nv_bfloat16><<<g, 256, 0, c->stream>>>((const double2*)x_dev, x_lp_dev, tb.n, nrhs);
    else
        k_multi_pack<float><<<g, 256, 0, c->stream>>>((const double2*)x_dev, x_lp_dev, tb.n, nrhs);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status gs_lowp_unpack_multi(gs_ctx* c, int type, int dir, int inverse, int prec, int nrhs,
                               const void* x_lp_dev, void* x_dev) {
    if (!c) return GS_EINVAL;
    if (nrhs < 1 || nrhs > kMaxRhs) return set_err(c, GS_EINVAL, "nrhs %d not in 1..%d", nrhs, kMaxRhs);
    if (prec != GS_F32 && prec != GS_BF16) return set_err(c, GS_EINVAL, "precision %d", prec);
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    if (!x_dev || !x_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    LowpTables tb;
    if ((s = lowp_tables(c, p, prec, &tb)) != GS_OK) return s;
    const int g = grid_for(tb.n * nrhs, 256, c->num_sms * 8);
    if (prec == GS_BF16)
        k_multi_unpack<__nv_bfloat16><<<g, 256, 0, c->stream>>>(x_lp_dev, (double2*)x_dev, tb.n, nrhs);
    else
        k_multi_unpack<float><<<g, 256, 0, c->stream>>>(x_lp_dev, (double2*)x_dev, tb.n, nrhs);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status wilson_apply_lowp_multi(gs_ctx* c, int type, int dir, int inverse, int prec, int nrhs,
                                  const void* x_lp_dev, void* y_lp_dev) {
    if (!c) return GS_EINVAL;
    if (nrhs < 1 || nrhs > kMaxRhs) return set_err(c, GS_EINVAL, "nrhs %d not in 1..%d", nrhs, kMaxRhs);
    if (prec != GS_F32 && prec != GS_BF16) return set_err(c, GS_EINVAL, "precision %d", prec);
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    if (!x_lp_dev || !y_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    LowpTables tb;
    if ((s = lowp_tables(c, p, prec, &tb)) != GS_OK) return s;
    MArgs a;
    a.in = x_lp_dev;
    a.out = y_lp_dev;
    a.links = tb.links;
    a.nbr = tb.nbr;
    a.n = tb.n;
    a.N = nrhs;
    a.diag = (float)(c->m0 + 4.0);
    const int B = 128;
    const int64_t g = (tb.n * nrhs + B - 1) / B;
    int slot = -1;
    if (c->prof.on && (s = prof_begin(c, &slot)) != GS_OK) return s;
    if (prec == GS_BF16) k_dslash_multi<__nv_bfloat16><<<(int)g, B, 0, c->stream>>>(a);
    else k_dslash_multi<float><<<(int)g, B, 0, c->stream>>>(a);
    c->launches++;
    c->stencil_sites += tb.n * nrhs;
    GS_CHECK_LAUNCH(c);
    if (slot >= 0) {
        // per launch: spinor in + out for every source, the 12-real links once
        const double sb = (double)lp_spinor_bytes(prec), lb = (prec == GS_BF16) ? 24.0 : 48.0;
        c->prof.ran_host[slot] = 1;
        GS_CUDA(c, cudaMemcpy(c->prof.ran_dev + slot, c->prof.ran_host + slot, sizeof(int),
                              cudaMemcpyHostToDevice));
        return prof_end_work(c, slot, prec, tb.n * nrhs, tb.hops * nrhs,
                             (168.0 * tb.hops + 48.0 * tb.n) * nrhs,
                             2.0 * sb * tb.n * nrhs + lb * 0.5 * tb.hops);
    }
    return GS_OK;
}

gs_status schur_solve_multi(gs_ctx* c, int type, int dir, int inverse, int nrhs, const void* f_dev,
                            void* x_dev, const gs_solve_opts* opts, gs_solve_stats* stats) {
    if (!c) return GS_EINVAL;
    gs_solve_opts o;
    gs_default_opts(&o);
    if (opts) o = *opts;
    gs_solve_stats st;
    memset(&st, 0, sizeof st);
    const long long l0 = c->launches, s0 = c->stencil_sites;
    auto finish = [&](gs_status s) {
        st.status = s;
        st.kernel_launches = c->launches - l0;
        st.stencil_sites = c->stencil_sites - s0;
        if (stats) *stats = st;
        return s;
    };
    if (nrhs < 1 || nrhs > kMaxRhs)
        return finish(set_err(c, GS_EINVAL, "nrhs %d not in 1..%d", nrhs, kMaxRhs));
    if (!f_dev || !x_dev) return finish(set_err(c, GS_EINVAL, "null vector"));
    if (type != GS_TYPE_I && type != GS_TYPE_II)
        return finish(set_err(c, GS_EINVAL, "unknown permutation type %d", type));
    if (o.inner_prec != GS_F32 && o.inner_prec != GS_BF16)
        return finish(set_err(c, GS_EINVAL, "schur_solve_multi runs low-precision inner solves: "
                                            "inner_prec must be GS_F32 or GS_BF16"));
    if (!(o.tol > 0.0) || !(o.inner_tol > 0.0) || o.restart < 1 || o.restart > kMaxRestart ||
        o.inner_max_iter < 1 || !(o.lowp_tol >= 0.0) || o.lowp_tol >= 1.0 ||
        (o.inner_relax && (!(o.relax_cap > 0.0) || o.relax_cap >= 1.0)))
        return finish(set_err(c, GS_EINVAL, "invalid solver options"));
    if (!c->have_gauge) return finish(set_err(c, GS_ENOGAUGE, "no gauge field set"));
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return finish(s);
    // batch shape: the sources share launches only where one source leaves the
    // GPU latency bound (measured on GB300: 12 sources on 8^4 3.3x faster
    // together, on 16^4 0.9x); otherwise one at a time, single-source solver
    const bool together = c->opt_multi_batch == 1 ||
                          (c->opt_multi_batch == 0 && (c->V - p->nb) <= kBatchMaxRestSites);
    if (!together && nrhs > 1) {
        const int64_t V = c->V;
        gs_status worst = GS_OK;
        for (int j = 0; j < nrhs; ++j) {
            gs_solve_stats sj;
            memset(&sj, 0, sizeof sj);
            const gs_status e = ::schur_solve(c, type, dir, inverse, (const double2*)f_dev + (size_t)j * V * kSiteC,
                                              (double2*)x_dev + (size_t)j * V * kSiteC, &o, &sj);
            if (e != GS_OK && e != GS_MAXITER) return finish(e);
            if (e == GS_MAXITER) worst = e;
            st.outer_iters = st.outer_iters > sj.outer_iters ? st.outer_iters : sj.outer_iters;
            st.inner_solves += sj.inner_solves;
            st.inner_iters += sj.inner_iters;
            st.inner_max_seen = st.inner_max_seen > sj.inner_max_seen ? st.inner_max_seen : sj.inner_max_seen;
            st.outer_residual = st.outer_residual > sj.outer_residual ? st.outer_residual : sj.outer_residual;
            st.true_residual = st.true_residual > sj.true_residual ? st.true_residual : sj.true_residual;
            st.inner_residual = st.inner_residual > sj.inner_residual ? st.inner_residual : sj.inner_residual;
            st.lowp_cycles += sj.lowp_cycles;
            st.lowp_fallbacks += sj.lowp_fallbacks;
        }
        return finish(worst);
    }
    MultiWork* m = multi_of(c);
    if ((s = multi_fixed(c, m)) != GS_OK) return finish(s);
    const int N = nrhs;
    const int64_t V = c->V, nb = p->nb, nr = V - nb;
    const size_t fb = (size_t)N * V * kSiteC * sizeof(double2);
    if ((s = grow(c, (void**)&m->F, &m->capF, fb)) != GS_OK ||
        (s = grow(c, (void**)&m->Z, &m->capZ, fb)) != GS_OK ||
        (s = grow(c, (void**)&m->X, &m->capX, fb)) != GS_OK ||
        (s = grow(c, (void**)&m->wb, &m->capWB, (size_t)N * nb * kSiteC * sizeof(double2))) != GS_OK)
        return finish(s);
    double2 *F = m->F, *Z = m->Z, *X = m->X, *WB = m->wb;
    const double2* f = (const double2*)f_dev;
    double2* x = (double2*)x_dev;
    gs_status inner_flag = GS_OK;
    auto run = [&]() -> gs_status {
        // label order; the rest parts of all sources side by side: [N][nr][12]
        double2* Fr = Z;  // f_r of every source, contiguous per source
        for (int j = 0; j < N; ++j) {
            gs_status e = launch_gather(c, p->perm, f + (size_t)j * V * kSiteC, F + (size_t)j * V * kSiteC, V);
            if (e != GS_OK) return e;
            GS_CUDA(c, cudaMemcpyAsync(Fr + (size_t)j * nr * kSiteC, F + ((size_t)j * V + nb) * kSiteC,
                                       (size_t)nr * kSiteC * sizeof(double2), cudaMemcpyDeviceToDevice,
                                       c->stream));
        }
        double2* Zr = X;  // D_rr^-1 f_r, [N][nr][12]
        gs_status e = inner_solve_multi(c, p, N, Fr, Zr, o, st);
        if (e == GS_MAXITER) inner_flag = e;
        else if (e != GS_OK) return e;
        StencilArgs a;
        memset(&a, 0, sizeof a);
        a.diag = c->m0 + 4.0;
        a.plan = p;
        a.nbr = p->nbr;
        a.links = p->links;
        for (int j = 0; j < N; ++j) {  // w_j = f_b - D_br z_j
            a.out = WB + (size_t)j * nb * kSiteC;
            a.o0 = 0;
            a.n_out = nb;
            a.inA = Zr + (size_t)j * nr * kSiteC;
            a.a0 = nb;
            a.a1 = V;
            a.b1 = V;
            a.negate = 1;
            a.addend = F + (size_t)j * V * kSiteC;
            if ((e = launch_stencil_f64(c, a)) != GS_OK) return e;
        }
        // x_b of every source into m->xb-like contiguous storage: reuse Z (free now)
        double2* XB = Z;
        e = outer_gmres_multi(c, p, N, WB, XB, o, st);
        if (e == GS_MAXITER) inner_flag = e;
        else if (e != GS_OK) return e;
        // back-substitution: rhs_j = f_r - D_rb x_b  ([N][nr][12] in X), x_r = D_rr^-1 rhs
        double2* R = X;
        for (int j = 0; j < N; ++j) {
            a.out = R + (size_t)j * nr * kSiteC;
            a.o0 = nb;
            a.n_out = nr;
            a.inA = XB + (size_t)j * nb * kSiteC;
            a.a0 = 0;
            a.a1 = nb;
            a.b1 = nb;
            a.negate = 1;
            a.addend = F + ((size_t)j * V + nb) * kSiteC;
            if ((e = launch_stencil_f64(c, a)) != GS_OK) return e;
        }
        // solution pieces into F (label order, per source): x_b then x_r
        for (int j = 0; j < N; ++j)
            GS_CUDA(c, cudaMemcpyAsync(F + (size_t)j * V * kSiteC, XB + (size_t)j * nb * kSiteC,
                                       (size_t)nb * kSiteC * sizeof(double2), cudaMemcpyDeviceToDevice,
                                       c->stream));
        double2* XR = Z;  // XB was copied out; Z is free again
        e = inner_solve_multi(c, p, N, R, XR, o, st);
        if (e == GS_MAXITER) inner_flag = e;
        else if (e != GS_OK) return e;
        for (int j = 0; j < N; ++j) {
            GS_CUDA(c, cudaMemcpyAsync(F + ((size_t)j * V + nb) * kSiteC, XR + (size_t)j * nr * kSiteC,
                                       (size_t)nr * kSiteC * sizeof(double2), cudaMemcpyDeviceToDevice,
                                       c->stream));
            if ((e = launch_scatter(c, p->perm, F + (size_t)j * V * kSiteC, x + (size_t)j * V * kSiteC, V)) !=
                GS_OK)
                return e;
        }
        // FP64 true residuals ||f_j - D x_j|| / ||f_j||
        const Plan* id = c->plans[0];
        StencilArgs rd;
        memset(&rd, 0, sizeof rd);
        rd.o0 = 0;
        rd.n_out = V;
        rd.a0 = 0;
        rd.a1 = V;
        rd.b1 = V;
        rd.diag = c->m0 + 4.0;
        rd.negate = 1;
        rd.plan = id;
        rd.nbr = id->nbr;
        rd.links = id->links;
        double worst = 0.0;
        for (int j = 0; j < N; ++j) {
            rd.out = F;
            rd.inA = x + (size_t)j * V * kSiteC;
            rd.addend = f + (size_t)j * V * kSiteC;
            if ((e = launch_stencil_f64(c, rd)) != GS_OK) return e;
            if ((e = launch_norm2(c, m->red, F, V * kSiteC, m->rr64)) != GS_OK) return e;
            if ((e = launch_norm2(c, m->red, f + (size_t)j * V * kSiteC, V * kSiteC, m->rr64 + 1)) != GS_OK)
                return e;
            GS_CUDA(c, cudaMemcpyAsync(m->rr64_host, m->rr64, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                       c->stream));
            GS_CUDA(c, cudaStreamSynchronize(c->stream));
            const double r = m->rr64_host[1] > 0.0 ? sqrt(m->rr64_host[0] / m->rr64_host[1]) : 0.0;
            worst = std::max(worst, r);
        }
        st.true_residual = worst;
        return inner_flag;
    };
    s = run();
    cudaStreamSynchronize(c->stream);
    return finish(s);
}

}  // extern "C"
