// BLAS-1 and fused Krylov-update kernels (FP64, complex interleaved).
//
// Reductions are deterministic: every block writes its partial sums, and the
// last block to finish (an atomic ticket after a fence; no waiting) adds the
// partials in a fixed order and finishes the scalar algebra on the device.
// Solver scalars therefore never leave the GPU inside an iteration; the host
// only polls the `done` flag every few iterations.
//
// BiCGStab (H. A. van der Vorst 1992) is split into five launches per
// iteration:  K1 v = A p (+ <rhat,v> -> alpha, in the stencil),
//             K2 s = r - alpha v, x += alpha p, ||s||^2 (early exit),
//             K3 t = A s (+ <t,s>, <t,t> -> omega, in the stencil),
//             K4 x += omega s, r = s - omega t, <rhat,r>, ||r||^2 -> beta, test,
//             K5 p = r + beta (p - omega v).
#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr int kBlas = 256;
constexpr int kDotChunk = 8;   // vectors per block of the multi-dot

// Block-reduce NV doubles; the last block gets the grand totals in thread 0.
// Returns true (block-uniform) in the last block only.
template <int NV>
__device__ bool reduce_last(double (&v)[NV], RedScratch red, double (&tot)[NV]) {
    __shared__ double sm[kBlas / 32][NV];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) sm[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double* part = red.partial + (int64_t)blockIdx.x * kMaxRedVals;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = 0.0;
            for (int w = 0; w < nw; ++w) x += sm[w][q];
            part[q] = x;
        }
        __threadfence();
        const unsigned prev = atomicAdd(red.counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile double* part = red.partial + (int64_t)b * kMaxRedVals;
#pragma unroll
        for (int q = 0; q < NV; ++q) s[q] += part[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = s[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) sm[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = 0.0;
            for (int w = 0; w < nw; ++w) x += sm[w][q];
            tot[q] = x;
        }
        *red.counter = 0u;
    }
    return true;
}

// ---------------------------------------------------------------------------
// BiCGStab kernels (n = number of complex entries)
// ---------------------------------------------------------------------------

// x = 0, r = rhat = p = b; rho = ||b||^2; stop at once if b == 0.
__global__ void k_bicg_init(const double2* __restrict__ b, double2* __restrict__ x,
                            double2* __restrict__ r, double2* __restrict__ rhat,
                            double2* __restrict__ p, int64_t n, double tol, BicgState* st,
                            RedScratch red) {
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 bi = b[i];
        x[i] = make_double2(0.0, 0.0);
        r[i] = bi;
        rhat[i] = bi;
        p[i] = bi;
        v[0] = fma(bi.x, bi.x, fma(bi.y, bi.y, v[0]));
    }
    double tot[1];
    if (reduce_last<1>(v, red, tot) && threadIdx.x == 0) {
        st->bb = tot[0];
        st->rr = tot[0];
        st->rho = make_double2(tot[0], 0.0);
        st->alpha = st->omega = st->beta = make_double2(0.0, 0.0);
        st->tol2 = tol * tol * tot[0];
        st->iter = 0;
        st->status = isfinite(tot[0]) ? GS_OK : GS_NONFINITE;
        st->done = (tot[0] == 0.0 || !isfinite(tot[0])) ? 1 : 0;
        publish(st);
    }
}

// s = r - alpha v ; x += alpha p ; ||s||^2 (early convergence on s)
__global__ void k_bicg_s(const double2* __restrict__ r, const double2* __restrict__ v,
                         const double2* __restrict__ p, double2* __restrict__ s,
                         double2* __restrict__ x, int64_t n, BicgState* st, RedScratch red) {
    if (st->done) return;
    const double2 al = st->alpha;
    double acc[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 vi = v[i], ri = r[i], pi = p[i];
        double2 si;
        si.x = ri.x - (al.x * vi.x - al.y * vi.y);
        si.y = ri.y - (al.x * vi.y + al.y * vi.x);
        s[i] = si;
        double2 xi = x[i];
        xi.x = fma(al.x, pi.x, fma(-al.y, pi.y, xi.x));
        xi.y = fma(al.x, pi.y, fma(al.y, pi.x, xi.y));
        x[i] = xi;
        acc[0] = fma(si.x, si.x, fma(si.y, si.y, acc[0]));
    }
    double tot[1];
    if (reduce_last<1>(acc, red, tot) && threadIdx.x == 0) {
        if (!isfinite(tot[0])) {
            st->status = GS_NONFINITE;
            st->done = 1;
        } else if (tot[0] <= st->tol2) {
            st->rr = tot[0];
            st->iter += 1;
            st->done = 1;
        }
        if (st->done) publish(st);
    }
}

// x += omega s ; r = s - omega t ; rho' = <rhat, r>, ||r||^2 ; beta ; test.
__global__ void k_bicg_xr(const double2* __restrict__ s, const double2* __restrict__ t,
                          const double2* __restrict__ rhat, double2* __restrict__ x,
                          double2* __restrict__ r, int64_t n, BicgState* st, RedScratch red) {
    if (st->done) return;
    const double2 om = st->omega;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 si = s[i], ti = t[i], hi = rhat[i];
        double2 xi = x[i];
        xi.x = fma(om.x, si.x, fma(-om.y, si.y, xi.x));
        xi.y = fma(om.x, si.y, fma(om.y, si.x, xi.y));
        x[i] = xi;
        double2 ri;
        ri.x = si.x - (om.x * ti.x - om.y * ti.y);
        ri.y = si.y - (om.x * ti.y + om.y * ti.x);
        r[i] = ri;
        acc[0] = fma(hi.x, ri.x, fma(hi.y, ri.y, acc[0]));
        acc[1] = fma(hi.x, ri.y, fma(-hi.y, ri.x, acc[1]));
        acc[2] = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[2]));
    }
    double tot[3];
    if (reduce_last<3>(acc, red, tot) && threadIdx.x == 0) {
        const double2 rho_new = make_double2(tot[0], tot[1]);
        st->rr = tot[2];
        st->iter += 1;
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
            st->status = GS_NONFINITE;
            st->done = 1;
        } else if (tot[2] <= st->tol2) {
            st->done = 1;
        } else if ((om.x == 0.0 && om.y == 0.0) || (rho_new.x == 0.0 && rho_new.y == 0.0)) {
            st->status = GS_BREAKDOWN;
            st->done = 1;
        } else {
            st->beta = cmul(cdiv(rho_new, st->rho), cdiv(st->alpha, om));
            st->rho = rho_new;
        }
        publish(st);
    }
}

// p = r + beta (p - omega v)
__global__ void k_bicg_p(const double2* __restrict__ r, const double2* __restrict__ v,
                         double2* __restrict__ p, int64_t n, const BicgState* st) {
    if (st->done) return;
    const double2 be = st->beta, om = st->omega;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 vi = v[i], ri = r[i];
        double2 pi = p[i];
        double2 q;  // p - omega v
        q.x = pi.x - (om.x * vi.x - om.y * vi.y);
        q.y = pi.y - (om.x * vi.y + om.y * vi.x);
        pi.x = fma(be.x, q.x, fma(-be.y, q.y, ri.x));
        pi.y = fma(be.x, q.y, fma(be.y, q.x, ri.y));
        p[i] = pi;
    }
}

// ---------------------------------------------------------------------------
// generic BLAS-1
// ---------------------------------------------------------------------------

// out[k] (+)= <X_k, y> = sum conj(X_k) y, k < nvec.  grid = (gx, ceil(nvec / chunk)).
__global__ void k_multidot(const double2* __restrict__ X, int64_t ld, const double2* __restrict__ y,
                           int64_t n, int nvec, int chunk, double2* out, int accumulate, double* partial,
                           unsigned int* counter) {
    // block (bx, c): the dots of vectors chunk c .. chunk c + chunk - 1 (chunk
    // <= 8) with y over the block's strided range (y read once for them); the
    // last block adds the per-block partials of every vector in block order
    __shared__ double sm[kBlas / 32][2 * kDotChunk];
    __shared__ bool am_last;
    const int k0 = blockIdx.y * chunk;
    const int nk = nvec - k0 < chunk ? nvec - k0 : chunk;
    double a[2 * kDotChunk];
#pragma unroll
    for (int q = 0; q < 2 * kDotChunk; ++q) a[q] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 w = y[i];
#pragma unroll
        for (int q = 0; q < kDotChunk; ++q) {
            if (q < nk) {
                const double2 u = X[(int64_t)(k0 + q) * ld + i];
                a[2 * q] = fma(u.x, w.x, fma(u.y, w.y, a[2 * q]));
                a[2 * q + 1] = fma(u.x, w.y, fma(-u.y, w.x, a[2 * q + 1]));
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < 2 * kDotChunk; ++q) {
        if (q < 2 * nk) {  // block-uniform
            double v = a[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) sm[warp][q] = v;
        }
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
        const unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int kk = threadIdx.x; kk < nvec; kk += blockDim.x) {
        double s0 = 0.0, s1 = 0.0;
        const double* part = partial + (int64_t)kk * gridDim.x * 2;
        // L2 loads of the partials (all written before the counter reached
        // nblocks); independent, so they are in flight together
#pragma unroll 8
        for (unsigned b = 0; b < gridDim.x; ++b) {
            s0 += __ldcg(part + 2 * b);
            s1 += __ldcg(part + 2 * b + 1);
        }
        if (accumulate) {
            out[kk].x += s0;
            out[kk].y += s1;
        } else {
            out[kk] = make_double2(s0, s1);
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// y += sign * sum_k coef[k] X_k
__global__ void k_multiaxpy(const double2* __restrict__ X, int64_t ld, int nvec,
                            const double2* __restrict__ coef, double2* __restrict__ y, int64_t n,
                            double sign) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < nvec; ++k) {
            const double2 c = __ldg(coef + k);
            const double2 u = X[(int64_t)k * ld + i];
            cfma(acc, c, u);
        }
        double2 yi = y[i];
        yi.x = fma(sign, acc.x, yi.x);
        yi.y = fma(sign, acc.y, yi.y);
        y[i] = yi;
    }
}

__global__ void k_norm2(const double2* __restrict__ x, int64_t n, double* out, RedScratch red) {
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 u = x[i];
        v[0] = fma(u.x, u.x, fma(u.y, u.y, v[0]));
    }
    double tot[1];
    if (reduce_last<1>(v, red, tot) && threadIdx.x == 0) *out = tot[0];
}

__global__ void k_scale_copy(const double2* __restrict__ x, double2* __restrict__ y, int64_t n,
                             double a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 u = x[i];
        y[i] = make_double2(a * u.x, a * u.y);
    }
}

// y = a x + b y
__global__ void k_axpby(double2 a, const double2* __restrict__ x, double2 b, double2* __restrict__ y,
                        int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 u = x[i];
        double2 t = cmul(b, y[i]);
        cfma(t, a, u);
        y[i] = t;
    }
}

}  // namespace

static int red_grid(gs_ctx* c, int64_t n) {
    return grid_for(n, kBlas, c->num_sms * 4 < kMaxRedBlocks ? c->num_sms * 4 : kMaxRedBlocks);
}
static int plain_grid(gs_ctx* c, int64_t n) { return grid_for(n, kBlas, c->num_sms * 16); }

gs_status launch_bicg_init(gs_ctx* c, InnerWork& w, const double2* b, double2* x, int64_t n,
                           double tol) {
    k_bicg_init<<<red_grid(c, n), kBlas, 0, c->stream>>>(b, x, w.r, w.rhat, w.p, n, tol, w.st,
                                                         w.red);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_bicg_s_update(gs_ctx* c, InnerWork& w, double2* x, int64_t n) {
    k_bicg_s<<<red_grid(c, n), kBlas, 0, c->stream>>>(w.r, w.v, w.p, w.s, x, n, w.st, w.red);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_bicg_xr_update(gs_ctx* c, InnerWork& w, double2* x, int64_t n) {
    k_bicg_xr<<<red_grid(c, n), kBlas, 0, c->stream>>>(w.s, w.t, w.rhat, x, w.r, n, w.st, w.red);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_bicg_p_update(gs_ctx* c, InnerWork& w, int64_t n) {
    k_bicg_p<<<plain_grid(c, n), kBlas, 0, c->stream>>>(w.r, w.v, w.p, n, w.st);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_multidot(gs_ctx* c, RedScratch red, const double2* X, int64_t ld, int nvec,
                          const double2* y, int64_t n, double2* dev_out, int accumulate) {
    if (nvec <= 0) return GS_OK;
    // enough blocks in flight to stream long vectors at HBM bandwidth, within
    // the partial scratch (nvec x gx complex)
    // long vectors: eight vectors per block against one load of y; short
    // ones: one vector per block (more blocks, short reduction tails)
    const int chunk = n >= 65536 ? kDotChunk : 1;
    const int nchunks = (nvec + chunk - 1) / chunk;
    int64_t cap = (int64_t)c->num_sms * 8 / nchunks;
    if (cap < 64) cap = 64;
    if (cap > kRedScratchDoubles / (2 * nvec)) cap = kRedScratchDoubles / (2 * nvec);
    const int gx = grid_for(n, kBlas, (int)cap);
    dim3 g(gx, nchunks);
    k_multidot<<<g, kBlas, 0, c->stream>>>(X, ld, y, n, nvec, chunk, dev_out, accumulate, red.partial,
                                           red.counter);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_multiaxpy(gs_ctx* c, const double2* X, int64_t ld, int nvec, const double2* coef,
                           double2* y, int64_t n, int sign) {
    if (nvec <= 0) return GS_OK;
    k_multiaxpy<<<plain_grid(c, n), kBlas, 0, c->stream>>>(X, ld, nvec, coef, y, n,
                                                           sign > 0 ? 1.0 : -1.0);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_norm2(gs_ctx* c, RedScratch red, const double2* x, int64_t n, double* dev_out) {
    k_norm2<<<red_grid(c, n), kBlas, 0, c->stream>>>(x, n, dev_out, red);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_scale_copy(gs_ctx* c, const double2* x, double2* y, int64_t n, double a) {
    k_scale_copy<<<plain_grid(c, n), kBlas, 0, c->stream>>>(x, y, n, a);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_axpby(gs_ctx* c, double2 a, const double2* x, double2 b, double2* y, int64_t n) {
    k_axpby<<<plain_grid(c, n), kBlas, 0, c->stream>>>(a, x, b, y, n);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

}  // namespace gs
