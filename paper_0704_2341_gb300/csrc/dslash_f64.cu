// FP64 Wilson-Dirac stencil on label-ordered vectors, restricted to label
// ranges: the blocks D_bb, D_br, D_rb, D_rr of the permuted operator P D P^T
// (Section 1 of the paper: the 2x2 partition) and the full D (identity plan).
//
//   (D psi)(x) = (m0 + 4) psi(x) - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
//                                   + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
//
// gamma matrices in the DeGrand-Rossi chiral basis: g_mu = [[0, X], [X^dag, 0]]
// with X_0 = [[0,i],[i,0]], X_1 = [[0,-1],[1,0]], X_2 = diag(i,-i), X_3 = 1.
// Then (1 -+ g_mu) psi = [h; -+ X^dag h] with h = psi_up -+ X psi_lo, so each hop
// multiplies only the two-spinor h by the link (spin projection) and the
// lower half of the result is X^dag applied to (g_back - g_fwd).
//
// GB300 design: FP64 runs at ~1/60 of the FP32 rate on this part, so the
// kernel is bound by the FP64 pipe, not by HBM.  To keep every SM sub-partition
// busy even on 8^4 lattices, a block of 4 warps covers 32 sites and warp w
// handles direction mu = w (forward and backward hop) for all 32 sites: the
// direction is warp-uniform, so the spin projection specialises without
// divergence.  The four partial 24-double results meet in shared memory
// (SoA, bank-conflict free) and warp w then finishes spin component w of the
// 32 sites.  Links are stored pre-multiplied by -1/2 (exact in binary).
#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr int kSitesPerBlock = 32;
constexpr int kThreads = 128;

struct Half {  // two spin components x three colours
    double2 v[2][3];
};

// h = psi_up - X_mu psi_lo (FWD) or psi_up + X_mu psi_lo (!FWD)
template <int MU, bool FWD>
__device__ __forceinline__ void project(const double2 (&p)[12], Half& h) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 s0 = p[0 + c], s1 = p[3 + c], s2 = p[6 + c], s3 = p[9 + c];
        if (MU == 0) {  // X psi_lo = (i s3, i s2)
            h.v[0][c] = FWD ? csubi(s0, s3) : caddi(s0, s3);
            h.v[1][c] = FWD ? csubi(s1, s2) : caddi(s1, s2);
        } else if (MU == 1) {  // X psi_lo = (-s3, s2)
            h.v[0][c] = FWD ? cadd(s0, s3) : csub(s0, s3);
            h.v[1][c] = FWD ? csub(s1, s2) : cadd(s1, s2);
        } else if (MU == 2) {  // X psi_lo = (i s2, -i s3)
            h.v[0][c] = FWD ? csubi(s0, s2) : caddi(s0, s2);
            h.v[1][c] = FWD ? caddi(s1, s3) : csubi(s1, s3);
        } else {  // X psi_lo = (s2, s3)
            h.v[0][c] = FWD ? csub(s0, s2) : cadd(s0, s2);
            h.v[1][c] = FWD ? csub(s1, s3) : cadd(s1, s3);
        }
    }
}

// lower = X_mu^dag d
template <int MU>
__device__ __forceinline__ void xdag(const double2 (&d)[2][3], double2 (&lo)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) {  // X^dag = [[0,-i],[-i,0]]
            lo[0][c] = cmulmi(d[1][c]);
            lo[1][c] = cmulmi(d[0][c]);
        } else if (MU == 1) {  // X^dag = [[0,1],[-1,0]]
            lo[0][c] = d[1][c];
            lo[1][c] = cneg(d[0][c]);
        } else if (MU == 2) {  // X^dag = diag(-i, i)
            lo[0][c] = cmulmi(d[0][c]);
            lo[1][c] = cmuli(d[1][c]);
        } else {
            lo[0][c] = d[0][c];
            lo[1][c] = d[1][c];
        }
    }
}

__device__ __forceinline__ void load_spinor(const double2* __restrict__ src, double2 (&p)[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = __ldg(src + k);
}

__device__ __forceinline__ void load_link(const double2* __restrict__ src, double2 (&u)[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldg(src + k);
}

// The 24 doubles of one direction's contribution for one site.
template <int MU>
__device__ __forceinline__ void hop_mu(const StencilArgs& a, int64_t j, bool valid,
                                       double2 (&up)[2][3], double2 (&lo)[2][3]) {
    double2 gf[2][3], acc[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) gf[s][c] = acc[s][c] = make_double2(0.0, 0.0);
    if (valid) {
        const int2 nb = __ldg(a.nbr + j * 4 + MU);
        const int64_t lf = nb.x, lb = nb.y;
        const double2* srcf = nullptr;
        const double2* srcb = nullptr;
        if (lf >= a.a0 && lf < a.a1) srcf = a.inA + (lf - a.a0) * kSiteC;
        else if (lf >= a.a1 && lf < a.b1) srcf = a.inB + (lf - a.a1) * kSiteC;
        if (lb >= a.a0 && lb < a.a1) srcb = a.inA + (lb - a.a0) * kSiteC;
        else if (lb >= a.a1 && lb < a.b1) srcb = a.inB + (lb - a.a1) * kSiteC;
        if (srcf) {
            double2 p[12], u[9];
            Half h;
            load_spinor(srcf, p);
            project<MU, true>(p, h);
            load_link(a.links + (j * 4 + MU) * kLinkC, u);
            // g_f = U h  (row a of U times the colour vector)
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    double2 t = cmul(u[3 * r + 0], h.v[s][0]);
                    cfma(t, u[3 * r + 1], h.v[s][1]);
                    cfma(t, u[3 * r + 2], h.v[s][2]);
                    gf[s][r] = t;
                    acc[s][r] = t;
                }
        }
        if (srcb) {
            double2 p[12], u[9];
            Half h;
            load_spinor(srcb, p);
            project<MU, false>(p, h);
            load_link(a.links + (lb * 4 + MU) * kLinkC, u);
            // acc += U^dag h  (row a of U^dag = conj of column a of U)
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    double2 t = acc[s][r];
                    ccfma(t, u[0 + r], h.v[s][0]);
                    ccfma(t, u[3 + r], h.v[s][1]);
                    ccfma(t, u[6 + r], h.v[s][2]);
                    acc[s][r] = t;
                }
        }
    }
    // up = g_f + g_b = acc ; d = g_b - g_f = acc - 2 g_f
    double2 d[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            up[s][c] = acc[s][c];
            d[s][c] = make_double2(fma(-2.0, gf[s][c].x, acc[s][c].x),
                                   fma(-2.0, gf[s][c].y, acc[s][c].y));
        }
    xdag<MU>(d, lo);
}

template <int EPI>
__global__ void __launch_bounds__(kThreads) k_dslash_f64(StencilArgs a) {
    const bool skip = a.st != nullptr && a.st->done;
    if (a.ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.ran = skip ? 0 : 1;
    if (skip) return;
    __shared__ double red[4][24][kSitesPerBlock];
    __shared__ double bred[4][kMaxRedVals];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    double e0 = 0.0, e1 = 0.0, e2 = 0.0;  // epilogue partial sums

    for (int64_t base = (int64_t)blockIdx.x * kSitesPerBlock; base < a.n_out;
         base += (int64_t)gridDim.x * kSitesPerBlock) {
        // phase 1: warp `warp` computes direction mu = warp for 32 sites
        {
            const int64_t k = base + lane;
            const bool valid = k < a.n_out;
            const int64_t j = a.o0 + k;
            double2 up[2][3], lo[2][3];
            switch (warp) {
                case 0: hop_mu<0>(a, j, valid, up, lo); break;
                case 1: hop_mu<1>(a, j, valid, up, lo); break;
                case 2: hop_mu<2>(a, j, valid, up, lo); break;
                default: hop_mu<3>(a, j, valid, up, lo); break;
            }
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    red[warp][(s * 3 + c) * 2 + 0][lane] = up[s][c].x;
                    red[warp][(s * 3 + c) * 2 + 1][lane] = up[s][c].y;
                    red[warp][(6 + s * 3 + c) * 2 + 0][lane] = lo[s][c].x;
                    red[warp][(6 + s * 3 + c) * 2 + 1][lane] = lo[s][c].y;
                }
        }
        __syncthreads();
        // phase 2: warp w finishes spin component w of the 32 sites
        {
            const int spin = warp;
            const int64_t k = base + lane;
            if (k < a.n_out) {
                const int64_t j = a.o0 + k;
                const double2* self = nullptr;
                if (j >= a.a0 && j < a.a1) self = a.inA + (j - a.a0) * kSiteC;
                else if (j >= a.a1 && j < a.b1) self = a.inB + (j - a.a1) * kSiteC;
                double2* dst = a.out + k * kSiteC + spin * 3;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int q = (spin * 3 + c) * 2;
                    double re = red[0][q][lane] + red[1][q][lane] + red[2][q][lane] + red[3][q][lane];
                    double im = red[0][q + 1][lane] + red[1][q + 1][lane] + red[2][q + 1][lane] +
                                red[3][q + 1][lane];
                    if (self) {
                        const double2 sv = __ldg(self + spin * 3 + c);
                        re = fma(a.diag, sv.x, re);
                        im = fma(a.diag, sv.y, im);
                    }
                    if (a.negate) {
                        re = -re;
                        im = -im;
                    }
                    if (a.addend) {
                        const double2 av = a.addend[k * kSiteC + spin * 3 + c];
                        re += av.x;
                        im += av.y;
                    }
                    dst[c] = make_double2(re, im);
                    if (EPI == EPI_DOT_RHAT_V) {  // <rhat, v> = sum conj(rhat) v
                        const double2 rv = a.epi_vec[k * kSiteC + spin * 3 + c];
                        e0 = fma(rv.x, re, fma(rv.y, im, e0));
                        e1 = fma(rv.x, im, fma(-rv.y, re, e1));
                    } else if (EPI == EPI_DOT_TS) {  // <t, s>, <t, t>
                        const double2 sv = a.epi_vec[k * kSiteC + spin * 3 + c];
                        e0 = fma(re, sv.x, fma(im, sv.y, e0));
                        e1 = fma(re, sv.y, fma(-im, sv.x, e1));
                        e2 = fma(re, re, fma(im, im, e2));
                    }
                }
            }
        }
        __syncthreads();
    }

    if constexpr (EPI == EPI_NONE) {
        return;
    } else {

    // block reduction of the epilogue sums, then the last block finishes
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        e0 += __shfl_xor_sync(0xffffffffu, e0, off);
        e1 += __shfl_xor_sync(0xffffffffu, e1, off);
        e2 += __shfl_xor_sync(0xffffffffu, e2, off);
    }
    if (lane == 0) {
        bred[warp][0] = e0;
        bred[warp][1] = e1;
        bred[warp][2] = e2;
    }
    __syncthreads();
    __shared__ bool am_last;
    if (threadIdx.x == 0) {
        double* part = a.red.partial + (int64_t)blockIdx.x * kMaxRedVals;
        part[0] = (bred[0][0] + bred[1][0]) + (bred[2][0] + bred[3][0]);
        part[1] = (bred[0][1] + bred[1][1]) + (bred[2][1] + bred[3][1]);
        part[2] = (bred[0][2] + bred[1][2]) + (bred[2][2] + bred[3][2]);
        __threadfence();
        const unsigned prev = atomicAdd(a.red.counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // deterministic: fixed per-thread strides then a fixed tree
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
        const volatile double* part = a.red.partial + (int64_t)b * kMaxRedVals;
        s0 += part[0];
        s1 += part[1];
        s2 += part[2];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if (lane == 0) {
        bred[warp][0] = s0;
        bred[warp][1] = s1;
        bred[warp][2] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s0 = (bred[0][0] + bred[1][0]) + (bred[2][0] + bred[3][0]);
        s1 = (bred[0][1] + bred[1][1]) + (bred[2][1] + bred[3][1]);
        s2 = (bred[0][2] + bred[1][2]) + (bred[2][2] + bred[3][2]);
        BicgState* st = a.st;
        if (EPI == EPI_DOT_RHAT_V) {
            const double2 den = make_double2(s0, s1);
            if (den.x == 0.0 && den.y == 0.0) {
                st->status = GS_BREAKDOWN;
                st->done = 1;
            } else {
                st->alpha = cdiv(st->rho, den);
                if (!isfinite(st->alpha.x) || !isfinite(st->alpha.y)) {
                    st->status = GS_NONFINITE;
                    st->done = 1;
                }
            }
        } else {
            // omega = <t,s>/<t,t>; t == 0 means s == 0 (D_rr is regular): omega = 0
            st->omega = (s2 > 0.0) ? make_double2(s0 / s2, s1 / s2) : make_double2(0.0, 0.0);
            if (!isfinite(st->omega.x) || !isfinite(st->omega.y)) {
                st->status = GS_NONFINITE;
                st->done = 1;
            }
        }
        if (st->done) publish(st);
        *a.red.counter = 0u;
    }
    }
}

}  // namespace

gs_status launch_stencil_f64(gs_ctx* c, const StencilArgs& args) {
    if (args.n_out <= 0) return GS_OK;
    StencilArgs a = args;
    int slot = -1;
    if (c->prof.on) {
        gs_status s = prof_begin(c, &slot);
        if (s != GS_OK) return s;
        a.ran = c->prof.ran_dev + slot;
    } else {
        a.ran = nullptr;
    }
    const int64_t blocks_needed = (a.n_out + kSitesPerBlock - 1) / kSitesPerBlock;
    int max_blocks = (a.epi == EPI_NONE) ? (1 << 30) : kMaxRedBlocks;
    const int g = (int)(blocks_needed < max_blocks ? blocks_needed : max_blocks);
    switch (a.epi) {
        case EPI_NONE: k_dslash_f64<EPI_NONE><<<g, kThreads, 0, c->stream>>>(a); break;
        case EPI_DOT_RHAT_V: k_dslash_f64<EPI_DOT_RHAT_V><<<g, kThreads, 0, c->stream>>>(a); break;
        default: k_dslash_f64<EPI_DOT_TS><<<g, kThreads, 0, c->stream>>>(a); break;
    }
    c->launches++;
    c->stencil_sites += a.n_out;
    GS_CHECK_LAUNCH(c);
    if (slot >= 0) return prof_end(c, slot, a.plan, a);
    return GS_OK;
}

// The same kernel launched on a caller's stream without a context (no
// profiling, no epilogue): used by the entry point that allocates nothing.
gs_status launch_stencil_f64_on(const StencilArgs& args, cudaStream_t stream) {
    if (args.n_out <= 0) return GS_OK;
    StencilArgs a = args;
    a.ran = nullptr;
    a.epi = EPI_NONE;
    a.st = nullptr;
    const int64_t g = (a.n_out + kSitesPerBlock - 1) / kSitesPerBlock;
    k_dslash_f64<EPI_NONE><<<(int)g, kThreads, 0, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ECUDA;
}

}  // namespace gs
