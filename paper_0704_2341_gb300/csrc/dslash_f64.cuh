// Device code of the FP64 Wilson stencil, shared by the stand-alone stencil
// kernel (dslash_f64.cu) and the persistent solver kernels (persistent.cu).
#pragma once

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

// CG: read through L2 only (coherent with writes of other blocks of the same
// kernel, as the persistent solvers need); otherwise the read-only cache path.
template <bool CG>
__device__ __forceinline__ void load_spinor(const double2* __restrict__ src, double2 (&p)[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = CG ? __ldcg(src + k) : __ldg(src + k);
}

__device__ __forceinline__ void load_link(const double2* __restrict__ src, double2 (&u)[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldg(src + k);
}

// The 24 doubles of one direction's contribution for one site.
template <int MU, bool CG>
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
            load_spinor<CG>(srcf, p);
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
            load_spinor<CG>(srcb, p);
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


// One tile of ts <= 32 output sites (lane l < ts handles site base + l):
// phase 1 (warp w = direction w, both hops, to shared memory) and phase 2
// (warp w sums spin component w, adds the diagonal term, negation and addend,
// stores, and accumulates the epilogue dots into e).
//   EPI_DOT_RHAT_V: e0 + i e1 = <rhat, out>;  EPI_DOT_TS: e0 + i e1 = <out, s>,
//   e2 = <out, out>;  EPI_DOT_TSR: as EPI_DOT_TS and e3 + i e4 = <rhat, out>.
template <int EPI, bool CG = false>
__device__ __forceinline__ void f64_tile(const StencilArgs& a, int64_t base, int ts,
                                         double (&red)[4][24][kSitesPerBlock], double (&e)[5]) {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
        // phase 1: warp `warp` computes direction mu = warp for the tile's sites
    {
        const int64_t k = base + lane;
        const bool valid = lane < ts && k < a.n_out;
        const int64_t j = a.o0 + k;
        double2 up[2][3], lo[2][3];
        switch (warp) {
            case 0: hop_mu<0, CG>(a, j, valid, up, lo); break;
            case 1: hop_mu<1, CG>(a, j, valid, up, lo); break;
            case 2: hop_mu<2, CG>(a, j, valid, up, lo); break;
            default: hop_mu<3, CG>(a, j, valid, up, lo); break;
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
    // phase 2: warp w finishes spin component w of the tile's sites
    {
        const int spin = warp;
        const int64_t k = base + lane;
        if (lane < ts && k < a.n_out) {
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
                    const double2 sv = CG ? __ldcg(self + spin * 3 + c) : __ldg(self + spin * 3 + c);
                    re = fma(a.diag, sv.x, re);
                    im = fma(a.diag, sv.y, im);
                }
                if (a.negate) {
                    re = -re;
                    im = -im;
                }
                if (a.addend) {
                    const double2 av = CG ? __ldcg(a.addend + k * kSiteC + spin * 3 + c) : a.addend[k * kSiteC + spin * 3 + c];
                    re += av.x;
                    im += av.y;
                }
                dst[c] = make_double2(re, im);
                if (EPI == EPI_DOT_RHAT_V) {  // <rhat, v> = sum conj(rhat) v
                    const double2 rv = CG ? __ldcg(a.epi_vec + k * kSiteC + spin * 3 + c) : a.epi_vec[k * kSiteC + spin * 3 + c];
                    e[0] = fma(rv.x, re, fma(rv.y, im, e[0]));
                    e[1] = fma(rv.x, im, fma(-rv.y, re, e[1]));
                } else if (EPI == EPI_DOT_TS || EPI == EPI_DOT_TSR) {  // <t, s>, <t, t>
                    const double2 sv = CG ? __ldcg(a.epi_vec + k * kSiteC + spin * 3 + c) : a.epi_vec[k * kSiteC + spin * 3 + c];
                    e[0] = fma(re, sv.x, fma(im, sv.y, e[0]));
                    e[1] = fma(re, sv.y, fma(-im, sv.x, e[1]));
                    e[2] = fma(re, re, fma(im, im, e[2]));
                    if (EPI == EPI_DOT_TSR) {  // <rhat, t>
                        const double2 rv = CG ? __ldcg(a.epi_vec2 + k * kSiteC + spin * 3 + c) : a.epi_vec2[k * kSiteC + spin * 3 + c];
                        e[3] = fma(rv.x, re, fma(rv.y, im, e[3]));
                        e[4] = fma(rv.x, im, fma(-rv.y, re, e[4]));
                    }
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace
}  // namespace gs
