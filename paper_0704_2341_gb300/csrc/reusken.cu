// The second-order Schur-complement approximation of Section 3:
//   S~_bb = D_bb - D_br M D_rb,  M = d^-1 + d~^-1 - d^-1 D_rr d~^-1,
// d the (site-block) diagonal of D_rr and d~ its block row sums,
//   d~_x = sum_{y in r} (D_rr)_{x,y}   (12 x 12, spin x colour, per rest site).
// For the Wilson operator d = (m0 + 4) 1, so with t = -D_rb x_b and
// w = d~^-1 t:  z = M t = w + (t - D_rr w) / (m0 + 4), and
// S~_bb x_b = (D [x_b; z])_b: three label-range stencil launches, one
// 12 x 12 block product per rest site and a combination.
//   d~_x = (m0 + 4) 1 + sum_mu [ (1 - gamma_mu) (x) L_mu(x)       (x + mu in r)
//                              + (1 + gamma_mu) (x) L_mu(x - mu)^dag (x - mu in r) ]
// with L = -1/2 U (the plan's links) and, in the chiral basis of the
// stencil, gamma_mu = [[0, X_mu], [X_mu^dag, 0]].  The inverses are built once
// per plan and gauge field (Gauss-Jordan with partial pivoting in FP64, one
// thread per rest site).
#include <math.h>

#include "block12.cuh"

namespace gs {
namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// entry (s, s') of gamma_mu (4 x 4, chiral basis of the stencil's projections)
__device__ double2 gamma_entry(int mu, int s, int sp) {
    // X_mu (2 x 2) as the upper-right block; X_mu^dag lower-left
    double2 X[2][2];
    const double2 z = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0), i1 = make_double2(0.0, 1.0);
    if (mu == 0) {
        X[0][0] = z; X[0][1] = i1; X[1][0] = i1; X[1][1] = z;
    } else if (mu == 1) {
        X[0][0] = z; X[0][1] = make_double2(-1.0, 0.0); X[1][0] = one; X[1][1] = z;
    } else if (mu == 2) {
        X[0][0] = i1; X[0][1] = z; X[1][0] = z; X[1][1] = make_double2(0.0, -1.0);
    } else {
        X[0][0] = one; X[0][1] = z; X[1][0] = z; X[1][1] = one;
    }
    if (s < 2 && sp >= 2) return X[s][sp - 2];
    if (s >= 2 && sp < 2) return zconj(X[sp][s - 2]);   // (X^dag)[s-2][sp] = conj(X[sp][s-2])
    return z;
}

// dtinv[k] = (d~ of rest label nb + k)^-1; status[0] set to 1 on a zero pivot
__global__ void k_reusken_dtinv(const int2* __restrict__ nbr, const double2* __restrict__ links, int64_t nb,
                                int64_t V, double diag, double2* __restrict__ dtinv, int* status) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < V - nb;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = nb + k;
        double2 A[12][12], B[12][12];
        for (int r = 0; r < 12; ++r)
            for (int q = 0; q < 12; ++q) A[r][q] = make_double2(r == q ? diag : 0.0, 0.0);
        for (int mu = 0; mu < 4; ++mu) {
            const int2 n2 = nbr[j * 4 + mu];
            for (int hop = 0; hop < 2; ++hop) {
                const int64_t l = hop == 0 ? n2.x : n2.y;
                if (l < nb) continue;  // neighbour not in r
                const double2* L = links + ((hop == 0 ? j : l) * 4 + mu) * 9;
                const double sg = hop == 0 ? -1.0 : 1.0;   // (1 - gamma) forward, (1 + gamma) backward
                for (int s = 0; s < 4; ++s)
                    for (int sp = 0; sp < 4; ++sp) {
                        double2 P = gamma_entry(mu, s, sp);
                        P = make_double2(sg * P.x + (s == sp ? 1.0 : 0.0), sg * P.y);
                        if (P.x == 0.0 && P.y == 0.0) continue;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) {
                                const double2 u = hop == 0 ? L[3 * a + b] : zconj(L[3 * b + a]);
                                const double2 v = zmul(P, u);
                                A[s * 3 + a][sp * 3 + b].x += v.x;
                                A[s * 3 + a][sp * 3 + b].y += v.y;
                            }
                    }
            }
        }
        const bool ok = invert12(A, B);
        if (!ok) atomicExch(status, 1);
        double2* out = dtinv + k * 144;
        for (int r = 0; r < 12; ++r)
            for (int q = 0; q < 12; ++q) out[r * 12 + q] = ok ? B[r][q] : make_double2(0.0, 0.0);
    }
}

// w[k] = dtinv[k] t[k] (12 x 12 block per rest site); one thread per (site, row)
__global__ void k_reusken_block(const double2* __restrict__ dtinv, const double2* __restrict__ t,
                                double2* __restrict__ w, int64_t nr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 12;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 12;
        const int r = (int)(i - k * 12);
        const double2* row = dtinv + k * 144 + r * 12;
        const double2* tk = t + k * 12;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const double2 a = row[q], b = tk[q];
            acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
            acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
        }
        w[i] = acc;
    }
}

// z = w + (t - u) / (m0 + 4)
__global__ void k_reusken_combine(const double2* __restrict__ w, const double2* __restrict__ t,
                                  const double2* __restrict__ u, double2* __restrict__ z, int64_t n,
                                  double inv_diag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = w[i], b = t[i], c = u[i];
        z[i] = make_double2(fma(b.x - c.x, inv_diag, a.x), fma(b.y - c.y, inv_diag, a.y));
    }
}

}  // namespace

static gs_status reusken_prepare(gs_ctx* c, Plan* p) {
    if (p->dtinv_ready) return GS_OK;
    const int64_t nr = c->V - p->nb;
    if (!p->dtinv) {
        if (cudaMalloc(&p->dtinv, (size_t)nr * 144 * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GS_ENOMEM, "allocating the Reusken block inverses failed");
        }
    }
    int* flag = nullptr;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, GS_ENOMEM, "allocating a status word failed");
    }
    GS_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    k_reusken_dtinv<<<grid_for(nr, 64, c->num_sms * 8), 64, 0, c->stream>>>(p->nbr, p->links, p->nb, c->V,
                                                                            c->m0 + 4.0, p->dtinv, flag);
    c->launches++;
    int h = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(flag);
    if (e != cudaSuccess) return set_err(c, GS_ECUDA, "Reusken block inverses: %s", cudaGetErrorString(e));
    if (h) return set_err(c, GS_NONFINITE, "a block row sum of D_rr is singular");
    p->dtinv_ready = true;
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status schur_apply_approx(gs_ctx* c, int type, int dir, int inverse, int order, const void* xb_dev,
                             void* yb_dev) {
    if (!c) return GS_EINVAL;
    if (order == 2) return schur_apply_reusken(c, type, dir, inverse, xb_dev, yb_dev);
    if (order != 1) return set_err(c, GS_EINVAL, "approximation order %d is not 1 or 2", order);
    if (!xb_dev || !yb_dev) return set_err(c, GS_EINVAL, "null vector");
    if (type != GS_TYPE_I && type != GS_TYPE_II) return set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    const int64_t nb = p->nb, V = c->V, nr = V - nb;
    if ((s = ensure_inner(c, nr)) != GS_OK) return s;
    double2* t = c->inner.rhs;
    double2* z = c->inner.sol;
    const double2* xb = (const double2*)xb_dev;
    // first order: D_rr replaced by its diagonal d = (m0 + 4) 1, so with
    // t = -D_rb x_b, z = t / (m0 + 4) and S~_bb x_b = (D [x_b; z])_b
    StencilArgs a;
    memset(&a, 0, sizeof a);
    a.diag = c->m0 + 4.0;
    a.plan = p;
    a.nbr = p->nbr;
    a.links = p->links;
    a.out = t;
    a.o0 = nb;
    a.n_out = nr;
    a.inA = xb;
    a.a0 = 0;
    a.a1 = nb;
    a.b1 = nb;
    a.negate = 1;
    if ((s = launch_stencil_f64(c, a)) != GS_OK) return s;
    if ((s = launch_scale_copy(c, t, z, nr * kSiteC, 1.0 / (c->m0 + 4.0))) != GS_OK) return s;
    a.out = (double2*)yb_dev;
    a.o0 = 0;
    a.n_out = nb;
    a.inA = xb;
    a.a0 = 0;
    a.a1 = nb;
    a.inB = z;
    a.b1 = V;
    a.negate = 0;
    return launch_stencil_f64(c, a);
}

gs_status schur_apply_reusken(gs_ctx* c, int type, int dir, int inverse, const void* xb_dev, void* yb_dev) {
    if (!c) return GS_EINVAL;
    if (!xb_dev || !yb_dev) return set_err(c, GS_EINVAL, "null vector");
    if (type != GS_TYPE_I && type != GS_TYPE_II) return set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    if ((s = reusken_prepare(c, p)) != GS_OK) return s;
    const int64_t nb = p->nb, V = c->V, nr = V - nb;
    if ((s = ensure_inner(c, nr)) != GS_OK) return s;
    double2* t = c->inner.rhs;
    double2* z = c->inner.sol;
    double2* w = c->inner.r;
    double2* u = c->inner.v;
    const double2* xb = (const double2*)xb_dev;
    StencilArgs a;
    memset(&a, 0, sizeof a);
    a.diag = c->m0 + 4.0;
    a.plan = p;
    a.nbr = p->nbr;
    a.links = p->links;
    // t = -D_rb x_b
    a.out = t;
    a.o0 = nb;
    a.n_out = nr;
    a.inA = xb;
    a.a0 = 0;
    a.a1 = nb;
    a.b1 = nb;
    a.negate = 1;
    if ((s = launch_stencil_f64(c, a)) != GS_OK) return s;
    // w = d~^-1 t
    const int g = grid_for(nr * 12, 256, c->num_sms * 16);
    k_reusken_block<<<g, 256, 0, c->stream>>>(p->dtinv, t, w, nr);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    // u = D_rr w
    a.out = u;
    a.inA = w;
    a.a0 = nb;
    a.a1 = V;
    a.b1 = V;
    a.negate = 0;
    if ((s = launch_stencil_f64(c, a)) != GS_OK) return s;
    // z = w + (t - u) / (m0 + 4) = M t
    k_reusken_combine<<<g, 256, 0, c->stream>>>(w, t, u, z, nr * 12, 1.0 / (c->m0 + 4.0));
    c->launches++;
    GS_CHECK_LAUNCH(c);
    // y_b = (D [x_b; z])_b = D_bb x_b - D_br M D_rb x_b
    a.out = (double2*)yb_dev;
    a.o0 = 0;
    a.n_out = nb;
    a.inA = xb;
    a.a0 = 0;
    a.a1 = nb;
    a.inB = z;
    a.b1 = V;
    return launch_stencil_f64(c, a);
}

}  // extern "C"
