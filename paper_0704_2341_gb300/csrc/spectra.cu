// Extreme parts of the spectrum of the Wilson operator on the GPU: the
// 2-norm condition number of D (Table 1's second row, read as
// sigma_max / sigma_min) by Lanczos on the Hermitian D^H D, and the
// eigenvalues of D with the smallest real part by Arnoldi (where the spectrum
// approaches or surrounds the origin, unpreconditioned BiCGStab stalls).
//
// D^H D is applied as D, gamma_5, D, gamma_5 (gamma_5-hermiticity,
// D^H = gamma_5 D gamma_5; gamma_5 = diag(1, 1, -1, -1) in the chiral basis).
// The Krylov vectors live on the GPU; the small projected problems (a real
// symmetric tridiagonal matrix, a complex upper Hessenberg matrix) are solved
// on the host: extreme eigenvalues of the tridiagonal by Sturm-sequence
// bisection, all eigenvalues of the Hessenberg matrix by the shifted QR
// algorithm (Givens rotations, Wilkinson shifts, deflation).
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "gs_internal.cuh"

namespace gs {
namespace {

using cplx = std::complex<double>;

// y = gamma_5 x: spin components 2 and 3 change sign
__global__ void k_gamma5(const double2* __restrict__ x, double2* __restrict__ y, int64_t nsites) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsites * kSiteC;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(i % kSiteC);
        const double2 v = x[i];
        y[i] = comp < 6 ? v : make_double2(-v.x, -v.y);
    }
}

gs_status gamma5(gs_ctx* c, const double2* x, double2* y) {
    k_gamma5<<<grid_for(c->V * kSiteC, 256, c->num_sms * 16), 256, 0, c->stream>>>(x, y, c->V);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status apply_D(gs_ctx* c, const double2* x, double2* y) {
    const Plan* p = c->plans[0];
    StencilArgs a;
    memset(&a, 0, sizeof a);
    a.out = y;
    a.o0 = 0;
    a.n_out = c->V;
    a.inA = x;
    a.a0 = 0;
    a.a1 = c->V;
    a.b1 = c->V;
    a.diag = c->m0 + 4.0;
    a.plan = p;
    a.nbr = p->nbr;
    a.links = p->links;
    return launch_stencil_f64(c, a);
}

// y = D^H D x  (tmp: one scratch vector)
gs_status apply_DhD(gs_ctx* c, const double2* x, double2* y, double2* tmp) {
    gs_status s;
    if ((s = apply_D(c, x, tmp)) != GS_OK) return s;
    if ((s = gamma5(c, tmp, y)) != GS_OK) return s;
    if ((s = apply_D(c, y, tmp)) != GS_OK) return s;
    return gamma5(c, tmp, y);
}

// number of eigenvalues of the symmetric tridiagonal (a, b) below x
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, int m, double x) {
    int cnt = 0;
    double q = a[0] - x;
    if (q < 0.0) ++cnt;
    for (int i = 1; i < m; ++i) {
        const double qq = (q != 0.0) ? q : 1e-300;
        q = a[i] - x - b[i - 1] * b[i - 1] / qq;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// the k-th smallest eigenvalue (k = 0 .. m-1) of the tridiagonal, by bisection
double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int m, int k) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {   // Gershgorin bounds
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(fabs(lo), fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, m, mid) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Last component of the unit eigenvector of the tridiagonal for its
// eigenvalue theta, by three steps of inverse iteration (T - theta' 1) z = y,
// theta' a hair off theta, each solved by Gaussian elimination with partial
// pivoting between neighbouring rows.
double tridiag_last_component(const std::vector<double>& a, const std::vector<double>& b, int m, double theta) {
    if (m == 1) return 1.0;
    const double scale = std::max(fabs(theta), 1e-300);
    const double th = theta + 1e-12 * scale;
    std::vector<double> y(m, 1.0 / sqrt((double)m));
    for (int it = 0; it < 3; ++it) {
        // rows as (d, u, w): diagonal, first and second super-diagonal (fill-in)
        std::vector<double> d(m), u(m, 0.0), w(m, 0.0), r(y);
        for (int i = 0; i < m; ++i) {
            d[i] = a[i] - th;
            if (i < m - 1) u[i] = b[i];
        }
        std::vector<double> lo(m, 0.0);   // sub-diagonal of the row below
        for (int i = 0; i < m - 1; ++i) lo[i] = b[i];
        for (int i = 0; i < m - 1; ++i) {
            // rows i and i + 1; pivot on the larger of d[i], lo[i]
            if (fabs(lo[i]) > fabs(d[i])) {
                std::swap(d[i], lo[i]);
                const double ui = u[i], wi = w[i];
                u[i] = d[i + 1];
                w[i] = (i + 1 < m - 1) ? u[i + 1] : 0.0;
                d[i + 1] = ui;
                if (i + 1 < m - 1) u[i + 1] = wi;
                std::swap(r[i], r[i + 1]);
            }
            if (d[i] == 0.0) d[i] = 1e-300;
            const double f = lo[i] / d[i];
            d[i + 1] -= f * u[i];
            if (i + 1 < m - 1) u[i + 1] -= f * w[i];
            r[i + 1] -= f * r[i];
        }
        if (d[m - 1] == 0.0) d[m - 1] = 1e-300;
        std::vector<double> z(m);
        for (int i = m - 1; i >= 0; --i) {
            double v = r[i];
            if (i + 1 < m) v -= u[i] * z[i + 1];
            if (i + 2 < m) v -= w[i] * z[i + 2];
            z[i] = v / d[i];
        }
        double nz = 0.0;
        for (double v : z) nz += v * v;
        nz = sqrt(nz);
        if (!(nz > 0.0) || !isfinite(nz)) break;
        for (int i = 0; i < m; ++i) y[i] = z[i] / nz;
    }
    return y[m - 1];
}

// All eigenvalues of the n x n complex upper Hessenberg matrix H (row-major,
// destroyed) by the shifted QR algorithm.  Returns false if an eigenvalue did
// not converge in 60 iterations.
bool hessenberg_eigenvalues(std::vector<cplx>& H, int n, std::vector<cplx>& ev) {
    auto h = [&](int i, int j) -> cplx& { return H[(size_t)i * n + j]; };
    ev.assign(n, cplx(0.0));
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0;
    while (hi >= 0) {
        // deflate at the lowest negligible subdiagonal entry of the active block
        int l = hi;
        while (l > 0) {
            const double sc = std::abs(h(l - 1, l - 1)) + std::abs(h(l, l));
            if (std::abs(h(l, l - 1)) <= eps * (sc > 0.0 ? sc : 1.0)) {
                h(l, l - 1) = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {
            ev[hi] = h(hi, hi);
            --hi;
            iter = 0;
            continue;
        }
        if (++iter > 60) return false;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 closer to h(hi, hi)
        cplx mu;
        {
            const cplx a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
            const cplx tr = a + d, det = a * d - b * c;
            const cplx disc = std::sqrt(tr * tr - 4.0 * det);
            const cplx e1 = 0.5 * (tr + disc), e2 = 0.5 * (tr - disc);
            mu = std::abs(e1 - d) < std::abs(e2 - d) ? e1 : e2;
            if (iter % 11 == 10) mu += std::abs(h(hi, hi - 1));   // exceptional shift
        }
        // one QR step on the active block l..hi: H - mu = Q R, H <- R Q + mu
        std::vector<cplx> cs(hi - l), sn(hi - l);
        for (int k = l; k <= hi; ++k) h(k, k) -= mu;
        for (int k = l; k < hi; ++k) {
            const cplx x = h(k, k), y = h(k + 1, k);
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            cplx c = 1.0, s = 0.0;
            if (r > 0.0) {
                c = x / r;
                s = y / r;
            }
            cs[k - l] = c;
            sn[k - l] = s;
            // rows k, k + 1 <- G [rows k, k + 1], G = [[conj c, conj s], [-s, c]]
            for (int j = k; j < n; ++j) {
                const cplx u = h(k, j), v = h(k + 1, j);
                h(k, j) = std::conj(c) * u + std::conj(s) * v;
                h(k + 1, j) = -s * u + c * v;
            }
        }
        for (int k = l; k < hi; ++k) {
            const cplx c = cs[k - l], s = sn[k - l];
            // columns k, k + 1 <- [columns k, k + 1] G^H
            for (int i = 0; i <= std::min(k + 2, hi); ++i) {
                const cplx u = h(i, k), v = h(i, k + 1);
                h(i, k) = u * c + v * s;
                h(i, k + 1) = -u * std::conj(s) + v * std::conj(c);
            }
        }
        for (int k = l; k <= hi; ++k) h(k, k) += mu;
    }
    return true;
}

struct KrylovWork {
    double2* basis = nullptr;   // Arnoldi: (m + 1) vectors; Lanczos: 3
    double2* w = nullptr;
    double2* tmp = nullptr;
    double2* dots = nullptr;    // device [2 (m + 2) + 1]
    double2* dots_host = nullptr;
    void release() {
        cudaFree(basis);
        cudaFree(w);
        cudaFree(tmp);
        cudaFree(dots);
        if (dots_host) cudaFreeHost(dots_host);
        basis = w = tmp = dots = dots_host = nullptr;
    }
};

gs_status krylov_alloc(gs_ctx* c, KrylovWork& k, int nvec, int ndots) {
    const size_t vb = (size_t)c->V * kSiteC * sizeof(double2);
    if (cudaMalloc(&k.basis, vb * nvec) != cudaSuccess || cudaMalloc(&k.w, vb) != cudaSuccess ||
        cudaMalloc(&k.tmp, vb) != cudaSuccess || cudaMalloc(&k.dots, ndots * sizeof(double2)) != cudaSuccess ||
        cudaHostAlloc((void**)&k.dots_host, ndots * sizeof(double2), 0) != cudaSuccess) {
        cudaGetLastError();
        k.release();
        return set_err(c, GS_ENOMEM, "allocating the Krylov basis (%d vectors) failed", nvec);
    }
    return GS_OK;
}

gs_status read_dots(gs_ctx* c, KrylovWork& k, int n) {
    GS_CUDA(c, cudaMemcpyAsync(k.dots_host, k.dots, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_condition_number(gs_ctx* c, const void* start_dev, int max_steps, double tol, double* kappa_out,
                              double* sigma_min_out, double* sigma_max_out, int* steps_out) {
    if (!c) return GS_EINVAL;
    if (!start_dev || !kappa_out) return set_err(c, GS_EINVAL, "null argument");
    if (max_steps < 2 || !(tol > 0.0)) return set_err(c, GS_EINVAL, "bad step limit or tolerance");
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    const int64_t n = c->V * kSiteC;
    KrylovWork k;
    gs_status s = krylov_alloc(c, k, 3, 4);
    if (s != GS_OK) return s;
    std::vector<double> a, b;
    double lmin = 0.0, lmax = 0.0, res_min = 0.0, res_max = 0.0;
    int steps = 0;
    auto run = [&]() -> gs_status {
        gs_status e;
        double2* q[3] = {k.basis, k.basis + n, k.basis + 2 * n};
        // q0 = start / ||start||
        if ((e = launch_norm2(c, c->red, (const double2*)start_dev, n, (double*)k.dots)) != GS_OK) return e;
        if ((e = read_dots(c, k, 1)) != GS_OK) return e;
        const double s0 = sqrt(k.dots_host[0].x);
        if (!(s0 > 0.0) || !isfinite(s0)) return set_err(c, GS_EINVAL, "the start vector is zero or not finite");
        if ((e = launch_scale_copy(c, (const double2*)start_dev, q[0], n, 1.0 / s0)) != GS_OK) return e;
        GS_CUDA(c, cudaMemsetAsync(q[2], 0, (size_t)n * sizeof(double2), c->stream));   // q_{-1}
        double beta_prev = 0.0;
        for (int j = 0; j < max_steps; ++j) {
            double2* qj = q[j % 3];
            double2* qm = q[(j + 2) % 3];
            double2* qn = q[(j + 1) % 3];
            // w = A q_j - beta_{j-1} q_{j-1}; alpha = <q_j, w>; w -= alpha q_j
            if ((e = apply_DhD(c, qj, k.w, k.tmp)) != GS_OK) return e;
            if ((e = launch_axpby(c, make_double2(-beta_prev, 0.0), qm, make_double2(1.0, 0.0), k.w, n)) != GS_OK)
                return e;
            if ((e = launch_multidot(c, c->red, qj, n, 1, k.w, n, k.dots, 0)) != GS_OK) return e;
            if ((e = read_dots(c, k, 1)) != GS_OK) return e;
            const double alpha = k.dots_host[0].x;
            if ((e = launch_axpby(c, make_double2(-alpha, 0.0), qj, make_double2(1.0, 0.0), k.w, n)) != GS_OK)
                return e;
            if ((e = launch_norm2(c, c->red, k.w, n, (double*)k.dots)) != GS_OK) return e;
            if ((e = read_dots(c, k, 1)) != GS_OK) return e;
            const double beta = sqrt(k.dots_host[0].x);
            if (!isfinite(alpha) || !isfinite(beta)) return set_err(c, GS_NONFINITE, "non-finite Lanczos coefficient");
            a.push_back(alpha);
            steps = j + 1;
            const bool last = beta == 0.0 || j + 1 == max_steps;
            if (steps % 20 == 0 || last) {
                // extreme Ritz values and their residual estimates
                // beta_j |last component of the Ritz vector| (Paige)
                lmin = tridiag_eig(a, b, steps, 0);
                lmax = tridiag_eig(a, b, steps, steps - 1);
                res_min = beta * fabs(tridiag_last_component(a, b, steps, lmin));
                res_max = beta * fabs(tridiag_last_component(a, b, steps, lmax));
                if (res_min <= tol * fabs(lmin) && res_max <= tol * fabs(lmax)) return GS_OK;
            }
            if (beta == 0.0) return GS_OK;   // an invariant subspace: T is exact there
            b.push_back(beta);
            if ((e = launch_scale_copy(c, k.w, qn, n, 1.0 / beta)) != GS_OK) return e;
            beta_prev = beta;
        }
        return set_err(c, GS_MAXITER, "Lanczos: extreme eigenvalues not converged in %d steps (residual "
                                      "estimates %.2e, %.2e)", max_steps, res_min, res_max);
    };
    s = run();
    if (c->stream) cudaStreamSynchronize(c->stream);
    k.release();
    if (steps_out) *steps_out = steps;
    if (s == GS_OK || s == GS_MAXITER) {
        const double smin = sqrt(lmin > 0.0 ? lmin : 0.0), smax = sqrt(lmax > 0.0 ? lmax : 0.0);
        *kappa_out = smin > 0.0 ? smax / smin : INFINITY;
        if (sigma_min_out) *sigma_min_out = smin;
        if (sigma_max_out) *sigma_max_out = smax;
    }
    return s;
}

gs_status gs_leftmost_eigenvalues(gs_ctx* c, const void* start_dev, int m, int k_want, double* re_out,
                                  double* im_out, int* found_out) {
    if (!c) return GS_EINVAL;
    if (!start_dev || !re_out || !im_out) return set_err(c, GS_EINVAL, "null argument");
    const int64_t n = c->V * kSiteC;
    if (m < 2 || m > 4096 || m > n) return set_err(c, GS_EINVAL, "Krylov dimension %d not in 2..min(4096, N)", m);
    if (k_want < 1 || k_want > m) return set_err(c, GS_EINVAL, "k = %d not in 1..m", k_want);
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    KrylovWork kw;
    gs_status s = krylov_alloc(c, kw, m + 1, 2 * (m + 2) + 1);
    if (s != GS_OK) return s;
    std::vector<cplx> H((size_t)(m + 1) * m, cplx(0.0));
    int steps = 0;
    auto run = [&]() -> gs_status {
        gs_status e;
        double2* V = kw.basis;
        if ((e = launch_norm2(c, c->red, (const double2*)start_dev, n, (double*)kw.dots)) != GS_OK) return e;
        if ((e = read_dots(c, kw, 1)) != GS_OK) return e;
        const double s0 = sqrt(kw.dots_host[0].x);
        if (!(s0 > 0.0) || !isfinite(s0)) return set_err(c, GS_EINVAL, "the start vector is zero or not finite");
        if ((e = launch_scale_copy(c, (const double2*)start_dev, V, n, 1.0 / s0)) != GS_OK) return e;
        for (int j = 0; j < m; ++j) {
            // w = D v_j, orthogonalised twice against v_0 .. v_j (CGS2)
            if ((e = apply_D(c, V + (size_t)j * n, kw.w)) != GS_OK) return e;
            double2* h1 = kw.dots;
            double2* h2 = kw.dots + (m + 2);
            if ((e = launch_multidot(c, c->red, V, n, j + 1, kw.w, n, h1, 0)) != GS_OK) return e;
            if ((e = launch_multiaxpy(c, V, n, j + 1, h1, kw.w, n, -1)) != GS_OK) return e;
            if ((e = launch_multidot(c, c->red, V, n, j + 1, kw.w, n, h2, 0)) != GS_OK) return e;
            if ((e = launch_multiaxpy(c, V, n, j + 1, h2, kw.w, n, -1)) != GS_OK) return e;
            if ((e = launch_norm2(c, c->red, kw.w, n, (double*)(kw.dots + 2 * (m + 2)))) != GS_OK) return e;
            if ((e = read_dots(c, kw, 2 * (m + 2) + 1)) != GS_OK) return e;
            for (int i = 0; i <= j; ++i)
                H[(size_t)i * m + j] = cplx(kw.dots_host[i].x + kw.dots_host[m + 2 + i].x,
                                            kw.dots_host[i].y + kw.dots_host[m + 2 + i].y);
            const double hn = sqrt(kw.dots_host[2 * (m + 2)].x);
            if (!isfinite(hn)) return set_err(c, GS_NONFINITE, "non-finite Arnoldi norm");
            steps = j + 1;
            if (j + 1 < m) H[(size_t)(j + 1) * m + j] = hn;
            if (hn == 0.0) break;   // invariant subspace: its eigenvalues are exact
            if ((e = launch_scale_copy(c, kw.w, V + (size_t)(j + 1) * n, n, 1.0 / hn)) != GS_OK) return e;
        }
        return GS_OK;
    };
    s = run();
    if (c->stream) cudaStreamSynchronize(c->stream);
    kw.release();
    if (s != GS_OK) return s;
    // Ritz values: the eigenvalues of the leading steps x steps block of H
    std::vector<cplx> Hm((size_t)steps * steps);
    for (int i = 0; i < steps; ++i)
        for (int j = 0; j < steps; ++j) Hm[(size_t)i * steps + j] = H[(size_t)i * m + j];
    std::vector<cplx> ev;
    if (!hessenberg_eigenvalues(Hm, steps, ev))
        return set_err(c, GS_MAXITER, "the QR iteration on the Hessenberg matrix did not converge");
    std::sort(ev.begin(), ev.end(), [](const cplx& x, const cplx& y) {
        return x.real() < y.real() || (x.real() == y.real() && x.imag() < y.imag());
    });
    const int found = std::min(k_want, steps);
    for (int i = 0; i < found; ++i) {
        re_out[i] = ev[i].real();
        im_out[i] = ev[i].imag();
    }
    if (found_out) *found_out = found;
    return GS_OK;
}

}  // extern "C"
