// The cyclic-reduction V-cycle preconditioner of Section 4 on the GPU, and
// BiCGStab on D x = f, plain or right-preconditioned by it (Table 1's two
// solvers).
//
// Levels.  Level 0 is D on the lattice, blocked by the permutation of the
// first coarsening step (the context's plan: label-range stencils).  Level
// l + 1 is the Section 3 approximation S~ of level l's operator on level l's
// coarse set, indexed by level l's coarse labels in order; when it is not the
// coarsest, it is blocked by its own permutation, built by the same
// closed-form label kernel for the coarse extents (Type I halves every
// extent, Type II(mu) halves L_mu; the inverse types have the same counts),
// and stored as a block-sparse matrix (12 x 12 complex blocks, rows and
// columns in its label order).  The coarsest level is inverted exactly: its
// operator is assembled as a dense matrix and inverted once by Gauss-Jordan
// elimination with partial pivoting.
//
// Assembly by probing.  The sparsity pattern of S~ = A_bb - A_br M A_rb
// (M = d^-1 + d~^-1 - d^-1 A_rr d~^-1, or d^-1 at first order) follows from
// level l's pattern; its columns are coloured so that no two columns of one
// colour share a row, and S~ is applied (the tested level-0 apply of
// schur_apply_reusken / schur_apply_approx, or the block-sparse form below)
// to the 12 component probes of each colour; each result row holds one
// block column of its colour's block.
//
// One application x = V_l(f), the block UL solve of Section 1 with the exact
// Schur complement replaced by the next level:
//   F = P_l f;  z = A_rr^-1 F_r;  w_b = F_b - A_br z;  x_b = V_{l+1}(w_b);
//   x_r = A_rr^-1 (F_r - A_rb x_b);  x = P_l^T [x_b; x_r],
// the rest-set inverses by BiCGStab to a tolerance (1e-2 in the paper):
// level 0 with the library's inner FP64 BiCGStab, lower levels with a
// BiCGStab over the block-sparse rest block.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "block12.cuh"

namespace gs {
namespace {

using cplx = std::complex<double>;

// ---------------------------------------------------------------------------
// block-sparse operators (12 x 12 complex blocks, rows / columns in labels)
// ---------------------------------------------------------------------------
struct BsrArgs {
    double2* out;
    int64_t o0, n_out;           // output rows o0 .. o0 + n_out - 1
    const double2* inA;          // input labels [a0, a1) from inA, [a1, b1) from inB
    int64_t a0, a1;
    const double2* inB;
    int64_t b1;
    const double2* addend;       // out = addend + sign * sum (may be null)
    int negate;
    const int32_t* rowptr;
    const int32_t* col;
    const double2* val;          // [nnzb][12][12], row-major blocks
};

constexpr int kBsrRows = 8;      // rows per block of 96 threads (12 per row)

// out[k] = [addend[k]] + sign * sum_{b in row o0 + k, col j in the input
// ranges} val_b in(j); thread (row, a) computes component a.
__global__ void __launch_bounds__(96) k_bsr_apply(BsrArgs a) {
    const int comp = threadIdx.x % 12;
    const int rloc = threadIdx.x / 12;
    for (int64_t k = (int64_t)blockIdx.x * kBsrRows + rloc; k < a.n_out;
         k += (int64_t)gridDim.x * kBsrRows) {
        const int64_t row = a.o0 + k;
        double2 acc = make_double2(0.0, 0.0);
        const int32_t e = a.rowptr[row + 1];
        for (int32_t b = a.rowptr[row]; b < e; ++b) {
            const int64_t j = a.col[b];
            const double2* src;
            if (j >= a.a0 && j < a.a1) src = a.inA + (j - a.a0) * kSiteC;
            else if (j >= a.a1 && j < a.b1) src = a.inB + (j - a.a1) * kSiteC;
            else continue;
            const double2* v = a.val + (int64_t)b * 144 + comp * 12;
#pragma unroll
            for (int q = 0; q < 12; ++q) cfma(acc, v[q], src[q]);
        }
        if (a.negate) acc = make_double2(-acc.x, -acc.y);
        if (a.addend) acc = cadd(acc, a.addend[k * kSiteC + comp]);
        a.out[k * kSiteC + comp] = acc;
    }
}

// out[k] = B[k] in[k], 12 x 12 block per site; thread per (site, row)
__global__ void k_block_mul(const double2* __restrict__ B, const double2* __restrict__ in,
                            double2* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * 12;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 12;
        const int r = (int)(i - k * 12);
        const double2* row = B + k * 144 + r * 12;
        const double2* x = in + k * 12;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 12; ++q) cfma(acc, row[q], x[q]);
        out[i] = acc;
    }
}

// For rest row k (label nb + k): d[k] = its diagonal block, dt[k] = the sum of
// its blocks in rest columns (the block row sum over r); thread per element.
__global__ void k_rest_diag_rowsum(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   const double2* __restrict__ val, int64_t nb, int64_t nr,
                                   double2* __restrict__ d, double2* __restrict__ dt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr * 144;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 144;
        const int e = (int)(i - k * 144);
        const int64_t row = nb + k;
        double2 dd = make_double2(0.0, 0.0), ss = make_double2(0.0, 0.0);
        for (int32_t b = rowptr[row]; b < rowptr[row + 1]; ++b) {
            const int64_t j = col[b];
            if (j < nb) continue;
            const double2 v = val[(int64_t)b * 144 + e];
            ss = cadd(ss, v);
            if (j == row) dd = v;
        }
        d[i] = dd;
        dt[i] = ss;
    }
}

// in place: blocks[k] <- blocks[k]^-1 (one thread per block); status = 1 on a
// singular block
__global__ void k_block_inverse(double2* __restrict__ blocks, int64_t n, int* status) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double2 A[12][12], B[12][12];
        double2* blk = blocks + k * 144;
        for (int r = 0; r < 12; ++r)
            for (int q = 0; q < 12; ++q) A[r][q] = blk[r * 12 + q];
        const bool ok = invert12(A, B);
        if (!ok) atomicExch(status, 1);
        for (int r = 0; r < 12; ++r)
            for (int q = 0; q < 12; ++q) blk[r * 12 + q] = ok ? B[r][q] : make_double2(0.0, 0.0);
    }
}

// probe vector of colour c, component k: e[j][q] = (colour[j] == c && q == k)
__global__ void k_probe_fill(const int32_t* __restrict__ colour, int c, int k, double2* __restrict__ e,
                             int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * 12;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / 12;
        const int q = (int)(i - j * 12);
        e[i] = make_double2((colour[j] == c && q == k) ? 1.0 : 0.0, 0.0);
    }
}

// block column k of the blocks selected for one colour: sel[i] >= 0 is the
// destination of row i's block of that colour, y the probe's result.
//   dense == 0: sel[i] is a block index, val[sel][a][k] = y[i][a]
//   dense != 0: sel[i] is the column site j, A[12 i + a][12 j + k] = y[i][a]
__global__ void k_probe_scatter(const int32_t* __restrict__ sel, const double2* __restrict__ y, int k,
                                double2* __restrict__ dst, int64_t n, int dense) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * 12;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / 12;
        const int a = (int)(t - i * 12);
        const int32_t s = sel[i];
        if (s < 0) continue;
        if (dense) dst[(i * 12 + a) * (n * 12) + (int64_t)s * 12 + k] = y[t];
        else dst[(int64_t)s * 144 + a * 12 + k] = y[t];
    }
}

// ---------------------------------------------------------------------------
// dense in-place Gauss-Jordan inversion with partial pivoting (coarsest level)
// ---------------------------------------------------------------------------
constexpr int kGjThreads = 1024;

// step k, one block: pivot row of column k (largest modulus among rows >= k,
// the first on ties), row swap, row k scaled by the pivot's inverse, column
// k moved into f (f[k] = 0) and cleared.  status = 1 on a zero pivot.
__global__ void __launch_bounds__(kGjThreads) k_gj_pivot(double2* __restrict__ A, int64_t N, int64_t k,
                                                        int32_t* __restrict__ piv, double2* __restrict__ f,
                                                        int* status) {
    __shared__ double sbest[kGjThreads / 32];
    __shared__ int64_t sidx[kGjThreads / 32];
    __shared__ int64_t s_p;
    __shared__ double2 s_inv;
    double best = -1.0;
    int64_t bi = N;
    for (int64_t i = k + threadIdx.x; i < N; i += blockDim.x) {
        const double2 v = A[i * N + k];
        const double m = v.x * v.x + v.y * v.y;
        if (m > best || (m == best && i < bi)) {
            best = m;
            bi = i;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        sbest[threadIdx.x >> 5] = best;
        sidx[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = -1.0;
        int64_t p = N;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            if (sbest[w] > b || (sbest[w] == b && sidx[w] < p)) {
                b = sbest[w];
                p = sidx[w];
            }
        if (!(b > 0.0) || !isfinite(b) || p >= N) {
            atomicExch(status, 1);
            p = k;
            b = 1.0;
        }
        s_p = p;
        piv[k] = (int32_t)p;
        const double2 pv = A[p * N + k];
        const double inv = 1.0 / (pv.x * pv.x + pv.y * pv.y);
        s_inv = make_double2(pv.x * inv, -pv.y * inv);
    }
    __syncthreads();
    const int64_t p = s_p;
    if (p != k)
        for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
            const double2 t = A[k * N + j];
            A[k * N + j] = A[p * N + j];
            A[p * N + j] = t;
        }
    __syncthreads();
    const double2 inv = s_inv;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x)
        A[k * N + j] = (j == k) ? inv : cmul(A[k * N + j], inv);
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        if (i == k) {
            f[i] = make_double2(0.0, 0.0);
        } else {
            f[i] = A[i * N + k];
            A[i * N + k] = make_double2(0.0, 0.0);
        }
    }
}

// step k: A[i][j] -= f[i] A[k][j] for every row i != k
__global__ void k_gj_eliminate(double2* __restrict__ A, int64_t N, int64_t k, const double2* __restrict__ f) {
    const int64_t total = N * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / N;
        if (i == k) continue;
        const int64_t j = t - i * N;
        const double2 fi = f[i];
        if (fi.x == 0.0 && fi.y == 0.0) continue;
        const double2 akj = A[k * N + j];
        double2 v = A[t];
        v.x -= fi.x * akj.x - fi.y * akj.y;
        v.y -= fi.x * akj.y + fi.y * akj.x;
        A[t] = v;
    }
}

// undo the row interchanges on the columns of the inverse (last step first)
__global__ void k_gj_unscramble(double2* __restrict__ A, int64_t N, const int32_t* __restrict__ piv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2* row = A + i * N;
        for (int64_t k = N - 1; k >= 0; --k) {
            const int64_t p = piv[k];
            if (p != k) {
                const double2 t = row[k];
                row[k] = row[p];
                row[p] = t;
            }
        }
    }
}

// y = A x, dense N x N (row-major); one warp per row
__global__ void k_dense_gemv(const double2* __restrict__ A, const double2* __restrict__ x,
                             double2* __restrict__ y, int64_t N) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < N; i += warps) {
        double2 acc = make_double2(0.0, 0.0);
        const double2* row = A + i * N;
        for (int64_t j = lane; j < N; j += 32) cfma(acc, row[j], x[j]);
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) y[i] = acc;
    }
}

}  // namespace
}  // namespace gs

using namespace gs;

namespace {

struct HostCsr {                 // a block pattern on the host: rows of column lists
    std::vector<int32_t> row;    // [n + 1]
    std::vector<int32_t> col;
};

struct VLevel {
    int type = 0, dir = 0, inverse = 0;   // the coarsening of this level
    int dims[4] = {0, 0, 0, 0};           // extents of this level's lattice
    int64_t n = 0, nb = 0;                // sites, coarse sites
    Plan* plan = nullptr;                 // level 0: the context's plan
    int32_t* perm = nullptr;              // levels >= 1: label -> site (device)
    int32_t* label = nullptr;             // site -> label (device)
    HostCsr pat;                          // levels >= 1: the pattern in label order
    int32_t* rowptr = nullptr;            // levels >= 1: BSR (device)
    int32_t* col = nullptr;
    double2* val = nullptr;
    double2* dinv = nullptr;              // [nr][144] (built with the next level)
    double2* dtinv = nullptr;
    // workspace (device)
    double2 *F = nullptr, *X = nullptr, *Z = nullptr, *T = nullptr, *Wb = nullptr;
    double2 *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr;
};

}  // namespace

struct gs_vcycle {
    gs_ctx* c = nullptr;
    int nlev = 0;                        // levels, the last one the coarsest
    int order = 2;
    double rest_tol = 1e-2;
    int rest_maxit = 100000;
    std::vector<VLevel> lev;             // 0 .. nlev - 2 are blocked levels
    int coarse_dims[4] = {0, 0, 0, 0};
    int64_t nc = 0;                      // coarsest sites
    double2* Ac = nullptr;               // coarsest operator, dense [12 nc][12 nc]
    double2* Ainv = nullptr;             // its inverse
    int colours[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // statistics of the rest-set solves since the last reset
    long long rest_solves = 0, rest_iters = 0, rest_unconverged = 0;
    int rest_max_seen = 0;
    // outer BiCGStab workspace (full lattice)
    double2 *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr,
            *ph = nullptr, *sh = nullptr;
    double2* dot_dev = nullptr;          // device scalars of the host-driven solvers
    double2* dot_host = nullptr;         // pinned
};

namespace {

gs_status vc_alloc(gs_ctx* c, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(c, GS_ENOMEM, "V-cycle: device allocation of %zu bytes failed", bytes);
    }
    return GS_OK;
}

int plain_blocks(gs_ctx* c, int64_t n, int block) { return grid_for(n, block, c->num_sms * 16); }

gs_status bsr_launch(gs_ctx* c, const BsrArgs& a) {
    if (a.n_out <= 0) return GS_OK;
    const int g = grid_for(a.n_out, kBsrRows, c->num_sms * 32);
    k_bsr_apply<<<g, 96, 0, c->stream>>>(a);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

BsrArgs bsr_args(const VLevel& L) {
    BsrArgs a;
    memset(&a, 0, sizeof a);
    a.rowptr = L.rowptr;
    a.col = L.col;
    a.val = L.val;
    return a;
}

gs_status block_mul(gs_ctx* c, const double2* B, const double2* in, double2* out, int64_t n) {
    if (n <= 0) return GS_OK;
    k_block_mul<<<plain_blocks(c, n * 12, 256), 256, 0, c->stream>>>(B, in, out, n);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// <a, b> = sum conj(a) b over n complex entries, read back to the host
gs_status vc_dot(gs_vcycle* vc, const double2* a, const double2* b, int64_t n, cplx* out) {
    gs_ctx* c = vc->c;
    gs_status s = launch_multidot(c, c->red, a, n, 1, b, n, vc->dot_dev, 0);
    if (s != GS_OK) return s;
    GS_CUDA(c, cudaMemcpyAsync(vc->dot_host, vc->dot_dev, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = cplx(vc->dot_host[0].x, vc->dot_host[0].y);
    return GS_OK;
}

gs_status vc_norm(gs_vcycle* vc, const double2* a, int64_t n, double* out) {
    cplx d;
    gs_status s = vc_dot(vc, a, a, n, &d);
    *out = sqrt(d.real() > 0.0 ? d.real() : 0.0);
    if (!isfinite(d.real())) *out = d.real();
    return s;
}

gs_status axpby(gs_ctx* c, cplx a, const double2* x, cplx b, double2* y, int64_t n) {
    return launch_axpby(c, make_double2(a.real(), a.imag()), x, make_double2(b.real(), b.imag()), y, n);
}

// z = A_rr^-1 b on a block-sparse level (levels >= 1): van der Vorst's
// BiCGStab, x0 = 0, shadow residual b, stopped when ||s|| or ||r|| <=
// tol ||b|| or after maxit steps (the last iterate is kept).
gs_status bsr_rest_bicgstab(gs_vcycle* vc, VLevel& L, const double2* b, double2* x) {
    gs_ctx* c = vc->c;
    const int64_t nb = L.nb, nr = L.n - L.nb, n = nr * kSiteC;
    const size_t bytes = (size_t)n * sizeof(double2);
    gs_status s;
    GS_CUDA(c, cudaMemsetAsync(x, 0, bytes, c->stream));
    double bnorm;
    if ((s = vc_norm(vc, b, n, &bnorm)) != GS_OK) return s;
    if (!isfinite(bnorm)) return set_err(c, GS_NONFINITE, "V-cycle: non-finite rest-set right-hand side");
    vc->rest_solves++;
    if (bnorm == 0.0) return GS_OK;
    const double target = vc->rest_tol * bnorm;
    GS_CUDA(c, cudaMemcpyAsync(L.r, b, bytes, cudaMemcpyDeviceToDevice, c->stream));
    GS_CUDA(c, cudaMemcpyAsync(L.rhat, b, bytes, cudaMemcpyDeviceToDevice, c->stream));
    GS_CUDA(c, cudaMemsetAsync(L.p, 0, bytes, c->stream));
    GS_CUDA(c, cudaMemsetAsync(L.v, 0, bytes, c->stream));
    BsrArgs A = bsr_args(L);
    A.o0 = nb;
    A.n_out = nr;
    A.a0 = nb;
    A.a1 = L.n;
    A.b1 = L.n;
    cplx rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int it = 0;
    bool conv = false;
    while (!conv && it < vc->rest_maxit) {
        ++it;
        cplx rho;
        if ((s = vc_dot(vc, L.rhat, L.r, n, &rho)) != GS_OK) return s;
        if (rho == 0.0) break;
        const cplx beta = (rho / rho_old) * (alpha / omega);
        // p = r + beta (p - omega v)
        if ((s = axpby(c, -omega, L.v, 1.0, L.p, n)) != GS_OK) return s;
        if ((s = axpby(c, 1.0, L.r, beta, L.p, n)) != GS_OK) return s;
        A.out = L.v;
        A.inA = L.p;
        if ((s = bsr_launch(c, A)) != GS_OK) return s;
        cplx rv;
        if ((s = vc_dot(vc, L.rhat, L.v, n, &rv)) != GS_OK) return s;
        alpha = rho / rv;
        // s = r - alpha v
        GS_CUDA(c, cudaMemcpyAsync(L.s, L.r, bytes, cudaMemcpyDeviceToDevice, c->stream));
        if ((s = axpby(c, -alpha, L.v, 1.0, L.s, n)) != GS_OK) return s;
        double sn;
        if ((s = vc_norm(vc, L.s, n, &sn)) != GS_OK) return s;
        if (!isfinite(sn)) return set_err(c, GS_NONFINITE, "V-cycle: non-finite rest-set residual");
        if (sn <= target) {
            if ((s = axpby(c, alpha, L.p, 1.0, x, n)) != GS_OK) return s;
            conv = true;
            break;
        }
        A.out = L.t;
        A.inA = L.s;
        if ((s = bsr_launch(c, A)) != GS_OK) return s;
        cplx ts, tt;
        if ((s = vc_dot(vc, L.t, L.s, n, &ts)) != GS_OK) return s;
        if ((s = vc_dot(vc, L.t, L.t, n, &tt)) != GS_OK) return s;
        omega = tt.real() > 0.0 ? ts / tt : cplx(0.0);
        // x += alpha p + omega s ; r = s - omega t
        if ((s = axpby(c, alpha, L.p, 1.0, x, n)) != GS_OK) return s;
        if ((s = axpby(c, omega, L.s, 1.0, x, n)) != GS_OK) return s;
        GS_CUDA(c, cudaMemcpyAsync(L.r, L.s, bytes, cudaMemcpyDeviceToDevice, c->stream));
        if ((s = axpby(c, -omega, L.t, 1.0, L.r, n)) != GS_OK) return s;
        rho_old = rho;
        double rn;
        if ((s = vc_norm(vc, L.r, n, &rn)) != GS_OK) return s;
        if (!isfinite(rn)) return set_err(c, GS_NONFINITE, "V-cycle: non-finite rest-set residual");
        conv = rn <= target;
        if (omega == 0.0) break;
    }
    vc->rest_iters += it;
    if (it > vc->rest_max_seen) vc->rest_max_seen = it;
    if (!conv) vc->rest_unconverged++;
    return GS_OK;
}

// z = A_rr^-1 b at level l (level 0: the library's inner FP64 BiCGStab on D_rr)
gs_status rest_solve(gs_vcycle* vc, int l, const double2* b, double2* z) {
    gs_ctx* c = vc->c;
    VLevel& L = vc->lev[l];
    if (l > 0) return bsr_rest_bicgstab(vc, L, b, z);
    gs_solve_opts o;
    gs_default_opts(&o);
    o.inner_tol = vc->rest_tol;
    o.inner_max_iter = vc->rest_maxit;
    gs_solve_stats st;
    memset(&st, 0, sizeof st);
    gs_status s = inner_solve_f64(c, L.plan, b, z, o, st);
    vc->rest_solves++;
    vc->rest_iters += st.inner_iters;
    if (st.inner_max_seen > vc->rest_max_seen) vc->rest_max_seen = st.inner_max_seen;
    if (s == GS_MAXITER) {
        vc->rest_unconverged++;
        return GS_OK;
    }
    return s;
}

// level 0's label-range stencil on the context's plan
StencilArgs stencil0(gs_ctx* c, const Plan* p) {
    StencilArgs a;
    memset(&a, 0, sizeof a);
    a.diag = c->m0 + 4.0;
    a.plan = p;
    a.nbr = p->nbr;
    a.links = p->links;
    return a;
}

// out (level-l rows [o0, o0 + n_out)) = addend - A x over input range [a0, b1)
// (x indexed from a0); A = D at level 0, the block-sparse operator below
gs_status level_residual_part(gs_vcycle* vc, int l, double2* out, int64_t o0, int64_t n_out,
                              const double2* x, int64_t a0, int64_t b1, const double2* addend) {
    gs_ctx* c = vc->c;
    VLevel& L = vc->lev[l];
    if (l == 0) {
        StencilArgs a = stencil0(c, L.plan);
        a.out = out;
        a.o0 = o0;
        a.n_out = n_out;
        a.inA = x;
        a.a0 = a0;
        a.a1 = b1;
        a.b1 = b1;
        a.negate = 1;
        a.addend = addend;
        return launch_stencil_f64(c, a);
    }
    BsrArgs a = bsr_args(L);
    a.out = out;
    a.o0 = o0;
    a.n_out = n_out;
    a.inA = x;
    a.a0 = a0;
    a.a1 = b1;
    a.b1 = b1;
    a.negate = 1;
    a.addend = addend;
    return bsr_launch(c, a);
}

// x = V_l(f), f and x in level l's own order (level 0: site order)
gs_status vc_apply(gs_vcycle* vc, int l, const double2* f, double2* x) {
    gs_ctx* c = vc->c;
    gs_status s;
    if (l == vc->nlev - 1) {
        const int64_t N = vc->nc * 12;
        k_dense_gemv<<<grid_for(N, 8, c->num_sms * 32), 256, 0, c->stream>>>(vc->Ainv, f, x, N);
        c->launches++;
        GS_CHECK_LAUNCH(c);
        return GS_OK;
    }
    VLevel& L = vc->lev[l];
    const int64_t n = L.n, nb = L.nb, nr = n - nb;
    const int32_t* perm = l == 0 ? L.plan->perm : L.perm;
    if ((s = launch_gather(c, perm, f, L.F, n)) != GS_OK) return s;
    // z = A_rr^-1 F_r
    if ((s = rest_solve(vc, l, L.F + nb * kSiteC, L.Z)) != GS_OK) return s;
    // w_b = F_b - A_br z
    if ((s = level_residual_part(vc, l, L.Wb, 0, nb, L.Z, nb, n, L.F)) != GS_OK) return s;
    // x_b = V_{l+1}(w_b)
    if ((s = vc_apply(vc, l + 1, L.Wb, L.X)) != GS_OK) return s;
    // x_r = A_rr^-1 (F_r - A_rb x_b)
    if ((s = level_residual_part(vc, l, L.T, nb, nr, L.X, 0, nb, L.F + nb * kSiteC)) != GS_OK) return s;
    if ((s = rest_solve(vc, l, L.T, L.X + nb * kSiteC)) != GS_OK) return s;
    return launch_scatter(c, perm, L.X, x, n);
}

// y = S~ x on level l's coarse set (l >= 1, block-sparse), x and y of nb
// sites in level l's label order; the Section 3 expression with the level's
// own d and d~:  t' = -A_rb x,  z' = M t',  y = A_bb x + A_br z'.
gs_status bsr_schur_approx(gs_vcycle* vc, int l, const double2* x, double2* y) {
    gs_ctx* c = vc->c;
    VLevel& L = vc->lev[l];
    const int64_t n = L.n, nb = L.nb, nr = n - nb;
    gs_status s;
    // scratch: T = t', Z = z', r = w, v = u (rest vectors of this level)
    BsrArgs a = bsr_args(L);
    a.out = L.T;
    a.o0 = nb;
    a.n_out = nr;
    a.inA = x;
    a.a0 = 0;
    a.a1 = nb;
    a.b1 = nb;
    a.negate = 1;
    if ((s = bsr_launch(c, a)) != GS_OK) return s;
    if (vc->order == 1) {
        if ((s = block_mul(c, L.dinv, L.T, L.Z, nr)) != GS_OK) return s;
    } else {
        // w = d~^-1 t'; u = A_rr w; z' = d^-1 (t' - u) + w
        if ((s = block_mul(c, L.dtinv, L.T, L.r, nr)) != GS_OK) return s;
        a.out = L.v;
        a.inA = L.r;
        a.a0 = nb;
        a.a1 = n;
        a.b1 = n;
        a.negate = 0;
        if ((s = bsr_launch(c, a)) != GS_OK) return s;
        if ((s = launch_axpby(c, make_double2(1.0, 0.0), L.T, make_double2(-1.0, 0.0), L.v, nr * kSiteC)) !=
            GS_OK)
            return s;   // v = t' - u
        if ((s = block_mul(c, L.dinv, L.v, L.Z, nr)) != GS_OK) return s;
        if ((s = launch_axpby(c, make_double2(1.0, 0.0), L.r, make_double2(1.0, 0.0), L.Z, nr * kSiteC)) !=
            GS_OK)
            return s;
    }
    a.out = y;
    a.o0 = 0;
    a.n_out = nb;
    a.inA = x;
    a.a0 = 0;
    a.a1 = nb;
    a.inB = L.Z;
    a.b1 = n;
    a.negate = 0;
    return bsr_launch(c, a);
}

// The pattern of S~ = A_bb - A_br M A_rb on the coarse labels [0, nb) of a
// level with pattern `A` (every row lists its own label too).
void schur_pattern(const HostCsr& A, int64_t nb, int order, HostCsr& out) {
    out.row.assign(nb + 1, 0);
    out.col.clear();
    std::vector<int32_t> mark(nb, -1);
    std::vector<int32_t> cols;
    for (int64_t i = 0; i < nb; ++i) {
        cols.clear();
        auto add = [&](int32_t j) {
            if (mark[j] != (int32_t)i) {
                mark[j] = (int32_t)i;
                cols.push_back(j);
            }
        };
        for (int32_t e = A.row[i]; e < A.row[i + 1]; ++e) {
            const int32_t j = A.col[e];
            if (j < nb) {
                add(j);
                continue;
            }
            // j = r1 in r: the columns reached through M's pattern and A_rb
            auto through = [&](int32_t r2) {
                for (int32_t e3 = A.row[r2]; e3 < A.row[r2 + 1]; ++e3)
                    if (A.col[e3] < nb) add(A.col[e3]);
            };
            through(j);
            if (order == 2)
                for (int32_t e2 = A.row[j]; e2 < A.row[j + 1]; ++e2)
                    if (A.col[e2] >= nb) through(A.col[e2]);
        }
        std::sort(cols.begin(), cols.end());
        out.col.insert(out.col.end(), cols.begin(), cols.end());
        out.row[i + 1] = (int32_t)out.col.size();
    }
}

// Greedy colouring of the columns: two columns that share a row never share
// a colour.  Returns the number of colours.
int colour_columns(const HostCsr& P, int64_t n, std::vector<int32_t>& colour) {
    std::vector<int32_t> tr(n + 1, 0), tc(P.col.size());
    for (int32_t j : P.col) tr[j + 1]++;
    for (int64_t j = 0; j < n; ++j) tr[j + 1] += tr[j];
    {
        std::vector<int32_t> fill(tr.begin(), tr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int32_t e = P.row[i]; e < P.row[i + 1]; ++e) tc[fill[P.col[e]]++] = (int32_t)i;
    }
    colour.assign(n, -1);
    std::vector<int64_t> stamp;
    int ncol = 0;
    for (int64_t j = 0; j < n; ++j) {
        for (int32_t e = tr[j]; e < tr[j + 1]; ++e) {
            const int32_t i = tc[e];
            for (int32_t f = P.row[i]; f < P.row[i + 1]; ++f) {
                const int32_t cj = colour[P.col[f]];
                if (cj >= 0) stamp[cj] = j;
            }
        }
        int cc = 0;
        while (cc < ncol && stamp[cc] == j) ++cc;
        if (cc == ncol) {
            ++ncol;
            stamp.push_back(-1);
        }
        colour[j] = cc;
    }
    return ncol;
}

// Assemble level l + 1's operator by probing S~ of level l.  Natural index of
// the new operator = level l's coarse labels.  dense != 0: into vc->Ac
// (natural order); else into level l + 1's block-sparse storage, whose
// permutation (label[] on the host) must be built already.
gs_status probe_next(gs_vcycle* vc, int l, const HostCsr& P, const std::vector<int32_t>& label_next, bool dense,
                     int* ncolours) {
    gs_ctx* c = vc->c;
    VLevel& L = vc->lev[l];
    const int64_t nb = L.nb;
    std::vector<int32_t> colour;
    const int ncol = colour_columns(P, nb, colour);
    *ncolours = ncol;
    // per colour and row, the destination of that row's block of the colour
    std::vector<int32_t> sel((size_t)ncol * nb, -1);
    if (dense) {
        for (int64_t i = 0; i < nb; ++i)
            for (int32_t e = P.row[i]; e < P.row[i + 1]; ++e)
                sel[(size_t)colour[P.col[e]] * nb + i] = P.col[e];
    } else {
        VLevel& N = vc->lev[l + 1];
        for (int64_t i = 0; i < nb; ++i) {
            const int32_t Li = label_next[i];
            const int32_t* b0 = N.pat.col.data() + N.pat.row[Li];
            const int32_t* b1 = N.pat.col.data() + N.pat.row[Li + 1];
            for (int32_t e = P.row[i]; e < P.row[i + 1]; ++e) {
                const int32_t Lj = label_next[P.col[e]];
                const int32_t* hit = std::lower_bound(b0, b1, Lj);
                sel[(size_t)colour[P.col[e]] * nb + i] = (int32_t)(hit - N.pat.col.data());
            }
        }
    }
    int32_t *colour_dev = nullptr, *sel_dev = nullptr;
    double2 *e = nullptr, *y = nullptr;
    gs_status s = GS_OK;
    auto fail = [&](gs_status st) {
        cudaFree(colour_dev);
        cudaFree(sel_dev);
        cudaFree(e);
        cudaFree(y);
        return st;
    };
    if ((s = vc_alloc(c, (void**)&colour_dev, nb * sizeof(int32_t))) != GS_OK) return fail(s);
    if ((s = vc_alloc(c, (void**)&sel_dev, sel.size() * sizeof(int32_t))) != GS_OK) return fail(s);
    if ((s = vc_alloc(c, (void**)&e, nb * kSiteC * sizeof(double2))) != GS_OK) return fail(s);
    if ((s = vc_alloc(c, (void**)&y, nb * kSiteC * sizeof(double2))) != GS_OK) return fail(s);
    if (cudaMemcpyAsync(colour_dev, colour.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(sel_dev, sel.data(), sel.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess) {
        cudaGetLastError();
        return fail(set_err(c, GS_ECUDA, "V-cycle: copying the probe tables failed"));
    }
    double2* dst = dense ? vc->Ac : vc->lev[l + 1].val;
    const int g = plain_blocks(c, nb * 12, 256);
    for (int cc = 0; cc < ncol && s == GS_OK; ++cc)
        for (int k = 0; k < 12 && s == GS_OK; ++k) {
            k_probe_fill<<<g, 256, 0, c->stream>>>(colour_dev, cc, k, e, nb);
            c->launches++;
            if (l == 0) {
                s = schur_apply_approx(c, L.type, L.dir, L.inverse, vc->order, e, y);
            } else {
                s = bsr_schur_approx(vc, l, e, y);
            }
            if (s != GS_OK) break;
            k_probe_scatter<<<g, 256, 0, c->stream>>>(sel_dev + (size_t)cc * nb, y, k, dst, nb, dense ? 1 : 0);
            c->launches++;
        }
    if (s == GS_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
        s = set_err(c, GS_ECUDA, "V-cycle: probing failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    return fail(s);
}

gs_status alloc_level_work(gs_ctx* c, VLevel& L) {
    const int64_t n = L.n, nb = L.nb, nr = n - nb;
    const size_t sb = kSiteC * sizeof(double2);
    gs_status s;
    if ((s = vc_alloc(c, (void**)&L.F, n * sb)) != GS_OK) return s;
    if ((s = vc_alloc(c, (void**)&L.X, n * sb)) != GS_OK) return s;
    if ((s = vc_alloc(c, (void**)&L.Z, nr * sb)) != GS_OK) return s;
    if ((s = vc_alloc(c, (void**)&L.T, nr * sb)) != GS_OK) return s;
    if ((s = vc_alloc(c, (void**)&L.Wb, nb * sb)) != GS_OK) return s;
    double2** v[6] = {&L.r, &L.rhat, &L.p, &L.v, &L.s, &L.t};
    for (auto pp : v)
        if ((s = vc_alloc(c, (void**)pp, nr * sb)) != GS_OK) return s;
    return GS_OK;
}

void free_level(VLevel& L) {
    void* ptrs[] = {L.perm, L.label, L.rowptr, L.col, L.val, L.dinv, L.dtinv, L.F, L.X, L.Z, L.T, L.Wb,
                    L.r, L.rhat, L.p, L.v, L.s, L.t};
    for (void* p : ptrs) cudaFree(p);
}

// the pattern of level 0 (D on the plan's labels) from its neighbour table
gs_status level0_pattern(gs_ctx* c, const Plan* p, HostCsr& A) {
    const int64_t V = c->V;
    std::vector<int2> nb((size_t)V * 4);
    GS_CUDA(c, cudaMemcpyAsync(nb.data(), p->nbr, V * 4 * sizeof(int2), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    A.row.assign(V + 1, 0);
    A.col.clear();
    A.col.reserve(V * 9);
    for (int64_t i = 0; i < V; ++i) {
        int32_t cols[9];
        int k = 0;
        cols[k++] = (int32_t)i;
        for (int mu = 0; mu < 4; ++mu) {
            cols[k++] = nb[i * 4 + mu].x;
            cols[k++] = nb[i * 4 + mu].y;
        }
        std::sort(cols, cols + k);
        const int m = (int)(std::unique(cols, cols + k) - cols);
        A.col.insert(A.col.end(), cols, cols + m);
        A.row[i + 1] = (int32_t)A.col.size();
    }
    return GS_OK;
}

int64_t coarse_sites(const int d[4], int type, int dir, int out[4]) {
    for (int mu = 0; mu < 4; ++mu) out[mu] = d[mu];
    if (type == GS_TYPE_I)
        for (int mu = 0; mu < 4; ++mu) out[mu] = d[mu] / 2;
    else
        out[dir] = d[dir] / 2;
    return (int64_t)out[0] * out[1] * out[2] * out[3];
}

constexpr int64_t kMaxCoarsestSites = 1024;   // dense inverse of at most 12288 unknowns

gs_status vc_build(gs_vcycle* vc, int nsteps, const int* type, const int* dir, const int* inverse) {
    gs_ctx* c = vc->c;
    gs_status s;
    vc->nlev = nsteps + 1;
    vc->lev.resize(nsteps);
    int d[4] = {c->dims[0], c->dims[1], c->dims[2], c->dims[3]};
    HostCsr pat;   // pattern of the current level in its label order
    for (int l = 0; l < nsteps; ++l) {
        VLevel& L = vc->lev[l];
        L.type = type[l];
        L.dir = type[l] == GS_TYPE_II ? dir[l] : 0;
        L.inverse = inverse[l] ? 1 : 0;
        for (int mu = 0; mu < 4; ++mu) L.dims[mu] = d[mu];
        L.n = (int64_t)d[0] * d[1] * d[2] * d[3];
        if (l == 0) {
            if ((s = get_plan(c, L.type, L.dir, L.inverse, &L.plan)) != GS_OK) return s;
            L.nb = L.plan->nb;
            if ((s = level0_pattern(c, L.plan, pat)) != GS_OK) return s;
        }
        // (levels >= 1: n, nb, perm, label and the block-sparse operator were
        // made by the previous step)
        if ((s = alloc_level_work(c, L)) != GS_OK) return s;
        // the next level: its extents, its permutation (unless coarsest), its operator
        int dn[4];
        const int64_t nnext = coarse_sites(d, L.type, L.dir, dn);
        if (nnext != L.nb) return set_err(c, GS_EINVAL, "V-cycle: level %d's coarse set does not match its extents", l);
        HostCsr P;
        schur_pattern(pat, L.nb, vc->order, P);
        if (l > 0) {
            // this level's own d^-1 and d~^-1 for its S~
            const int64_t nr = L.n - L.nb;
            if ((s = vc_alloc(c, (void**)&L.dinv, nr * 144 * sizeof(double2))) != GS_OK) return s;
            if ((s = vc_alloc(c, (void**)&L.dtinv, nr * 144 * sizeof(double2))) != GS_OK) return s;
            k_rest_diag_rowsum<<<plain_blocks(c, nr * 144, 256), 256, 0, c->stream>>>(L.rowptr, L.col, L.val, L.nb,
                                                                                     nr, L.dinv, L.dtinv);
            c->launches++;
            int* flag = (int*)(c->scal_dev + 40);
            GS_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
            k_block_inverse<<<grid_for(nr, 64, c->num_sms * 8), 64, 0, c->stream>>>(L.dinv, nr, flag);
            k_block_inverse<<<grid_for(nr, 64, c->num_sms * 8), 64, 0, c->stream>>>(L.dtinv, nr, flag);
            c->launches += 2;
            int h = 0;
            GS_CUDA(c, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            GS_CUDA(c, cudaStreamSynchronize(c->stream));
            if (h) return set_err(c, GS_NONFINITE, "V-cycle: a 12 x 12 block of level %d's rest set is singular", l);
        }
        const bool last = (l == nsteps - 1);
        int ncol = 0;
        if (last) {
            if (nnext > kMaxCoarsestSites)
                return set_err(c, GS_ETOOLARGE,
                               "V-cycle: the coarsest level has %lld sites; its dense inverse takes at most %lld "
                               "(add a coarsening step)",
                               (long long)nnext, (long long)kMaxCoarsestSites);
            vc->nc = nnext;
            for (int mu = 0; mu < 4; ++mu) vc->coarse_dims[mu] = dn[mu];
            const int64_t N = nnext * 12;
            if ((s = vc_alloc(c, (void**)&vc->Ac, N * N * sizeof(double2))) != GS_OK) return s;
            if ((s = vc_alloc(c, (void**)&vc->Ainv, N * N * sizeof(double2))) != GS_OK) return s;
            GS_CUDA(c, cudaMemsetAsync(vc->Ac, 0, N * N * sizeof(double2), c->stream));
            if ((s = probe_next(vc, l, P, std::vector<int32_t>(), true, &ncol)) != GS_OK) return s;
        } else {
            VLevel& N = vc->lev[l + 1];
            for (int mu = 0; mu < 4; ++mu) N.dims[mu] = dn[mu];
            N.n = nnext;
            if ((s = vc_alloc(c, (void**)&N.perm, nnext * sizeof(int32_t))) != GS_OK) return s;
            if ((s = vc_alloc(c, (void**)&N.label, nnext * sizeof(int32_t))) != GS_OK) return s;
            const int ndir = type[l + 1] == GS_TYPE_II ? dir[l + 1] : 0;
            if ((s = build_labels(c, dn, type[l + 1], ndir, inverse[l + 1], N.perm, N.label, &N.nb)) != GS_OK)
                return s;
            std::vector<int32_t> lab(nnext), perm(nnext);
            GS_CUDA(c, cudaMemcpyAsync(lab.data(), N.label, nnext * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
            GS_CUDA(c, cudaMemcpyAsync(perm.data(), N.perm, nnext * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
            GS_CUDA(c, cudaStreamSynchronize(c->stream));
            // the next level's pattern in its label order
            N.pat.row.assign(nnext + 1, 0);
            N.pat.col.clear();
            std::vector<int32_t> cols;
            for (int64_t Li = 0; Li < nnext; ++Li) {
                const int32_t i = perm[Li];
                cols.clear();
                for (int32_t e = P.row[i]; e < P.row[i + 1]; ++e) cols.push_back(lab[P.col[e]]);
                std::sort(cols.begin(), cols.end());
                N.pat.col.insert(N.pat.col.end(), cols.begin(), cols.end());
                N.pat.row[Li + 1] = (int32_t)N.pat.col.size();
            }
            const int64_t nnzb = (int64_t)N.pat.col.size();
            if ((s = vc_alloc(c, (void**)&N.rowptr, (nnext + 1) * sizeof(int32_t))) != GS_OK) return s;
            if ((s = vc_alloc(c, (void**)&N.col, nnzb * sizeof(int32_t))) != GS_OK) return s;
            if ((s = vc_alloc(c, (void**)&N.val, nnzb * 144 * sizeof(double2))) != GS_OK) return s;
            GS_CUDA(c, cudaMemcpyAsync(N.rowptr, N.pat.row.data(), (nnext + 1) * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, c->stream));
            GS_CUDA(c, cudaMemcpyAsync(N.col, N.pat.col.data(), nnzb * sizeof(int32_t), cudaMemcpyHostToDevice,
                                       c->stream));
            GS_CUDA(c, cudaMemsetAsync(N.val, 0, nnzb * 144 * sizeof(double2), c->stream));
            if ((s = probe_next(vc, l, P, lab, false, &ncol)) != GS_OK) return s;
            pat = N.pat;
        }
        vc->colours[l] = ncol;
        for (int mu = 0; mu < 4; ++mu) d[mu] = dn[mu];
    }
    // the coarsest level: keep its operator, invert a copy
    const int64_t N = vc->nc * 12;
    GS_CUDA(c, cudaMemcpyAsync(vc->Ainv, vc->Ac, N * N * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    int32_t* piv = nullptr;
    double2* f = nullptr;
    if ((s = vc_alloc(c, (void**)&piv, N * sizeof(int32_t))) != GS_OK) return s;
    if ((s = vc_alloc(c, (void**)&f, N * sizeof(double2))) != GS_OK) {
        cudaFree(piv);
        return s;
    }
    int* flag = (int*)(c->scal_dev + 40);
    cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    const int ge = grid_for(N * N, 256, c->num_sms * 16);
    for (int64_t k = 0; k < N; ++k) {
        k_gj_pivot<<<1, kGjThreads, 0, c->stream>>>(vc->Ainv, N, k, piv, f, flag);
        k_gj_eliminate<<<ge, 256, 0, c->stream>>>(vc->Ainv, N, k, f);
    }
    k_gj_unscramble<<<grid_for(N, 128, c->num_sms * 4), 128, 0, c->stream>>>(vc->Ainv, N, piv);
    c->launches += 2 * N + 1;
    int h = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(piv);
    cudaFree(f);
    if (e != cudaSuccess) return set_err(c, GS_ECUDA, "V-cycle: coarsest inverse: %s", cudaGetErrorString(e));
    if (h) return set_err(c, GS_NONFINITE, "V-cycle: the coarsest operator is singular");
    return GS_OK;
}

void vc_free(gs_vcycle* vc) {
    for (VLevel& L : vc->lev) free_level(L);
    vc->lev.clear();
    void* ptrs[] = {vc->Ac, vc->Ainv, vc->r, vc->rhat, vc->p, vc->v, vc->s, vc->t, vc->ph, vc->sh, vc->dot_dev};
    for (void* p : ptrs) cudaFree(p);
    if (vc->dot_host) cudaFreeHost(vc->dot_host);
    cudaGetLastError();
}

void reset_rest_stats(gs_vcycle* vc) {
    vc->rest_solves = vc->rest_iters = vc->rest_unconverged = 0;
    vc->rest_max_seen = 0;
}

void rest_stats(const gs_vcycle* vc, gs_solve_stats& st) {
    st.inner_solves = (int)vc->rest_solves;
    st.inner_iters = vc->rest_iters;
    st.inner_max_seen = vc->rest_max_seen;
    st.lowp_fallbacks = vc->rest_unconverged;   // rest-set solves stopped at their limit
}

// y = D x on the full lattice, site order
gs_status apply_d(gs_ctx* c, const double2* x, double2* y) {
    const Plan* p = c->plans[0];
    StencilArgs a = stencil0(c, p);
    a.out = y;
    a.o0 = 0;
    a.n_out = c->V;
    a.inA = x;
    a.a0 = 0;
    a.a1 = c->V;
    a.b1 = c->V;
    return launch_stencil_f64(c, a);
}

gs_status ensure_outer_work(gs_vcycle* vc) {
    if (vc->r) return GS_OK;
    gs_ctx* c = vc->c;
    const size_t bytes = (size_t)c->V * kSiteC * sizeof(double2);
    double2** v[8] = {&vc->r, &vc->rhat, &vc->p, &vc->v, &vc->s, &vc->t, &vc->ph, &vc->sh};
    for (auto pp : v) {
        gs_status s = vc_alloc(c, (void**)pp, bytes);
        if (s != GS_OK) return s;
    }
    return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_vcycle_create(gs_ctx* c, int nsteps, const int* type, const int* dir, const int* inverse,
                           int order, double rest_tol, int rest_max_iter, gs_vcycle** out) {
    if (!c) return GS_EINVAL;
    if (!out) return set_err(c, GS_EINVAL, "null output");
    *out = nullptr;
    if (nsteps < 1 || nsteps > 6) return set_err(c, GS_EINVAL, "V-cycle: %d coarsening steps not in 1..6", nsteps);
    if (!type || !dir || !inverse) return set_err(c, GS_EINVAL, "V-cycle: null level description");
    if (order != 1 && order != 2) return set_err(c, GS_EINVAL, "V-cycle: approximation order %d is not 1 or 2", order);
    if (!(rest_tol > 0.0) || rest_tol >= 1.0) return set_err(c, GS_EINVAL, "V-cycle: rest tolerance must be in (0, 1)");
    if (rest_max_iter < 1) return set_err(c, GS_EINVAL, "V-cycle: rest iteration limit must be positive");
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    for (int l = 0; l < nsteps; ++l)
        if (type[l] != GS_TYPE_I && type[l] != GS_TYPE_II)
            return set_err(c, GS_EINVAL, "V-cycle: unknown permutation type %d at level %d", type[l], l);
    gs_vcycle* vc = new gs_vcycle();
    vc->c = c;
    vc->order = order;
    vc->rest_tol = rest_tol;
    vc->rest_maxit = rest_max_iter;
    gs_status s = vc_alloc(c, (void**)&vc->dot_dev, 4 * sizeof(double2));
    if (s == GS_OK && cudaHostAlloc((void**)&vc->dot_host, 4 * sizeof(double2), 0) != cudaSuccess) {
        cudaGetLastError();
        s = set_err(c, GS_ENOMEM, "V-cycle: pinned allocation failed");
    }
    if (s == GS_OK) s = vc_build(vc, nsteps, type, dir, inverse);
    if (s != GS_OK) {
        if (c->stream) cudaStreamSynchronize(c->stream);
        vc_free(vc);
        delete vc;
        return s;
    }
    *out = vc;
    return GS_OK;
}

gs_status gs_vcycle_destroy(gs_vcycle* vc) {
    if (!vc) return GS_OK;
    if (vc->c && vc->c->stream) cudaStreamSynchronize(vc->c->stream);
    else cudaDeviceSynchronize();
    vc_free(vc);
    delete vc;
    return GS_OK;
}

gs_status gs_vcycle_level(const gs_vcycle* vc, int level, int dims_out[4], int64_t* sites, int64_t* blocks,
                          int* colours) {
    if (!vc || level < 0 || level >= vc->nlev) return GS_EINVAL;
    if (level == vc->nlev - 1) {
        if (dims_out)
            for (int mu = 0; mu < 4; ++mu) dims_out[mu] = vc->coarse_dims[mu];
        if (sites) *sites = vc->nc;
        if (blocks) *blocks = vc->nc * vc->nc;
        if (colours) *colours = 0;
        return GS_OK;
    }
    const VLevel& L = vc->lev[level];
    if (dims_out)
        for (int mu = 0; mu < 4; ++mu) dims_out[mu] = L.dims[mu];
    if (sites) *sites = L.n;
    if (blocks) *blocks = level == 0 ? 0 : (int64_t)L.pat.col.size();
    if (colours) *colours = vc->colours[level];
    return GS_OK;
}

gs_status gs_vcycle_operator_apply(gs_vcycle* vc, int level, const void* x_dev, void* y_dev) {
    if (!vc) return GS_EINVAL;
    gs_ctx* c = vc->c;
    if (level < 1 || level >= vc->nlev) return set_err(c, GS_EINVAL, "V-cycle: level %d not in 1..%d", level, vc->nlev - 1);
    if (!x_dev || !y_dev) return set_err(c, GS_EINVAL, "null vector");
    if (level == vc->nlev - 1) {
        const int64_t N = vc->nc * 12;
        k_dense_gemv<<<grid_for(N, 8, c->num_sms * 32), 256, 0, c->stream>>>(vc->Ac, (const double2*)x_dev,
                                                                            (double2*)y_dev, N);
        c->launches++;
        GS_CHECK_LAUNCH(c);
        return GS_OK;
    }
    VLevel& L = vc->lev[level];
    gs_status s;
    // y = P^T B (P x) in the level's natural order
    if ((s = launch_gather(c, L.perm, (const double2*)x_dev, L.F, L.n)) != GS_OK) return s;
    BsrArgs a = bsr_args(L);
    a.out = L.X;
    a.o0 = 0;
    a.n_out = L.n;
    a.inA = L.F;
    a.a0 = 0;
    a.a1 = L.n;
    a.b1 = L.n;
    if ((s = bsr_launch(c, a)) != GS_OK) return s;
    return launch_scatter(c, L.perm, L.X, (double2*)y_dev, L.n);
}

gs_status gs_vcycle_apply(gs_vcycle* vc, const void* f_dev, void* x_dev, gs_solve_stats* stats) {
    if (!vc) return GS_EINVAL;
    gs_ctx* c = vc->c;
    if (!f_dev || !x_dev) return set_err(c, GS_EINVAL, "null vector");
    gs_solve_stats st;
    memset(&st, 0, sizeof st);
    const long long l0 = c->launches;
    reset_rest_stats(vc);
    gs_status s = vc_apply(vc, 0, (const double2*)f_dev, (double2*)x_dev);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess && s == GS_OK) s = set_err(c, GS_ECUDA, "gs_vcycle_apply: %s", cudaGetErrorString(e));
    rest_stats(vc, st);
    st.status = s;
    st.kernel_launches = c->launches - l0;
    if (stats) *stats = st;
    return s;
}

gs_status gs_solve_bicgstab(gs_ctx* c, gs_vcycle* vc, const void* f_dev, void* x_dev, double tol, int max_iter,
                            gs_solve_stats* stats, double* rate_out, double* history, int history_cap) {
    if (!c) return GS_EINVAL;
    if (!f_dev || !x_dev) return set_err(c, GS_EINVAL, "null vector");
    if (!(tol > 0.0) || max_iter < 0) return set_err(c, GS_EINVAL, "bad tolerance or iteration limit");
    if (vc && vc->c != c) return set_err(c, GS_EINVAL, "the V-cycle belongs to another context");
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    gs_vcycle tmp;                       // plain solve: workspace of its own
    gs_vcycle* w = vc ? vc : &tmp;
    tmp.c = c;
    gs_solve_stats st;
    memset(&st, 0, sizeof st);
    const long long l0 = c->launches;
    std::vector<double> hist;
    gs_status s = GS_OK;
    auto run = [&]() -> gs_status {
        gs_status e;
        if (!w->dot_dev) {
            if ((e = vc_alloc(c, (void**)&w->dot_dev, 4 * sizeof(double2))) != GS_OK) return e;
            if (cudaHostAlloc((void**)&w->dot_host, 4 * sizeof(double2), 0) != cudaSuccess) {
                cudaGetLastError();
                return set_err(c, GS_ENOMEM, "pinned allocation failed");
            }
        }
        if ((e = ensure_outer_work(w)) != GS_OK) return e;
        if (vc) reset_rest_stats(vc);
        const int64_t n = c->V * kSiteC;
        const size_t bytes = (size_t)n * sizeof(double2);
        const double2* f = (const double2*)f_dev;
        double2* x = (double2*)x_dev;
        GS_CUDA(c, cudaMemsetAsync(x, 0, bytes, c->stream));
        double fnorm;
        if ((e = vc_norm(w, f, n, &fnorm)) != GS_OK) return e;
        if (!isfinite(fnorm)) return set_err(c, GS_NONFINITE, "non-finite right-hand side");
        hist.push_back(fnorm);
        if (fnorm == 0.0) return GS_OK;
        const double target = tol * fnorm;
        GS_CUDA(c, cudaMemcpyAsync(w->r, f, bytes, cudaMemcpyDeviceToDevice, c->stream));
        GS_CUDA(c, cudaMemcpyAsync(w->rhat, f, bytes, cudaMemcpyDeviceToDevice, c->stream));
        GS_CUDA(c, cudaMemsetAsync(w->p, 0, bytes, c->stream));
        GS_CUDA(c, cudaMemsetAsync(w->v, 0, bytes, c->stream));
        cplx rho_old = 1.0, alpha = 1.0, omega = 1.0;
        bool conv = false;
        int it = 0;
        while (!conv && it < max_iter) {
            ++it;
            cplx rho;
            if ((e = vc_dot(w, w->rhat, w->r, n, &rho)) != GS_OK) return e;
            if (rho == 0.0) return set_err(c, GS_BREAKDOWN, "BiCGStab breakdown (rho = 0) at step %d", it);
            const cplx beta = (rho / rho_old) * (alpha / omega);
            if ((e = axpby(c, -omega, w->v, 1.0, w->p, n)) != GS_OK) return e;
            if ((e = axpby(c, 1.0, w->r, beta, w->p, n)) != GS_OK) return e;
            const double2* ph = w->p;
            if (vc) {
                if ((e = vc_apply(vc, 0, w->p, w->ph)) != GS_OK) return e;
                ph = w->ph;
            }
            if ((e = apply_d(c, ph, w->v)) != GS_OK) return e;
            cplx rv;
            if ((e = vc_dot(w, w->rhat, w->v, n, &rv)) != GS_OK) return e;
            alpha = rho / rv;
            GS_CUDA(c, cudaMemcpyAsync(w->s, w->r, bytes, cudaMemcpyDeviceToDevice, c->stream));
            if ((e = axpby(c, -alpha, w->v, 1.0, w->s, n)) != GS_OK) return e;
            double sn;
            if ((e = vc_norm(w, w->s, n, &sn)) != GS_OK) return e;
            if (!isfinite(sn)) return set_err(c, GS_NONFINITE, "non-finite BiCGStab residual");
            if (sn <= target) {
                if ((e = axpby(c, alpha, ph, 1.0, x, n)) != GS_OK) return e;
                hist.push_back(sn);
                conv = true;
                break;
            }
            const double2* sh = w->s;
            if (vc) {
                if ((e = vc_apply(vc, 0, w->s, w->sh)) != GS_OK) return e;
                sh = w->sh;
            }
            if ((e = apply_d(c, sh, w->t)) != GS_OK) return e;
            cplx ts, tt;
            if ((e = vc_dot(w, w->t, w->s, n, &ts)) != GS_OK) return e;
            if ((e = vc_dot(w, w->t, w->t, n, &tt)) != GS_OK) return e;
            omega = tt.real() > 0.0 ? ts / tt : cplx(0.0);
            if ((e = axpby(c, alpha, ph, 1.0, x, n)) != GS_OK) return e;
            if ((e = axpby(c, omega, sh, 1.0, x, n)) != GS_OK) return e;
            GS_CUDA(c, cudaMemcpyAsync(w->r, w->s, bytes, cudaMemcpyDeviceToDevice, c->stream));
            if ((e = axpby(c, -omega, w->t, 1.0, w->r, n)) != GS_OK) return e;
            rho_old = rho;
            double rn;
            if ((e = vc_norm(w, w->r, n, &rn)) != GS_OK) return e;
            if (!isfinite(rn)) return set_err(c, GS_NONFINITE, "non-finite BiCGStab residual");
            hist.push_back(rn);
            conv = rn <= target;
            if (omega == 0.0 && !conv) return set_err(c, GS_BREAKDOWN, "BiCGStab breakdown (omega = 0) at step %d", it);
        }
        st.outer_iters = it;
        // the true residual of the returned x
        if ((e = apply_d(c, x, w->t)) != GS_OK) return e;
        GS_CUDA(c, cudaMemcpyAsync(w->s, f, bytes, cudaMemcpyDeviceToDevice, c->stream));
        if ((e = axpby(c, -1.0, w->t, 1.0, w->s, n)) != GS_OK) return e;
        double tr;
        if ((e = vc_norm(w, w->s, n, &tr)) != GS_OK) return e;
        st.true_residual = tr / fnorm;
        st.outer_residual = hist.back() / fnorm;
        if (!conv) return set_err(c, GS_MAXITER, "BiCGStab reached %d steps (residual %.3e)", it, st.outer_residual);
        return GS_OK;
    };
    s = run();
    if (vc) rest_stats(vc, st);
    st.status = s;
    st.kernel_launches = c->launches - l0;
    if (stats) *stats = st;
    if (rate_out) {
        // Section 4's average convergence rate: (||r_n|| / ||r_0||)^(1/n)
        double R = 0.0;
        if (hist.size() >= 2 && hist.front() > 0.0 && hist.back() > 0.0)
            R = pow(hist.back() / hist.front(), 1.0 / (double)(hist.size() - 1));
        *rate_out = R;
    }
    if (history)
        for (int k = 0; k < history_cap; ++k) history[k] = k < (int)hist.size() ? hist[k] : -1.0;
    if (!vc) {
        if (c->stream) cudaStreamSynchronize(c->stream);
        void* ptrs[] = {tmp.r, tmp.rhat, tmp.p, tmp.v, tmp.s, tmp.t, tmp.ph, tmp.sh, tmp.dot_dev};
        for (void* p : ptrs) cudaFree(p);
        if (tmp.dot_host) cudaFreeHost(tmp.dot_host);
        tmp.r = tmp.rhat = tmp.p = tmp.v = tmp.s = tmp.t = tmp.ph = tmp.sh = tmp.dot_dev = tmp.dot_host = nullptr;
    }
    return s;
}

}  // extern "C"
