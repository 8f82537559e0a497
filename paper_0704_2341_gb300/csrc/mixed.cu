// Mixed-precision inner solve of D_rr z = t.
//
// FP64 defect correction around a low-precision BiCGStab:
//   z = 0, r = t;  repeat { solve D_rr e = r / ||r|| approximately in FP32
//   arithmetic with FP32 or BF16 storage;  z += ||r|| e;  r = t - D_rr z in
//   FP64 }  until ||r|| <= tol ||t||.
// The true residual is recomputed with the FP64 stencil every cycle, so the
// result meets the same FP64 tolerance as the plain solve; the low-precision
// solve only has to reduce the residual by a few digits per cycle.  If a
// cycle stops making progress, the remaining correction is computed by the
// plain FP64 BiCGStab (the fallback, and the arbiter of the result).
//
// Low-precision layouts (compact rest-set index k = label - n_b):
//   spinors: SoA of 16-byte vectors, component-major: FP32 -> 6 float4 per
//            site ([6][n]), BF16 -> 3 x (8 bf16) per site ([3][n]);
//   links:   two rows of -1/2 U (12 reals), the third row rebuilt as
//            -2 conj(row0 x row1) (SU(3)); FP32 -> 3 float4 ([mu][3][n]),
//            BF16 -> 3 x (4 bf16) ([mu][3][n]);
//   neighbours: int2 [n][mu] compact indices, -1 for a neighbour outside r.
// One thread per site accumulates all eight hops in FP32 registers; the
// kernel is HBM bound (384 B/site FP32, 192 B/site BF16 algorithmic).
#include "lowp.cuh"

namespace gs {
namespace {
// ---------------------------------------------------------------------------
// low-precision BiCGStab vector kernels (thread per site)
// ---------------------------------------------------------------------------

// r = rhat = p = scale * r64 (AoS FP64 -> SoA S), x = 0, rho = ||r||^2.
template <class S>
__global__ void k_lp_init(const double2* __restrict__ r64, const double* __restrict__ rr64,
                          void* r, void* rhat, void* p, void* x, int64_t n, float tol,
                          LpState* st, float* partial, unsigned int* counter) {
    const double nrm2 = *rr64;
    const float scale = nrm2 > 0.0 ? (float)(1.0 / sqrt(nrm2)) : 0.f;
    float acc[1] = {0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[24], z[24];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const double2 v = r64[k * 12 + q];
            f[2 * q] = (float)v.x * scale;
            f[2 * q + 1] = (float)v.y * scale;
            z[2 * q] = z[2 * q + 1] = 0.f;
        }
        Store<S>::store_spinor(r, n, k, f);
        Store<S>::store_spinor(rhat, n, k, f);
        Store<S>::store_spinor(p, n, k, f);
        Store<S>::store_spinor(x, n, k, z);
        // norms of the stored (rounded) values
        Store<S>::load_spinor(r, n, k, f);
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[0] = fmaf(f[q], f[q], acc[0]);
    }
    float tot[1];
    if (lp_reduce_last<1>(acc, partial, counter, tot) && threadIdx.x == 0) {
        st->bb = tot[0];
        st->rr = tot[0];
        st->rho = make_float2(tot[0], 0.f);
        st->alpha = st->omega = st->beta = make_float2(0.f, 0.f);
        st->tol2 = tol * tol * tot[0];
        st->iter = 0;
        st->status = isfinite(tot[0]) ? GS_OK : GS_NONFINITE;
        st->done = (tot[0] == 0.f || !isfinite(tot[0])) ? 1 : 0;
        lp_publish(st);
    }
}

// s = r - alpha v ; x += alpha p ; ||s||^2
template <class S>
__global__ void k_lp_s(const void* r, const void* v, const void* p, void* s, void* x, int64_t n,
                       LpState* st, float* partial, unsigned int* counter) {
    if (st->done) return;
    const float2 al = st->alpha;
    float acc[1] = {0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float fr[24], fv[24], fp[24], fx[24];
        Store<S>::load_spinor(r, n, k, fr);
        Store<S>::load_spinor(v, n, k, fv);
        Store<S>::load_spinor(p, n, k, fp);
        Store<S>::load_spinor(x, n, k, fx);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float vr = fv[2 * q], vi = fv[2 * q + 1];
            fr[2 * q] -= al.x * vr - al.y * vi;
            fr[2 * q + 1] -= al.x * vi + al.y * vr;
            const float pr = fp[2 * q], pi = fp[2 * q + 1];
            fx[2 * q] = fmaf(al.x, pr, fmaf(-al.y, pi, fx[2 * q]));
            fx[2 * q + 1] = fmaf(al.x, pi, fmaf(al.y, pr, fx[2 * q + 1]));
        }
        Store<S>::store_spinor(s, n, k, fr);
        Store<S>::store_spinor(x, n, k, fx);
#pragma unroll
        for (int q = 0; q < 24; ++q) acc[0] = fmaf(fr[q], fr[q], acc[0]);
    }
    float tot[1];
    if (lp_reduce_last<1>(acc, partial, counter, tot) && threadIdx.x == 0) {
        if (!isfinite(tot[0])) {
            st->status = GS_NONFINITE;
            st->done = 1;
        } else if (tot[0] <= st->tol2) {
            st->rr = tot[0];
            st->iter += 1;
            st->done = 1;
        }
        if (st->done) lp_publish(st);
    }
}

// x += omega s ; r = s - omega t ; rho' = <rhat, r> ; ||r||^2 ; beta
template <class S>
__global__ void k_lp_xr(const void* s, const void* t, const void* rhat, void* x, void* r,
                        int64_t n, LpState* st, float* partial, unsigned int* counter) {
    if (st->done) return;
    const float2 om = st->omega;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float fs[24], ft[24], fh[24], fx[24];
        Store<S>::load_spinor(s, n, k, fs);
        Store<S>::load_spinor(t, n, k, ft);
        Store<S>::load_spinor(rhat, n, k, fh);
        Store<S>::load_spinor(x, n, k, fx);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float sr = fs[2 * q], si = fs[2 * q + 1];
            fx[2 * q] = fmaf(om.x, sr, fmaf(-om.y, si, fx[2 * q]));
            fx[2 * q + 1] = fmaf(om.x, si, fmaf(om.y, sr, fx[2 * q + 1]));
            const float tr = ft[2 * q], ti = ft[2 * q + 1];
            const float rr = sr - (om.x * tr - om.y * ti);
            const float ri = si - (om.x * ti + om.y * tr);
            fs[2 * q] = rr;
            fs[2 * q + 1] = ri;
            acc[0] = fmaf(fh[2 * q], rr, fmaf(fh[2 * q + 1], ri, acc[0]));
            acc[1] = fmaf(fh[2 * q], ri, fmaf(-fh[2 * q + 1], rr, acc[1]));
            acc[2] = fmaf(rr, rr, fmaf(ri, ri, acc[2]));
        }
        Store<S>::store_spinor(x, n, k, fx);
        Store<S>::store_spinor(r, n, k, fs);
    }
    float tot[3];
    if (lp_reduce_last<3>(acc, partial, counter, tot) && threadIdx.x == 0) {
        const float2 rho_new = make_float2(tot[0], tot[1]);
        st->rr = tot[2];
        st->iter += 1;
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
            st->status = GS_NONFINITE;
            st->done = 1;
        } else if (tot[2] <= st->tol2) {
            st->done = 1;
        } else if ((om.x == 0.f && om.y == 0.f) || (rho_new.x == 0.f && rho_new.y == 0.f)) {
            st->status = GS_BREAKDOWN;
            st->done = 1;
        } else {
            st->beta = cmulf2(cdivf_(rho_new, st->rho), cdivf_(st->alpha, om));
            st->rho = rho_new;
        }
        lp_publish(st);
    }
}

// p = r + beta (p - omega v)
template <class S>
__global__ void k_lp_p(const void* r, const void* v, void* p, int64_t n, const LpState* st) {
    if (st->done) return;
    const float2 be = st->beta, om = st->omega;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float fr[24], fv[24], fp[24];
        Store<S>::load_spinor(r, n, k, fr);
        Store<S>::load_spinor(v, n, k, fv);
        Store<S>::load_spinor(p, n, k, fp);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float vr = fv[2 * q], vi = fv[2 * q + 1];
            const float qr = fp[2 * q] - (om.x * vr - om.y * vi);
            const float qi = fp[2 * q + 1] - (om.x * vi + om.y * vr);
            fp[2 * q] = fmaf(be.x, qr, fmaf(-be.y, qi, fr[2 * q]));
            fp[2 * q + 1] = fmaf(be.x, qi, fmaf(be.y, qr, fr[2 * q + 1]));
        }
        Store<S>::store_spinor(p, n, k, fp);
    }
}

// z64 += sqrt(rr64) * e   (undo the normalisation of the cycle's right-hand side)
template <class S>
__global__ void k_lp_accum(const void* e, const double* __restrict__ rr64, double2* z64,
                           int64_t n) {
    const double scale = sqrt(*rr64);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[24];
        Store<S>::load_spinor(e, n, k, f);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            double2 z = z64[k * 12 + q];
            z.x = fma(scale, (double)f[2 * q], z.x);
            z.y = fma(scale, (double)f[2 * q + 1], z.y);
            z64[k * 12 + q] = z;
        }
    }
}

// complex128 AoS (n sites) <-> low-precision SoA
template <class S>
__global__ void k_lp_pack(const double2* __restrict__ x, void* y, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[24];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const double2 v = x[k * 12 + q];
            f[2 * q] = (float)v.x;
            f[2 * q + 1] = (float)v.y;
        }
        Store<S>::store_spinor(y, n, k, f);
    }
}

template <class S>
__global__ void k_lp_unpack(const void* x, double2* __restrict__ y, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[24];
        Store<S>::load_spinor(x, n, k, f);
#pragma unroll
        for (int q = 0; q < 12; ++q) y[k * 12 + q] = make_double2((double)f[2 * q], (double)f[2 * q + 1]);
    }
}

// compact rest-set neighbour table and low-precision links from a plan
template <class S>
__global__ void k_lp_tables(int64_t nb, int64_t n, const int2* __restrict__ nbr,
                            const double2* __restrict__ links64, int2* __restrict__ nbr_r,
                            void* links_lp) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = nb + k;
        for (int mu = 0; mu < 4; ++mu) {
            const int2 q = nbr[j * 4 + mu];
            nbr_r[k * 4 + mu] = make_int2(q.x >= nb ? (int)(q.x - nb) : -1,
                                          q.y >= nb ? (int)(q.y - nb) : -1);
            float f[12];
            const double2* u = links64 + (j * 4 + mu) * 9;  // rows 0 and 1
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                f[2 * c] = (float)u[c].x;
                f[2 * c + 1] = (float)u[c].y;
            }
            Store<S>::store_link(links_lp, n, mu, k, f);
        }
    }
}

int lp_block(int64_t n, int sms) {
    if (n >= (int64_t)sms * 4 * 128) return 128;
    if (n >= (int64_t)sms * 2 * 64) return 64;
    return 32;
}

// Launch the low-precision stencil (variant 1: thread per site; 2: warp per
// direction); with profiling on, bracket it by events and count its
// algorithmic work (168 flop per in-set hop + 48 per site; bytes: spinor in +
// out, one 12-real link per link used, each datum once).
template <class S>
gs_status launch_lp_stencil(gs_ctx* c, LpArgs a, long long hops, int variant, long long* launches) {
    int slot = -1;
    a.ran = nullptr;
    if (c->prof.on) {
        gs_status s = prof_begin(c, &slot);
        if (s != GS_OK) return s;
        a.ran = c->prof.ran_dev + slot;
    }
    if (variant == 2) {
        int64_t g = (a.n + kLpSites - 1) / kLpSites;
        if (a.epi != EPI_NONE && g > kMaxRedBlocks) g = kMaxRedBlocks;
        switch (a.epi) {
            case EPI_NONE: k_dslash_lp_dir<S, EPI_NONE><<<(int)g, kLpThreads, 0, c->stream>>>(a); break;
            case EPI_DOT_RHAT_V: k_dslash_lp_dir<S, EPI_DOT_RHAT_V><<<(int)g, kLpThreads, 0, c->stream>>>(a); break;
            default: k_dslash_lp_dir<S, EPI_DOT_TS><<<(int)g, kLpThreads, 0, c->stream>>>(a); break;
        }
    } else {
        // variants 1, 3, 4: thread per site with a register budget for
        // 4, 6 or 8 blocks of 128 threads per SM; 5, 6: the same with the
        // next direction's loads in flight (budget for 3 or 4 blocks)
        const int b = lp_block(a.n, c->num_sms);
        int64_t g = (a.n + b - 1) / b;
        if (a.epi != EPI_NONE && g > kMaxRedBlocks) g = kMaxRedBlocks;
#define GS_SITE_LAUNCH(MB)                                                                       \
        switch (a.epi) {                                                                         \
            case EPI_NONE: k_dslash_lp_site<S, EPI_NONE, MB><<<(int)g, b, 0, c->stream>>>(a); break; \
            case EPI_DOT_RHAT_V:                                                                 \
                k_dslash_lp_site<S, EPI_DOT_RHAT_V, MB><<<(int)g, b, 0, c->stream>>>(a); break;  \
            default: k_dslash_lp_site<S, EPI_DOT_TS, MB><<<(int)g, b, 0, c->stream>>>(a); break; \
        }
#define GS_PIPE_LAUNCH(MB)                                                                       \
        switch (a.epi) {                                                                         \
            case EPI_NONE: k_dslash_lp_pipe<S, EPI_NONE, MB><<<(int)g, b, 0, c->stream>>>(a); break; \
            case EPI_DOT_RHAT_V:                                                                 \
                k_dslash_lp_pipe<S, EPI_DOT_RHAT_V, MB><<<(int)g, b, 0, c->stream>>>(a); break;  \
            default: k_dslash_lp_pipe<S, EPI_DOT_TS, MB><<<(int)g, b, 0, c->stream>>>(a); break; \
        }
        if (variant == 3) {
            GS_SITE_LAUNCH(6)
        } else if (variant == 4) {
            GS_SITE_LAUNCH(8)
        } else if (variant == 5) {
            GS_PIPE_LAUNCH(3)
        } else if (variant == 6) {
            GS_PIPE_LAUNCH(4)
        } else {
            GS_SITE_LAUNCH(4)
        }
#undef GS_SITE_LAUNCH
#undef GS_PIPE_LAUNCH
    }
    ++*launches;
    GS_CHECK_LAUNCH(c);
    if (slot >= 0) {
        const double sb = (double)Store<S>::spinor_bytes, lb = (double)Store<S>::link_bytes;
        const int prec = sizeof(S) == 4 ? GS_F32 : GS_BF16;
        return prof_end_work(c, slot, prec, a.n, hops, 168.0 * hops + 48.0 * a.n,
                             2.0 * sb * a.n + lb * 0.5 * hops);
    }
    return GS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct LpWork {
    int prec = -1;
    int64_t cap = 0;
    void *x = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr,
         *t = nullptr;
    LpState* st = nullptr;
    float* partial = nullptr;
    unsigned int* counter = nullptr;
    double* rr64 = nullptr;       // device ||r||^2 of the current FP64 residual
    double* rr64_host = nullptr;  // pinned
};

struct LpPlanData {
    const Plan* plan = nullptr;
    int prec = -1;
    int64_t nb = 0;        // labels below nb are excluded (0 for the full lattice)
    int64_t n = 0;         // sites of the set
    long long hops = 0;    // in-set neighbour terms of one D application
    int variant = 0;       // stencil variant: 1/3/4 = thread per site (register budget for
                           // 4/6/8 blocks per SM), 2 = warp per direction, 5/6 = thread per
                           // site with the next direction's loads in flight (3/4 blocks)
    int2* nbr_r = nullptr;
    void* links = nullptr;
    LexDims lex{};         // the whole lattice: neighbours by arithmetic (identity plan)
};

static size_t spinor_bytes(int prec) { return prec == GS_BF16 ? 48 : 96; }
static gs_status ensure_lp(gs_ctx* c, int prec, int64_t n);
static size_t link_bytes(int prec) { return prec == GS_BF16 ? 24 : 48; }

}  // namespace gs
namespace gs {
gs_status persistent_bicg_lp(gs_ctx* c, int prec, const LpArgs& A, const LpArgs& C,
                             const double2* r64, const double* rr64, void* const* vecs, LpState* st,
                             int64_t n, float tol, int maxit);

struct MixedState {
    LpWork w;
    std::vector<LpPlanData> plans;
    double2* e64 = nullptr;  // FP64 correction of the fallback solve (rest set)
    int64_t e64_cap = 0;
    double2* zbak = nullptr; // z before a low-precision cycle's correction (restored if it fails)
    int64_t zbak_cap = 0;
};

static MixedState* mixed_of(gs_ctx* c) {
    if (!c->mixed) c->mixed = new MixedState();
    return (MixedState*)c->mixed;
}

void free_mixed(gs_ctx* c) {
    MixedState* m = (MixedState*)c->mixed;
    if (!m) return;
    void* bufs[] = {m->w.x, m->w.r, m->w.rhat, m->w.p, m->w.v, m->w.s, m->w.t};
    for (void* b : bufs) cudaFree(b);
    cudaFree(m->w.st);
    cudaFree(m->w.partial);
    cudaFree(m->w.counter);
    cudaFree(m->w.rr64);
    cudaFree(m->e64);
    cudaFree(m->zbak);
    if (m->w.rr64_host) cudaFreeHost(m->w.rr64_host);
    for (auto& pd : m->plans) {
        cudaFree(pd.nbr_r);
        cudaFree(pd.links);
    }
    delete m;
    c->mixed = nullptr;
}

static gs_status ensure_lp(gs_ctx* c, int prec, int64_t n) {
    MixedState* m = mixed_of(c);
    LpWork& w = m->w;
    if (w.st == nullptr) {
        if (cudaMalloc(&w.st, sizeof(LpState)) != cudaSuccess ||
            cudaMalloc(&w.partial, kMaxRedBlocks * kMaxRedVals * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&w.counter, sizeof(unsigned int)) != cudaSuccess ||
            cudaMalloc(&w.rr64, sizeof(double)) != cudaSuccess ||
            cudaHostAlloc(&w.rr64_host, sizeof(double), 0) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GS_ENOMEM, "allocating the mixed-precision state failed");
        }
        GS_CUDA(c, cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), c->stream));
        // the low-precision state publishes through the inner solver's mapped mirror
        gs_status s = ensure_inner(c, 1);
        if (s != GS_OK) return s;
        LpState init;
        memset(&init, 0, sizeof init);
        init.pub = c->inner.pub_dev;
        GS_CUDA(c, cudaMemcpyAsync(w.st, &init, sizeof init, cudaMemcpyHostToDevice, c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    const size_t need = (size_t)n * spinor_bytes(prec);
    if (w.cap < (int64_t)need) {
        void** bufs[] = {&w.x, &w.r, &w.rhat, &w.p, &w.v, &w.s, &w.t};
        for (void** b : bufs) {
            cudaFree(*b);
            *b = nullptr;
        }
        for (void** b : bufs)
            if (cudaMalloc(b, need) != cudaSuccess) {
                cudaGetLastError();
                return set_err(c, GS_ENOMEM, "allocating low-precision vectors failed");
            }
        w.cap = (int64_t)need;
    }
    return GS_OK;
}

// The autotuner: time every stencil variant on this set (2 warm-up and 5
// timed launches each, CUDA events, zeroed operands) and keep the fastest;
// a variant forced with gs_set_option skips the timing.
static gs_status lp_tune(gs_ctx* c, LpPlanData& pd) {
    if (c->opt_stencil_variant != 0) {
        pd.variant = c->opt_stencil_variant;
        return GS_OK;
    }
    gs_status s = ensure_lp(c, pd.prec, pd.n);
    if (s != GS_OK) return s;
    MixedState* m = mixed_of(c);
    const size_t bytes = (size_t)pd.n * spinor_bytes(pd.prec);
    GS_CUDA(c, cudaMemsetAsync(m->w.p, 0, bytes, c->stream));
    LpArgs a;
    memset(&a, 0, sizeof a);
    a.out = m->w.v;
    a.in = m->w.p;
    a.links = pd.links;
    a.nbr = pd.nbr_r;
    a.lex = pd.lex;
    a.n = pd.n;
    a.diag = (float)(c->m0 + 4.0);
    a.epi = EPI_NONE;
    cudaEvent_t e0, e1;
    GS_CUDA(c, cudaEventCreate(&e0));
    GS_CUDA(c, cudaEventCreate(&e1));
    float best = 0.f;
    const bool was_on = c->prof.on;
    c->prof.on = false;
    for (int v = 1; v <= 6; ++v) {
        long long l = 0;
        for (int r = 0; r < 7; ++r) {
            if (r == 2) GS_CUDA(c, cudaEventRecord(e0, c->stream));
            s = (pd.prec == GS_BF16) ? launch_lp_stencil<__nv_bfloat16>(c, a, pd.hops, v, &l)
                                     : launch_lp_stencil<float>(c, a, pd.hops, v, &l);
            if (s != GS_OK) break;
        }
        c->launches += l;
        if (s != GS_OK) break;
        GS_CUDA(c, cudaEventRecord(e1, c->stream));
        GS_CUDA(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        GS_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        if (v == 1 || ms < best) {
            best = ms;
            pd.variant = v;
        }
    }
    c->prof.on = was_on;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tuned_variant = pd.variant;
    return s;
}

// neighbour arithmetic of the whole lattice (LexDims): extents and the
// multiply-high constants of L0, L1, L2
static LexDims lex_dims(const int dims[4]) {
    LexDims d;
    memset(&d, 0, sizeof d);
    d.on = 1;
    for (int mu = 0; mu < 4; ++mu) d.L[mu] = dims[mu];
    for (int i = 0; i < 3; ++i) {
        const unsigned long long L = (unsigned long long)dims[i];
        int l = 0;
        while ((1ull << l) < L) ++l;
        d.sh[i] = l;
        d.mag[i] = (unsigned)((((1ull << 32) * ((1ull << l) - L)) / L) + 1ull);
    }
    return d;
}

static gs_status lp_plan(gs_ctx* c, const Plan* p, int prec, LpPlanData** out) {
    MixedState* m = mixed_of(c);
    for (auto& pd : m->plans)
        if (pd.plan == p && pd.prec == prec) {
            *out = &pd;
            return GS_OK;
        }
    LpPlanData pd;
    pd.plan = p;
    pd.prec = prec;
    // the identity plan stands for the whole lattice; a permutation for its rest set
    pd.nb = (p->type == 0) ? 0 : p->nb;
    pd.n = c->V - pd.nb;
    pd.hops = (p->type == 0) ? p->hops[0][0] : p->hops[1][1];
    if (p->type == 0) pd.lex = lex_dims(c->dims);
    const int64_t n = pd.n;
    if (cudaMalloc(&pd.nbr_r, (size_t)n * 4 * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&pd.links, (size_t)n * 4 * link_bytes(prec)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, GS_ENOMEM, "allocating low-precision links failed");
    }
    const int g = grid_for(n, 256, c->num_sms * 8);
    if (prec == GS_BF16)
        k_lp_tables<__nv_bfloat16><<<g, 256, 0, c->stream>>>(pd.nb, n, p->nbr, p->links, pd.nbr_r,
                                                             pd.links);
    else
        k_lp_tables<float><<<g, 256, 0, c->stream>>>(pd.nb, n, p->nbr, p->links, pd.nbr_r, pd.links);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    gs_status s = lp_tune(c, pd);
    if (s != GS_OK) return s;
    m->plans.push_back(pd);
    *out = &m->plans.back();
    return GS_OK;
}

gs_status lowp_tables(gs_ctx* c, const Plan* p, int prec, LowpTables* out) {
    gs_status s = ensure_lp(c, prec, c->V - ((p->type == 0) ? 0 : p->nb));
    if (s != GS_OK) return s;
    LpPlanData* pd = nullptr;
    if ((s = lp_plan(c, p, prec, &pd)) != GS_OK) return s;
    out->nbr = pd->nbr_r;
    out->links = pd->links;
    out->n = pd->n;
    out->nb = pd->nb;
    out->hops = pd->hops;
    return GS_OK;
}

void invalidate_mixed_links(gs_ctx* c) {
    MixedState* m = (MixedState*)c->mixed;
    if (!m) return;
    for (auto& pd : m->plans) {
        cudaFree(pd.nbr_r);
        cudaFree(pd.links);
    }
    m->plans.clear();
}

template <class S>
static gs_status lp_bicgstab(gs_ctx* c, LpPlanData* pd, int64_t n, float tol, int maxit,
                             int depth, int* iters_out, int* status_out) {
    MixedState* m = mixed_of(c);
    LpWork& w = m->w;
    const int bb = kLpRed;
    int gr = grid_for(n, bb, c->num_sms * 4 < kMaxRedBlocks ? c->num_sms * 4 : kMaxRedBlocks);
    int gp = grid_for(n, bb, c->num_sms * 16);
    LpArgs k1;
    memset(&k1, 0, sizeof k1);
    k1.out = w.v;
    k1.in = w.p;
    k1.links = pd->links;
    k1.nbr = pd->nbr_r;
    k1.lex = pd->lex;
    k1.n = n;
    k1.diag = (float)(c->m0 + 4.0);
    k1.epi = EPI_DOT_RHAT_V;
    k1.epi_vec = w.rhat;
    k1.st = w.st;
    k1.partial = w.partial;
    k1.counter = w.counter;
    LpArgs k3 = k1;
    k3.out = w.t;
    k3.in = w.s;
    k3.epi = EPI_DOT_TS;
    k3.epi_vec = w.s;
    InnerWork& iw = c->inner;
    volatile BicgPublic* pub = iw.pub_host;
    long long dummy = 0;
    gs_status s;
    int enq = 0;
    GS_CUDA(c, cudaEventRecord(iw.ev[0], c->stream));
    GS_CUDA(c, cudaEventSynchronize(iw.ev[0]));
    if (!pub->done) {
        for (int it = 0; it < maxit; ++it) {
            if (it >= depth) {
                GS_CUDA(c, cudaEventSynchronize(iw.ev[(it - depth) % 4]));
                if (pub->done) break;
            }
            if ((s = launch_lp_stencil<S>(c, k1, pd->hops, pd->variant, &dummy)) != GS_OK) return s;
            k_lp_s<S><<<gr, bb, 0, c->stream>>>(w.r, w.v, w.p, w.s, w.x, n, w.st, w.partial,
                                                 w.counter);
            if ((s = launch_lp_stencil<S>(c, k3, pd->hops, pd->variant, &dummy)) != GS_OK) return s;
            k_lp_xr<S><<<gr, bb, 0, c->stream>>>(w.s, w.t, w.rhat, w.x, w.r, n, w.st, w.partial,
                                                  w.counter);
            k_lp_p<S><<<gp, bb, 0, c->stream>>>(w.r, w.v, w.p, n, w.st);
            c->launches += 3;
            c->stencil_sites += 2 * n;
            GS_CHECK_LAUNCH(c);
            GS_CUDA(c, cudaEventRecord(iw.ev[it % 4], c->stream));
            enq = it + 1;
        }
        if (enq > 0) GS_CUDA(c, cudaEventSynchronize(iw.ev[(enq - 1) % 4]));
    }
    c->launches += dummy;
    *iters_out = pub->iter;
    *status_out = pub->status;
    return GS_OK;
}

// z = D_rr^-1 t to FP64 tolerance o.inner_tol, low-precision inner iterations.
gs_status inner_solve_mixed(gs_ctx* c, const Plan* p, const double2* t, double2* z,
                            const gs_solve_opts& o, gs_solve_stats& st) {
    const int prec = o.inner_prec;
    const int64_t n = c->V - p->nb;
    gs_status s = ensure_inner(c, n);
    if (s != GS_OK) return s;
    if ((s = ensure_lp(c, prec, n)) != GS_OK) return s;
    LpPlanData* pd = nullptr;
    if ((s = lp_plan(c, p, prec, &pd)) != GS_OK) return s;
    MixedState* m = mixed_of(c);
    LpWork& w = m->w;
    InnerWork& iw = c->inner;
    double2* r64 = iw.r;  // FP64 residual (rest set)
    const size_t vbytes = (size_t)n * kSiteC * sizeof(double2);
    GS_CUDA(c, cudaMemsetAsync(z, 0, vbytes, c->stream));
    GS_CUDA(c, cudaMemcpyAsync(r64, t, vbytes, cudaMemcpyDeviceToDevice, c->stream));
    RedScratch red = iw.red;
    if ((s = launch_norm2(c, red, r64, n * kSiteC, w.rr64)) != GS_OK) return s;
    GS_CUDA(c, cudaMemcpyAsync(w.rr64_host, w.rr64, sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    const double tt = *w.rr64_host;
    st.inner_solves += 1;
    if (!isfinite(tt)) return set_err(c, GS_NONFINITE, "non-finite right-hand side");
    if (tt == 0.0) return GS_OK;
    const double target = o.inner_tol * o.inner_tol * tt;
    const float lo_tol = (float)(o.lowp_tol > 0.0 ? o.lowp_tol : (prec == GS_BF16 ? 3e-2 : 1e-5));
    const int depth = (o.check_every >= 1 && o.check_every <= 4) ? o.check_every : 2;
    double rr = tt;
    int stalls = 0;
    long long iters_total = 0;
    const int gs_ = grid_for(n, kLpRed, c->num_sms * 4 < kMaxRedBlocks ? c->num_sms * 4 : kMaxRedBlocks);
    const int gp = grid_for(n, kLpRed, c->num_sms * 16);
    StencilArgs ra;
    memset(&ra, 0, sizeof ra);
    ra.out = r64;
    ra.o0 = p->nb;
    ra.n_out = n;
    ra.inA = z;
    ra.a0 = p->nb;
    ra.a1 = c->V;
    ra.b1 = c->V;
    ra.diag = c->m0 + 4.0;
    ra.negate = 1;
    ra.addend = t;
    ra.plan = p;
    ra.nbr = p->nbr;
    ra.links = p->links;
    if (m->zbak_cap < n) {
        cudaFree(m->zbak);
        m->zbak = nullptr;
        if (cudaMalloc(&m->zbak, vbytes) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GS_ENOMEM, "allocating the correction backup failed");
        }
        m->zbak_cap = n;
    }
    // A low-precision cycle that fails (a zero or non-finite scalar, e.g. a
    // network whose output is not finite) or whose correction leaves a
    // non-finite residual is discarded: z and r keep their values from before
    // the cycle and the plain FP64 BiCGStab below finishes the solve.
    int cycles = 0;
    for (; cycles < 100 && rr > target; ++cycles) {
        if (stalls >= 2) break;
        int it = 0, status = 0;
        if (o.inner_solver == GS_INNER_FGMRES_NET) {
            // flexible GMRES with the network as right preconditioner; its FP64
            // correction is added to z below in place of the low-precision one
            if (m->e64_cap < n) {
                cudaFree(m->e64);
                m->e64 = nullptr;
                if (cudaMalloc(&m->e64, (size_t)n * kSiteC * sizeof(double2)) != cudaSuccess) {
                    cudaGetLastError();
                    return set_err(c, GS_ENOMEM, "allocating the FP64 correction failed");
                }
                m->e64_cap = n;
            }
            s = inner_fgmres_net(c, p, r64, m->e64, lo_tol, o.inner_restart, &it);
            if (s == GS_NONFINITE || s == GS_BREAKDOWN) {
                iters_total += it;
                break;
            }
        } else if (c->opt_inner_kernel == 0) {
            // init + all iterations of the cycle in one cooperative launch
            LpArgs A;
            memset(&A, 0, sizeof A);
            A.out = w.v;
            A.in = w.p;
            A.links = pd->links;
            A.nbr = pd->nbr_r;
            A.lex = pd->lex;
            A.n = n;
            A.diag = (float)(c->m0 + 4.0);
            A.epi = EPI_DOT_RHAT_V;
            A.epi_vec = w.rhat;
            LpArgs C = A;
            C.out = w.t;
            C.in = w.s;
            C.epi = EPI_DOT_TS;
            C.epi_vec = w.s;
            void* vecs[7] = {w.x, w.r, w.rhat, w.p, w.v, w.s, w.t};
            int slot = -1;
            if (c->prof.on && (s = prof_begin(c, &slot)) != GS_OK) return s;
            s = persistent_bicg_lp(c, prec, A, C, r64, w.rr64, vecs, w.st, n, lo_tol,
                                   o.inner_max_iter);
            if (s != GS_OK) return s;
            if (slot >= 0) GS_CUDA(c, cudaEventRecord(c->prof.ev[2 * slot + 1], c->stream));
            GS_CUDA(c, cudaEventRecord(iw.ev[0], c->stream));
            GS_CUDA(c, cudaEventSynchronize(iw.ev[0]));
            volatile BicgPublic* pub = iw.pub_host;
            it = pub->iter;
            status = pub->status;
            if (slot >= 0) {
                // two low-precision D applications and the vector updates per iteration
                const double sb = (double)spinor_bytes(prec), lb = (double)link_bytes(prec);
                const double per_d_fl = 168.0 * pd->hops + 48.0 * n;
                const double per_d_by = 2.0 * sb * n + lb * 0.5 * pd->hops;
                c->prof.ran_host[slot] = 1;
                GS_CUDA(c, cudaMemcpy(c->prof.ran_dev + slot, c->prof.ran_host + slot, sizeof(int),
                                      cudaMemcpyHostToDevice));
                c->prof.pending.push_back({slot, 4, (long long)(2 * it * n),
                                           (long long)(2 * it * pd->hops),
                                           it * (2.0 * per_d_fl + 84.0 * 12.0 * n),
                                           it * (2.0 * per_d_by + 14.0 * sb * n)});
            }
        } else {
            if (prec == GS_BF16)
                k_lp_init<__nv_bfloat16><<<gs_, kLpRed, 0, c->stream>>>(
                    r64, w.rr64, w.r, w.rhat, w.p, w.x, n, lo_tol, w.st, w.partial, w.counter);
            else
                k_lp_init<float><<<gs_, kLpRed, 0, c->stream>>>(r64, w.rr64, w.r, w.rhat, w.p, w.x,
                                                                n, lo_tol, w.st, w.partial,
                                                                w.counter);
            c->launches++;
            GS_CHECK_LAUNCH(c);
            if (prec == GS_BF16)
                s = lp_bicgstab<__nv_bfloat16>(c, pd, n, lo_tol, o.inner_max_iter, depth, &it,
                                               &status);
            else
                s = lp_bicgstab<float>(c, pd, n, lo_tol, o.inner_max_iter, depth, &it, &status);
        }
        if (s != GS_OK) return s;
        iters_total += it;
        GS_CUDA(c, cudaMemcpyAsync(m->zbak, z, vbytes, cudaMemcpyDeviceToDevice, c->stream));
        // z += ||r|| e ; r = t - D_rr z (FP64) ; ||r||^2
        if (o.inner_solver == GS_INNER_FGMRES_NET) {
            if ((s = launch_axpby(c, make_double2(1.0, 0.0), m->e64, make_double2(1.0, 0.0), z,
                                  n * kSiteC)) != GS_OK)
                return s;
        } else {
            if (prec == GS_BF16)
                k_lp_accum<__nv_bfloat16><<<gp, kLpRed, 0, c->stream>>>(w.x, w.rr64, z, n);
            else
                k_lp_accum<float><<<gp, kLpRed, 0, c->stream>>>(w.x, w.rr64, z, n);
            c->launches++;
            GS_CHECK_LAUNCH(c);
        }
        if ((s = launch_stencil_f64(c, ra)) != GS_OK) return s;
        if ((s = launch_norm2(c, red, r64, n * kSiteC, w.rr64)) != GS_OK) return s;
        GS_CUDA(c, cudaMemcpyAsync(w.rr64_host, w.rr64, sizeof(double), cudaMemcpyDeviceToHost,
                                   c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        const double rr_new = *w.rr64_host;
        if (!isfinite(rr_new)) {
            // discard the cycle: z back to its previous value, r recomputed
            // from it (the same deterministic stencil, so rr is unchanged)
            GS_CUDA(c, cudaMemcpyAsync(z, m->zbak, vbytes, cudaMemcpyDeviceToDevice, c->stream));
            if ((s = launch_stencil_f64(c, ra)) != GS_OK) return s;
            break;
        }
        stalls = (rr_new > 0.25 * rr) ? stalls + 1 : 0;
        rr = rr_new;
    }
    st.inner_iters += iters_total;
    st.lowp_cycles += cycles;
    if (iters_total > st.inner_max_seen) st.inner_max_seen = (int)iters_total;
    if (rr > target) {
        // the plain FP64 solve finishes the correction: z += D_rr^-1 r
        gs_solve_opts o64 = o;
        o64.inner_prec = GS_F64;
        o64.inner_tol = sqrt(target / rr);
        if (m->e64_cap < n) {
            cudaFree(m->e64);
            m->e64 = nullptr;
            if (cudaMalloc(&m->e64, (size_t)n * kSiteC * sizeof(double2)) != cudaSuccess) {
                cudaGetLastError();
                return set_err(c, GS_ENOMEM, "allocating the FP64 correction failed");
            }
            m->e64_cap = n;
        }
        gs_solve_stats sub;
        memset(&sub, 0, sizeof sub);
        st.lowp_fallbacks += 1;
        // inside a batched call the block ledger counts only the low-precision
        // solver's cooperative blocks: the FP64 fallback there runs one launch
        // per phase instead of a cooperative grid of another block size
        const int keep_kernel = c->opt_inner_kernel;
        if (c->ledger) c->opt_inner_kernel = 1;
        gs_status si = inner_solve_f64(c, p, r64, m->e64, o64, sub);
        c->opt_inner_kernel = keep_kernel;
        st.inner_iters += sub.inner_iters;
        if (si != GS_OK && si != GS_MAXITER) return si;
        if ((s = launch_axpby(c, make_double2(1.0, 0.0), m->e64, make_double2(1.0, 0.0), z,
                              n * kSiteC)) != GS_OK)
            return s;
        rr *= sub.inner_residual * sub.inner_residual;
        if (si == GS_MAXITER) return si;
    }
    const double rel = sqrt(rr / tt);
    if (rel > st.inner_residual) st.inner_residual = rel;
    return GS_OK;
}

// ---------------------------------------------------------------------------
// ABI: low-precision vectors and the low-precision stencil
// ---------------------------------------------------------------------------
static gs_status lp_entry(gs_ctx* c, int type, int dir, int inverse, int prec, LpPlanData** pd) {
    if (!c) return GS_EINVAL;
    if (prec != GS_F32 && prec != GS_BF16)
        return set_err(c, GS_EINVAL, "low-precision calls take GS_F32 or GS_BF16, not %d", prec);
    if (type != 0 && type != GS_TYPE_I && type != GS_TYPE_II)
        return set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    return lp_plan(c, p, prec, pd);
}

// y = D_rr x on the rest set of plan p, FP32 storage ([6][n_r] float4), the
// autotuned stencil variant; for the FP32 flexible GMRES of the learned
// preconditioner.
gs_status lp_rr_apply_f32(gs_ctx* c, const Plan* p, const void* x, void* y) {
    LpPlanData* pd = nullptr;
    gs_status s = lp_plan(c, p, GS_F32, &pd);
    if (s != GS_OK) return s;
    LpArgs a;
    memset(&a, 0, sizeof a);
    a.out = y;
    a.in = x;
    a.links = pd->links;
    a.nbr = pd->nbr_r;
    a.lex = pd->lex;
    a.n = pd->n;
    a.diag = (float)(c->m0 + 4.0);
    a.epi = EPI_NONE;
    long long launches = 0;
    s = launch_lp_stencil<float>(c, a, pd->hops, pd->variant, &launches);
    c->launches += launches;
    c->stencil_sites += pd->n;
    return s;
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_lowp_pack(gs_ctx* c, int type, int dir, int inverse, int prec, const void* x_dev,
                       void* x_lp_dev) {
    LpPlanData* pd = nullptr;
    gs_status s = lp_entry(c, type, dir, inverse, prec, &pd);
    if (s != GS_OK) return s;
    if (!x_dev || !x_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    const int g = grid_for(pd->n, 256, c->num_sms * 8);
    if (prec == GS_BF16)
        k_lp_pack<__nv_bfloat16><<<g, 256, 0, c->stream>>>((const double2*)x_dev, x_lp_dev, pd->n);
    else
        k_lp_pack<float><<<g, 256, 0, c->stream>>>((const double2*)x_dev, x_lp_dev, pd->n);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status gs_lowp_unpack(gs_ctx* c, int type, int dir, int inverse, int prec,
                         const void* x_lp_dev, void* x_dev) {
    LpPlanData* pd = nullptr;
    gs_status s = lp_entry(c, type, dir, inverse, prec, &pd);
    if (s != GS_OK) return s;
    if (!x_dev || !x_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    const int g = grid_for(pd->n, 256, c->num_sms * 8);
    if (prec == GS_BF16)
        k_lp_unpack<__nv_bfloat16><<<g, 256, 0, c->stream>>>(x_lp_dev, (double2*)x_dev, pd->n);
    else
        k_lp_unpack<float><<<g, 256, 0, c->stream>>>(x_lp_dev, (double2*)x_dev, pd->n);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status wilson_apply_lowp(gs_ctx* c, int type, int dir, int inverse, int prec,
                            const void* x_lp_dev, void* y_lp_dev) {
    LpPlanData* pd = nullptr;
    gs_status s = lp_entry(c, type, dir, inverse, prec, &pd);
    if (s != GS_OK) return s;
    if (!x_lp_dev || !y_lp_dev) return set_err(c, GS_EINVAL, "null vector");
    LpArgs a;
    memset(&a, 0, sizeof a);
    a.out = y_lp_dev;
    a.in = x_lp_dev;
    a.links = pd->links;
    a.nbr = pd->nbr_r;
    a.lex = pd->lex;
    a.n = pd->n;
    a.diag = (float)(c->m0 + 4.0);
    a.epi = EPI_NONE;
    long long launches = 0;
    s = (prec == GS_BF16) ? launch_lp_stencil<__nv_bfloat16>(c, a, pd->hops, pd->variant, &launches)
                          : launch_lp_stencil<float>(c, a, pd->hops, pd->variant, &launches);
    c->launches += launches;
    c->stencil_sites += pd->n;
    return s;
}

}  // extern "C"
