// The C ABI (include/gschur.h): context management and the entry points
// wilson_apply, permute_sites, schur_apply and schur_solve.
#include <math.h>

#include "gs_internal.cuh"

using namespace gs;

namespace {

const char* kVersion = "gschur 0.1 (sm_103a)";

gs_status check_ctx(const gs_ctx* c) { return c ? GS_OK : GS_EINVAL; }

gs_status check_opts(gs_ctx* c, const gs_solve_opts& o) {
    if (!(o.tol > 0.0) || !(o.inner_tol > 0.0))
        return set_err(c, GS_EINVAL, "tolerances must be positive");
    if (o.restart < 1 || o.restart > kMaxRestart)
        return set_err(c, GS_EINVAL, "restart %d not in 1..%d", o.restart, kMaxRestart);
    if (o.max_iter < 0 || o.inner_max_iter < 1)
        return set_err(c, GS_EINVAL, "iteration limits must be positive");
    if (o.outer_solver != GS_GMRES && o.outer_solver != GS_BICGSTAB)
        return set_err(c, GS_EINVAL, "unknown outer solver %d", o.outer_solver);
    if (o.inner_prec != GS_F64 && o.inner_prec != GS_F32 && o.inner_prec != GS_BF16)
        return set_err(c, GS_EINVAL, "unknown inner precision %d", o.inner_prec);
    if (!(o.lowp_tol >= 0.0) || o.lowp_tol >= 1.0)
        return set_err(c, GS_EINVAL, "lowp_tol must be in [0, 1)");
    if (o.inner_relax && (!(o.relax_cap > 0.0) || o.relax_cap >= 1.0))
        return set_err(c, GS_EINVAL, "relax_cap must be in (0, 1)");
    if (o.inner_solver != GS_INNER_BICGSTAB && o.inner_solver != GS_INNER_FGMRES_NET)
        return set_err(c, GS_EINVAL, "unknown inner solver %d", o.inner_solver);
    if (o.inner_solver == GS_INNER_FGMRES_NET) {
        if (!c->net) return set_err(c, GS_EINVAL, "GS_INNER_FGMRES_NET needs a network (gs_set_net)");
        if (o.inner_prec == GS_F64)
            return set_err(c, GS_EINVAL, "GS_INNER_FGMRES_NET runs inside the mixed inner solve: "
                                         "inner_prec must be GS_F32 or GS_BF16");
        if (o.inner_restart < 1 || o.inner_restart > kMaxRestart)
            return set_err(c, GS_EINVAL, "inner_restart %d not in 1..%d", o.inner_restart, kMaxRestart);
    }
    return GS_OK;
}

void finish_stats(gs_ctx* c, gs_solve_stats* out, gs_solve_stats& st, gs_status s,
                  long long launches0, long long sites0) {
    st.status = s;
    st.kernel_launches = c->launches - launches0;
    st.stencil_sites = c->stencil_sites - sites0;
    if (out) *out = st;
}

}  // namespace

extern "C" {

const char* gs_version(void) { return kVersion; }

void gs_default_opts(gs_solve_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_iter = 3000;
    o->restart = 30;
    o->outer_solver = GS_GMRES;
    o->inner_tol = 1e-12;
    o->inner_max_iter = 5000;
    o->inner_prec = GS_F64;
    o->check_every = 2;
    o->lowp_tol = 0.0;
    o->inner_relax = 1;
    o->relax_cap = 1e-4;
    o->inner_solver = GS_INNER_BICGSTAB;
    o->inner_restart = 16;
}

const char* gs_last_error(const gs_ctx* c) { return c ? c->err.c_str() : "null context"; }

gs_status gs_create(gs_ctx** out, const int dims[4], double m0, void* stream) {
    if (!out || !dims) return GS_EINVAL;
    *out = nullptr;
    // V * 12 < 2^31; each extent is checked against what is left of that bound
    // before it multiplies V, so the product cannot overflow
    const int64_t kMaxSites = (((int64_t)1 << 31) - 1) / kSiteC;
    int64_t V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || dims[mu] > kMaxSites / V) return GS_EINVAL;
        V *= dims[mu];
    }
    if (!isfinite(m0)) return GS_EINVAL;
    gs_ctx* c = new gs_ctx();
    for (int mu = 0; mu < 4; ++mu) c->dims[mu] = dims[mu];
    c->V = V;
    c->m0 = m0;
    c->stream = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return GS_ECUDA;
    }
    const size_t vbytes = (size_t)V * kSiteC * sizeof(double2);
    bool ok = cudaMalloc(&c->U_abi, (size_t)V * 36 * sizeof(double2)) == cudaSuccess &&
              cudaMalloc(&c->full_a, vbytes) == cudaSuccess &&
              cudaMalloc(&c->full_b, vbytes) == cudaSuccess &&
              cudaMalloc(&c->full_c, vbytes) == cudaSuccess &&
              cudaMalloc(&c->scal_dev, 64 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->red.partial, kRedScratchDoubles * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->red.counter, sizeof(unsigned int)) == cudaSuccess &&
              cudaHostAlloc(&c->scal_host, 64 * sizeof(double), 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        gs_destroy(c);
        return GS_ENOMEM;
    }
    if (cudaMemsetAsync(c->red.counter, 0, sizeof(unsigned int), c->stream) != cudaSuccess) {
        cudaGetLastError();
        gs_destroy(c);
        return GS_ECUDA;
    }
    Plan* id = nullptr;
    gs_status s = get_plan(c, 0, 0, 0, &id);
    if (s != GS_OK) {
        gs_destroy(c);
        return s;
    }
    *out = c;
    return GS_OK;
}

gs_status gs_destroy(gs_ctx* c) {
    if (!c) return GS_OK;
    for (gs_ctx* l : c->lanes) gs_destroy(l);
    c->lanes.clear();
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_multi(c);
    free_net_ctx(c);
    free_mixed(c);
    free_persist(c);
    for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
    c->prof.ev.clear();
    cudaFree(c->prof.ran_dev);
    cudaFree(c->prof.phases_dev);
    if (c->prof.ran_host) cudaFreeHost(c->prof.ran_host);
    for (Plan* p : c->plans) free_plan(p);
    c->plans.clear();
    cudaFree(c->U_abi);
    cudaFree(c->full_a);
    cudaFree(c->full_b);
    cudaFree(c->full_c);
    cudaFree(c->scal_dev);
    cudaFree(c->red.partial);
    cudaFree(c->red.counter);
    if (c->scal_host) cudaFreeHost(c->scal_host);
    InnerWork& w = c->inner;
    cudaFree(w.r);
    cudaFree(w.rhat);
    cudaFree(w.p);
    cudaFree(w.v);
    cudaFree(w.s);
    cudaFree(w.t);
    cudaFree(w.rhs);
    cudaFree(w.sol);
    cudaFree(w.st);
    cudaFree(w.red.partial);
    cudaFree(w.red.counter);
    if (w.pub_host) cudaFreeHost(w.pub_host);
    for (int k = 0; k < 4; ++k)
        if (w.ev[k]) cudaEventDestroy(w.ev[k]);
    OuterWork& o = c->outer;
    cudaFree(o.basis);
    cudaFree(o.w);
    cudaFree(o.xb);
    cudaFree(o.wb);
    cudaFree(o.tmp);
    cudaFree(o.hbuf);
    cudaFree(o.y);
    cudaFree(o.red.partial);
    cudaFree(o.red.counter);
    if (o.hbuf_host) cudaFreeHost(o.hbuf_host);
    if (o.y_host) cudaFreeHost(o.y_host);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    cudaGetLastError();
    delete c;
    return GS_OK;
}

gs_status gs_set_option(gs_ctx* c, int option, int value) {
    if (!c) return GS_EINVAL;
    if (option == GS_OPT_STENCIL_VARIANT) {
        if (value < 0 || value > 6) return set_err(c, GS_EINVAL, "stencil variant %d not in 0..6", value);
        c->opt_stencil_variant = value;
        invalidate_mixed_links(c);  // re-tune / re-select on next use
        return GS_OK;
    }
    if (option == GS_OPT_INNER_KERNEL) {
        if (value < 0 || value > 1) return set_err(c, GS_EINVAL, "inner kernel %d not in 0..1", value);
        c->opt_inner_kernel = value;
        return GS_OK;
    }
    if (option == GS_OPT_NET_KERNEL) {
        if (value < 0 || value > 1) return set_err(c, GS_EINVAL, "network kernel %d not in 0..1", value);
        c->opt_net_kernel = value;
        return GS_OK;
    }
    if (option == GS_OPT_MULTI_BATCH) {
        if (value < 0 || value > 2) return set_err(c, GS_EINVAL, "multi-source batching %d not in 0..2", value);
        c->opt_multi_batch = value;
        return GS_OK;
    }
    if (option == GS_OPT_COOP_BLOCKS) {
        if (value < 0 || value > 65536) return set_err(c, GS_EINVAL, "cooperative block count %d not in 0..65536", value);
        c->opt_coop_blocks = value;
        return GS_OK;
    }
    if (option == GS_OPT_BATCH_LANES) {
        if (value < 0 || value > 64) return set_err(c, GS_EINVAL, "batch lanes %d not in 0..64", value);
        c->opt_batch_lanes = value;
        return GS_OK;
    }
    if (option == GS_OPT_WAIT_LIMIT_US) {
        if (value < 1 || value > 60000000)
            return set_err(c, GS_EINVAL, "wait limit %d us not in 1..60000000", value);
        c->wait_ns = (unsigned long long)value * 1000ull;
        return GS_OK;
    }
    return set_err(c, GS_EINVAL, "unknown option %d", option);
}

gs_status gs_get_option(gs_ctx* c, int option, int* value) {
    if (!c || !value) return GS_EINVAL;
    if (option == GS_OPT_STENCIL_VARIANT) {
        *value = c->opt_stencil_variant ? c->opt_stencil_variant : c->tuned_variant;
        return GS_OK;
    }
    if (option == GS_OPT_INNER_KERNEL) {
        *value = c->opt_inner_kernel;
        return GS_OK;
    }
    if (option == GS_OPT_NET_KERNEL) {
        *value = c->opt_net_kernel;
        return GS_OK;
    }
    if (option == GS_OPT_MULTI_BATCH) {
        *value = c->opt_multi_batch;
        return GS_OK;
    }
    if (option == GS_OPT_WAIT_LIMIT_US) {
        *value = (int)(c->wait_ns / 1000ull);
        return GS_OK;
    }
    if (option == GS_OPT_COOP_BLOCKS) {
        *value = c->opt_coop_blocks;
        return GS_OK;
    }
    if (option == GS_OPT_BATCH_LANES) {
        *value = c->opt_batch_lanes;
        return GS_OK;
    }
    return set_err(c, GS_EINVAL, "unknown option %d", option);
}

gs_status gs_selftest_wait(gs_ctx* c, int which) {
    if (check_ctx(c) != GS_OK) return GS_EINVAL;
    gs_status got = GS_OK;
    if (which == 0) {
        gs_status s = selftest_grid_timeout(c, &got);
        if (s != GS_OK) return s;
    } else if (which == 1) {
        int* err_dev = (int*)(c->scal_dev + 32);
        GS_CUDA(c, cudaMemsetAsync(err_dev, 0, sizeof(int), c->stream));
        gs_status s = selftest_mbar_timeout(c, err_dev);
        if (s != GS_OK) return s;
        int h = 0;
        GS_CUDA(c, cudaMemcpyAsync(&h, err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        got = (gs_status)h;
    } else {
        return set_err(c, GS_EINVAL, "unknown self-test %d", which);
    }
    if (got == GS_TIMEOUT)
        return set_err(c, GS_TIMEOUT, "%s wait ran out after %.3f ms, as the self-test intends",
                       which == 0 ? "grid-barrier" : "mbarrier", 1e-6 * (double)c->wait_ns);
    return set_err(c, got, "the self-test's wait did not run out (status %d)", (int)got);
}

gs_status gs_set_gauge(gs_ctx* c, const void* U_dev) {
    if (check_ctx(c) != GS_OK) return GS_EINVAL;
    if (!U_dev) return set_err(c, GS_EINVAL, "null gauge field");
    GS_CUDA(c, cudaMemcpyAsync(c->U_abi, U_dev, (size_t)c->V * 36 * sizeof(double2),
                               cudaMemcpyDeviceToDevice, c->stream));
    c->have_gauge = true;
    c->gauge_gen++;
    c->net_links_fresh = false;
    invalidate_mixed_links(c);
    for (Plan* p : c->plans) {
        gs_status s = pack_plan_links(c, p);
        if (s != GS_OK) return s;
    }
    return GS_OK;
}

gs_status wilson_apply(gs_ctx* c, const void* x_dev, void* y_dev) {
    if (check_ctx(c) != GS_OK) return GS_EINVAL;
    if (!x_dev || !y_dev) return set_err(c, GS_EINVAL, "null vector");
    if (!c->have_gauge) return set_err(c, GS_ENOGAUGE, "no gauge field set");
    const Plan* p = c->plans[0];
    StencilArgs a;
    memset(&a, 0, sizeof a);
    a.out = (double2*)y_dev;
    a.o0 = 0;
    a.n_out = c->V;
    a.inA = (const double2*)x_dev;
    a.a0 = 0;
    a.a1 = c->V;
    a.b1 = c->V;
    a.diag = c->m0 + 4.0;
    a.plan = p;
    a.nbr = p->nbr;
    a.links = p->links;
    return launch_stencil_f64(c, a);
}

gs_status permute_sites(gs_ctx* c, int type, int dir, int inverse, int transpose,
                        const void* x_dev, void* y_dev, int64_t* n_b_out) {
    if (check_ctx(c) != GS_OK) return GS_EINVAL;
    if (!x_dev || !y_dev) return set_err(c, GS_EINVAL, "null vector");
    if (type != GS_TYPE_I && type != GS_TYPE_II)
        return set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    if (n_b_out) *n_b_out = p->nb;
    if (transpose) return launch_scatter(c, p->perm, (const double2*)x_dev, (double2*)y_dev, c->V);
    return launch_gather(c, p->perm, (const double2*)x_dev, (double2*)y_dev, c->V);
}

gs_status gs_get_permutation(gs_ctx* c, int type, int dir, int inverse, int32_t* perm_dev,
                             int64_t* n_b_out) {
    if (check_ctx(c) != GS_OK) return GS_EINVAL;
    if (!perm_dev) return set_err(c, GS_EINVAL, "null output");
    if (type != GS_TYPE_I && type != GS_TYPE_II)
        return set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    Plan* p = nullptr;
    gs_status s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) return s;
    if (n_b_out) *n_b_out = p->nb;
    GS_CUDA(c, cudaMemcpyAsync(perm_dev, p->perm, (size_t)c->V * sizeof(int32_t),
                               cudaMemcpyDeviceToDevice, c->stream));
    return GS_OK;
}

gs_status gs_solve_rr(gs_ctx* c, int type, int dir, int inverse, const void* t_dev, void* z_dev,
                      const gs_solve_opts* opts, gs_solve_stats* stats) {
    if (check_ctx(c) != GS_OK) return GS_EINVAL;
    gs_solve_opts o;
    gs_default_opts(&o);
    if (opts) o = *opts;
    gs_solve_stats st;
    memset(&st, 0, sizeof st);
    const long long l0 = c->launches, s0 = c->stencil_sites;
    gs_status s = check_opts(c, o);
    if (s == GS_OK && (!t_dev || !z_dev)) s = set_err(c, GS_EINVAL, "null vector");
    if (s == GS_OK && type != GS_TYPE_I && type != GS_TYPE_II)
        s = set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (s == GS_OK && !c->have_gauge) s = set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    if (s == GS_OK) s = get_plan(c, type, dir, inverse, &p);
    if (s == GS_OK) {
        s = gs::inner_solve(c, p, (const double2*)t_dev, (double2*)z_dev, o, st);
        st.true_residual = st.inner_residual;   // ||t - D_rr z|| / ||t||, recomputed in FP64
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess && s == GS_OK) s = set_err(c, GS_ECUDA, "gs_solve_rr: %s", cudaGetErrorString(e));
    }
    finish_stats(c, stats, st, s, l0, s0);
    return s;
}

gs_status schur_apply(gs_ctx* c, int type, int dir, int inverse, const void* xb_dev, void* yb_dev,
                      const gs_solve_opts* opts, gs_solve_stats* stats) {
    if (check_ctx(c) != GS_OK) return GS_EINVAL;
    gs_solve_opts o;
    gs_default_opts(&o);
    if (opts) o = *opts;
    gs_solve_stats st;
    memset(&st, 0, sizeof st);
    const long long l0 = c->launches, s0 = c->stencil_sites;
    gs_status s = check_opts(c, o);
    if (s == GS_OK && (!xb_dev || !yb_dev)) s = set_err(c, GS_EINVAL, "null vector");
    if (s == GS_OK && type != GS_TYPE_I && type != GS_TYPE_II)
        s = set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (s == GS_OK && !c->have_gauge) s = set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    if (s == GS_OK) s = get_plan(c, type, dir, inverse, &p);
    if (s == GS_OK) {
        s = schur_apply_internal(c, p, (const double2*)xb_dev, (double2*)yb_dev, o, st);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess && s == GS_OK)
            s = set_err(c, GS_ECUDA, "schur_apply: %s", cudaGetErrorString(e));
    }
    finish_stats(c, stats, st, s, l0, s0);
    return s;
}

gs_status schur_solve(gs_ctx* c, int type, int dir, int inverse, const void* f_dev, void* x_dev,
                      const gs_solve_opts* opts, gs_solve_stats* stats) {
    if (check_ctx(c) != GS_OK) return GS_EINVAL;
    gs_solve_opts o;
    gs_default_opts(&o);
    if (opts) o = *opts;
    gs_solve_stats st;
    memset(&st, 0, sizeof st);
    const long long l0 = c->launches, s0 = c->stencil_sites;
    gs_status s = check_opts(c, o);
    if (s == GS_OK && (!f_dev || !x_dev)) s = set_err(c, GS_EINVAL, "null vector");
    if (s == GS_OK && type != GS_TYPE_I && type != GS_TYPE_II)
        s = set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (s == GS_OK && !c->have_gauge) s = set_err(c, GS_ENOGAUGE, "no gauge field set");
    Plan* p = nullptr;
    if (s == GS_OK) s = get_plan(c, type, dir, inverse, &p);
    if (s != GS_OK) {
        finish_stats(c, stats, st, s, l0, s0);
        return s;
    }
    const int64_t V = c->V, nb = p->nb, nr = V - nb;
    const double2* f = (const double2*)f_dev;
    double2* x = (double2*)x_dev;
    double2* F = c->full_a;  // P f (label order)
    double2* Z = c->full_b;  // r-vector temporaries
    double2* X = c->full_c;  // solution in label order
    gs_status inner_flag = GS_OK;
    auto run = [&]() -> gs_status {
        gs_status e = launch_gather(c, p->perm, f, F, V);
        if (e != GS_OK) return e;
        // w_b = f_b - D_br D_rr^-1 f_r
        e = gs::inner_solve(c, p, F + nb * kSiteC, Z, o, st);
        if (e == GS_MAXITER) inner_flag = e;
        else if (e != GS_OK) return e;
        e = ensure_outer(c, nb, o.restart);
        if (e != GS_OK) return e;
        double2* wb = c->outer.wb;
        StencilArgs a;
        memset(&a, 0, sizeof a);
        a.out = wb;
        a.o0 = 0;
        a.n_out = nb;
        a.inA = Z;
        a.a0 = nb;
        a.a1 = V;
        a.b1 = V;
        a.diag = c->m0 + 4.0;
        a.negate = 1;
        a.addend = F;
        a.plan = p;
    a.nbr = p->nbr;
        a.links = p->links;
        if ((e = launch_stencil_f64(c, a)) != GS_OK) return e;
        // S_bb x_b = w_b, x_b written into the b part of X
        e = outer_solve(c, p, wb, X, o, st);
        if (e == GS_MAXITER) inner_flag = e;
        else if (e != GS_OK) return e;
        // x_r = D_rr^-1 (f_r - D_rb x_b)
        a.out = Z;
        a.o0 = nb;
        a.n_out = nr;
        a.inA = X;
        a.a0 = 0;
        a.a1 = nb;
        a.b1 = nb;
        a.negate = 1;
        a.addend = F + nb * kSiteC;
        if ((e = launch_stencil_f64(c, a)) != GS_OK) return e;
        e = gs::inner_solve(c, p, Z, X + nb * kSiteC, o, st);
        if (e == GS_MAXITER) inner_flag = e;
        else if (e != GS_OK) return e;
        if ((e = launch_scatter(c, p->perm, X, x, V)) != GS_OK) return e;
        // true residual ||f - D x|| / ||f|| in FP64 on the full lattice
        const Plan* id = c->plans[0];
        StencilArgs rd;
        memset(&rd, 0, sizeof rd);
        rd.out = F;
        rd.o0 = 0;
        rd.n_out = V;
        rd.inA = x;
        rd.a0 = 0;
        rd.a1 = V;
        rd.b1 = V;
        rd.diag = c->m0 + 4.0;
        rd.negate = 1;
        rd.addend = f;
        rd.plan = id;
        rd.nbr = id->nbr;
        rd.links = id->links;
        if ((e = launch_stencil_f64(c, rd)) != GS_OK) return e;
        if ((e = launch_norm2(c, c->red, F, V * kSiteC, c->scal_dev)) != GS_OK) return e;
        if ((e = launch_norm2(c, c->red, f, V * kSiteC, c->scal_dev + 1)) != GS_OK) return e;
        GS_CUDA(c, cudaMemcpyAsync(c->scal_host, c->scal_dev, 2 * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        st.true_residual = c->scal_host[1] > 0.0 ? sqrt(c->scal_host[0] / c->scal_host[1]) : 0.0;
        return inner_flag;
    };
    s = run();
    finish_stats(c, stats, st, s, l0, s0);
    return s;
}

}  // extern "C"
