// Live timing of the stencil launches (gs_profile / gs_profile_read) and the
// algorithmic work each launch represents.
#include <mutex>

#include "gs_internal.cuh"

namespace gs {

// Which of the two label sets (b = [0, nb), r = [nb, V)) a range covers.
static void sets_of(int64_t lo, int64_t hi, int64_t nb, int64_t V, bool* has_b, bool* has_r) {
    *has_b = lo < nb && hi > 0;
    *has_r = hi > nb && lo < V;
}

void stencil_work(const gs_ctx* c, const Plan* p, const StencilArgs& a, long long* hops,
                  double* flops, double* bytes) {
    const int64_t V = c->V, nb = p->nb;
    bool ob, orr, ib, ir;
    sets_of(a.o0, a.o0 + a.n_out, nb, V, &ob, &orr);
    sets_of(a.a0, a.b1, nb, V, &ib, &ir);
    const bool out_set[2] = {ob, orr}, in_set[2] = {ib, ir};
    const int64_t set_size[2] = {nb, V - nb};
    long long h = 0;
    double link_uses = 0.0;
    long long diag_sites = 0;
    for (int o = 0; o < 2; ++o) {
        if (!out_set[o]) continue;
        if (in_set[o]) diag_sites += set_size[o];
        for (int i = 0; i < 2; ++i) {
            if (!in_set[i]) continue;
            h += p->hops[o][i];
            link_uses += (o == i) ? 0.5 * p->hops[o][i] : (double)p->hops[o][i];
        }
    }
    const int64_t in_sites = a.b1 - a.a0;
    *hops = h;
    *flops = 168.0 * h + 48.0 * diag_sites;
    *bytes = 192.0 * a.n_out + 192.0 * in_sites + 144.0 * link_uses +
             (a.addend ? 192.0 * a.n_out : 0.0);
}

// One event per device, recorded when profiling is first enabled there: the
// common origin of the launch timelines of every context on that device.
static std::mutex g_epoch_mutex;
static cudaEvent_t g_epoch[64] = {};

static gs_status device_epoch(gs_ctx* c, cudaEvent_t* out) {
    int dev = 0;
    GS_CUDA(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_err(c, GS_ECUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_epoch_mutex);
    if (!g_epoch[dev]) {
        GS_CUDA(c, cudaEventCreate(&g_epoch[dev]));
        GS_CUDA(c, cudaEventRecord(g_epoch[dev], c->stream));
        GS_CUDA(c, cudaEventSynchronize(g_epoch[dev]));
    }
    *out = g_epoch[dev];
    return GS_OK;
}

gs_status prof_harvest(gs_ctx* c) {
    Profiler& P = c->prof;
    if (P.pending.empty()) return GS_OK;
    GS_CUDA(c, cudaEventSynchronize(P.ev[2 * P.pending.back().slot + 1]));
    GS_CUDA(c, cudaMemcpy(P.ran_host, P.ran_dev, kProfSlots * sizeof(int), cudaMemcpyDeviceToHost));
    cudaEvent_t epoch = nullptr;
    gs_status se = device_epoch(c, &epoch);
    if (se != GS_OK) return se;
    for (const auto& q : P.pending) {
        if (!P.ran_host[q.slot]) continue;  // a queued launch that found the solve finished
        float ms = 0.f, t0 = 0.f, t1 = 0.f;
        GS_CUDA(c, cudaEventElapsedTime(&ms, P.ev[2 * q.slot], P.ev[2 * q.slot + 1]));
        GS_CUDA(c, cudaEventElapsedTime(&t0, epoch, P.ev[2 * q.slot]));
        GS_CUDA(c, cudaEventElapsedTime(&t1, epoch, P.ev[2 * q.slot + 1]));
        P.timeline[q.prec].push_back(t0);
        P.timeline[q.prec].push_back(t1);
        gs_kernel_profile& t = P.tot[q.prec];
        t.launches += 1;
        t.ms += ms;
        t.sites += q.sites;
        t.hops += q.hops;
        t.flops += q.flops;
        t.bytes += q.bytes;
    }
    P.pending.clear();
    return GS_OK;
}

gs_status prof_begin(gs_ctx* c, int* slot) {
    Profiler& P = c->prof;
    if ((int)P.pending.size() >= kProfSlots) {
        gs_status s = prof_harvest(c);
        if (s != GS_OK) return s;
    }
    *slot = (int)P.pending.size();
    GS_CUDA(c, cudaEventRecord(P.ev[2 * *slot], c->stream));
    return GS_OK;
}

gs_status prof_end(gs_ctx* c, int slot, const Plan* p, const StencilArgs& a) {
    long long hops;
    double flops, bytes;
    stencil_work(c, p, a, &hops, &flops, &bytes);
    return prof_end_work(c, slot, GS_F64, a.n_out, hops, flops, bytes);
}

gs_status prof_end_work(gs_ctx* c, int slot, int prec, long long sites, long long hops,
                        double flops, double bytes) {
    Profiler& P = c->prof;
    GS_CUDA(c, cudaEventRecord(P.ev[2 * slot + 1], c->stream));
    Profiler::Pending q;
    q.slot = slot;
    q.prec = prec;
    q.sites = sites;
    q.hops = hops;
    q.flops = flops;
    q.bytes = bytes;
    P.pending.push_back(q);
    return GS_OK;
}

}  // namespace gs

using namespace gs;

namespace {

// FP64 issue-rate probe: every thread runs kChains independent FMA chains
// (no chain waits on another), so the FP64 pipe, not latency, sets the rate.
constexpr int kChains = 8;
__global__ void __launch_bounds__(256) k_fp64_peak(double* out, int iters, double seed) {
    double a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = seed + 1e-3 * (q + threadIdx.x);
    const double m = 0.999999999, d = 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], m, d);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == 1234.5678) out[blockIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace

extern "C" {

gs_status gs_profile(gs_ctx* c, int enable) {
    if (!c) return GS_EINVAL;
    Profiler& P = c->prof;
    if (enable) {
        if (P.ev.empty()) {
            P.ev.resize(2 * kProfSlots);
            for (auto& e : P.ev) GS_CUDA(c, cudaEventCreate(&e));
            GS_CUDA(c, cudaMalloc(&P.ran_dev, kProfSlots * sizeof(int)));
            GS_CUDA(c, cudaHostAlloc(&P.ran_host, kProfSlots * sizeof(int), 0));
            GS_CUDA(c, cudaMalloc(&P.phases_dev, 16 * sizeof(unsigned long long)));
        }
        GS_CUDA(c, cudaMemsetAsync(P.phases_dev, 0, 16 * sizeof(unsigned long long), c->stream));
        gs_status s = prof_harvest(c);
        if (s != GS_OK) return s;
        cudaEvent_t epoch = nullptr;
        if ((s = device_epoch(c, &epoch)) != GS_OK) return s;
        for (auto& t : P.tot) t = gs_kernel_profile{};
        for (auto& t : P.timeline) t.clear();
        P.on = true;
    } else {
        gs_status s = prof_harvest(c);
        P.on = false;
        if (s != GS_OK) return s;
    }
    return GS_OK;
}

gs_status gs_profile_phases(gs_ctx* c, double* out, int n) {
    if (!c || !out || n < 15) return GS_EINVAL;
    unsigned long long h[16] = {};
    if (c->prof.phases_dev) {
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        GS_CUDA(c, cudaMemcpy(h, c->prof.phases_dev, sizeof h, cudaMemcpyDeviceToHost));
    }
    // marks: A work 0, sync 1, total 2; B work 3, sync 4, total 5; C 6, 7, 8;
    // D 9, 10, 11; E work 12, sync 13
    for (int i = 0; i < 14; ++i) out[i] = (double)h[i];
    out[14] = 0.0;
    return GS_OK;
}

gs_status gs_profile_read(gs_ctx* c, int prec, gs_kernel_profile* out) {
    if (!c || !out) return GS_EINVAL;
    if (prec < 0 || prec > 4) return set_err(c, GS_EINVAL, "unknown profile family %d", prec);
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    gs_status s = prof_harvest(c);
    if (s != GS_OK) return s;
    *out = c->prof.tot[prec];
    return GS_OK;
}

gs_status gs_profile_timeline(gs_ctx* c, int family, double* out, int cap, int* n_out) {
    if (!c || !n_out || (cap > 0 && !out)) return GS_EINVAL;
    if (family < 0 || family > 4) return set_err(c, GS_EINVAL, "unknown profile family %d", family);
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    gs_status s = prof_harvest(c);
    if (s != GS_OK) return s;
    const std::vector<double>& t = c->prof.timeline[family];
    *n_out = (int)(t.size() / 2);
    for (int i = 0; i < cap && i < (int)t.size(); ++i) out[i] = t[i];
    return GS_OK;
}

gs_status gs_fp64_peak(gs_ctx* c, double* tflops_out) {
    if (!c || !tflops_out) return GS_EINVAL;
    const int blocks = c->num_sms * 8, iters = 1 << 14;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GS_CUDA(c, cudaEventCreate(&e0));
    GS_CUDA(c, cudaEventCreate(&e1));
    double* sink = c->scal_dev;
    float best = 0.f;
    for (int rep = 0; rep < 6; ++rep) {   // the first launch warms up; the fastest counts
        GS_CUDA(c, cudaEventRecord(e0, c->stream));
        k_fp64_peak<<<blocks, 256, 0, c->stream>>>(sink, iters, 1.0);
        GS_CUDA(c, cudaEventRecord(e1, c->stream));
        GS_CUDA(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        GS_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    c->launches += 6;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * kChains * (double)iters * blocks * 256.0;
    *tflops_out = best > 0.f ? flops / (best * 1e-3) / 1e12 : 0.0;
    return GS_OK;
}

}  // extern "C"
