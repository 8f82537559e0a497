// Internal declarations of the gschur CUDA library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <condition_variable>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gschur.h"

namespace gs {

// ---------------------------------------------------------------------------
// complex double helpers (interleaved re, im in a double2)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// a + i*b and a - i*b
__host__ __device__ __forceinline__ double2 caddi(double2 a, double2 b) { return make_double2(a.x - b.y, a.y + b.x); }
__host__ __device__ __forceinline__ double2 csubi(double2 a, double2 b) { return make_double2(a.x + b.y, a.y - b.x); }
__host__ __device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }    // i*a
__host__ __device__ __forceinline__ double2 cmulmi(double2 a) { return make_double2(a.y, -a.x); }   // -i*a
// acc += a*b with fused multiply-adds
__host__ __device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a)*b
__host__ __device__ __forceinline__ void ccfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

constexpr int kNc = 3;
constexpr int kNs = 4;
constexpr int kSiteC = 12;   // complex numbers per site spinor
constexpr int kLinkC = 9;    // complex numbers per SU(3) link

// ---------------------------------------------------------------------------
// device-side solver state (one per inner solve workspace)
// ---------------------------------------------------------------------------
struct BicgState {
    double2 rho;      // <rhat, r>
    double2 alpha;
    double2 omega;
    double2 beta;
    double rr;        // ||r||^2
    double bb;        // ||b||^2
    double tol2;      // (tol)^2 * ||b||^2
    int done;         // 1 when converged or failed: kernels become no-ops
    int status;       // GS_OK / GS_BREAKDOWN / GS_NONFINITE
    int iter;         // completed iterations
    int pad;
    struct BicgPublic* pub;  // host-mapped mirror the host polls (device pointer)
};

// The part of the solver state the host reads while iterations are queued:
// written by the last block of the kernels that change it, followed by a
// system-scope fence, into pinned host memory mapped into the device.
struct BicgPublic {
    int done;
    int status;
    int iter;
    int pad;
    double rr;
    double bb;
};

__device__ __forceinline__ void publish(BicgState* st) {
    BicgPublic* p = st->pub;
    if (p) {
        p->rr = st->rr;
        p->bb = st->bb;
        p->iter = st->iter;
        p->status = st->status;
        __threadfence_system();
        p->done = st->done;
        __threadfence_system();
    }
}

// ---------------------------------------------------------------------------
// a permutation plan: label order, neighbour table and label-ordered links
// ---------------------------------------------------------------------------
struct Plan {
    int type = 0;          // 0 = identity (site order), GS_TYPE_I, GS_TYPE_II
    int dir = 0;
    int inverse = 0;
    int64_t nb = 0;        // coarse count (labels [0, nb) are b)
    int32_t* perm = nullptr;     // [V] label -> site
    int32_t* label = nullptr;    // [V] site -> label
    int2* nbr = nullptr;         // [V][4] (fwd label, bwd label) per mu, label-indexed
    double2* links = nullptr;    // [V][4][9] -1/2 U_mu(perm[j]) in label order
    bool links_ready = false;
    long long hops[2][2] = {{0, 0}, {0, 0}};  // [out set][in set] in-set neighbour terms (0 = b, 1 = r)
    double2* dtinv = nullptr;    // [V - nb][12][12] inverse block row sums of D_rr (Reusken), lazily
    bool dtinv_ready = false;
};

// Event-timed stencil launches (gs_profile).
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;      // 2 per slot
    struct Pending {
        int slot;
        int prec;                     // GS_F64 / GS_F32 / GS_BF16 stencil
        long long sites, hops;
        double flops, bytes;
    };
    std::vector<Pending> pending;
    int* ran_dev = nullptr;           // per slot: 1 if the launch did work (not an early exit)
    int* ran_host = nullptr;          // pinned
    gs_kernel_profile tot[5] = {};    // stencil F64/F32/BF16, persistent solver F64 / low precision
    std::vector<double> timeline[5];  // per family: (start, end) ms of each launch since the device epoch
    unsigned long long* phases_dev = nullptr;  // [16] cycles per phase of the persistent FP64 solver
};
constexpr int kProfSlots = 2048;

// Reduction scratch for one chain of fused reductions.
struct RedScratch {
    double* partial = nullptr;     // [kRedScratchDoubles]
    unsigned int* counter = nullptr;
};
constexpr int kMaxRedBlocks = 1024;
constexpr int kMaxRedVals = 8;
constexpr int kMaxRestart = 64;
// covers kMaxRedBlocks * kMaxRedVals and the multi-dot (up to 1008 blocks per
// vector x 65 vectors x 2)
constexpr int64_t kRedScratchDoubles = 131072;

// Inner-solver workspace (vectors of n_r sites).
struct InnerWork {
    int64_t cap_sites = 0;
    double2 *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr;
    double2 *rhs = nullptr, *sol = nullptr;  // right-hand side and solution of S_bb's inner solve
    BicgState* st = nullptr;       // device
    BicgPublic* pub_host = nullptr;  // pinned, mapped
    BicgPublic* pub_dev = nullptr;   // device alias of pub_host
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    RedScratch red;
};

// Outer-solver workspace (vectors of n_b sites).
struct OuterWork {
    int64_t cap_sites = 0;
    int cap_m = 0;
    double2* basis = nullptr;   // [(m+1)][nb*12]
    double2* w = nullptr;
    double2* xb = nullptr;
    double2* wb = nullptr;
    double2* tmp = nullptr;
    double2* hbuf = nullptr;    // device: h (m+2), h2 (m+2), (||w||^2, 0)
    double2* hbuf_host = nullptr;  // pinned copy
    double2* y = nullptr;       // device coefficients (m+1 entries)
    double2* y_host = nullptr;  // pinned
    RedScratch red;
};

}  // namespace gs

struct gs_ctx;

namespace gs {
// The blocks of the persistent solver kernels of one schur_solve_batched
// call.  Those kernels all have 128 threads and the same registers, so their
// blocks are interchangeable and the GPU holds per_sm x SMs of them at once.
// held[] records, per running solve, the blocks its kernel may have in
// flight: its last grid (its previous kernel has finished before it launches
// again), or nothing before its first launch.  A grid is granted only from
// blocks no other solve holds, so the cooperative grids of all running
// solves always fit on the GPU together; a solve that has not launched yet
// is counted at `reserve` when the others are granted blocks, so it finds
// room at its first launch.
struct BlockLedger {
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<int> running{0};
    int64_t reserve = 1;
    struct Entry {
        const gs_ctx* ctx;
        int64_t blocks;
        bool launched;
    };
    std::vector<Entry> held;
};
void ledger_enter(BlockLedger* L, const gs_ctx* c);
void ledger_leave(BlockLedger* L, const gs_ctx* c);
// blocks for c's next cooperative grid: at most want and target, never more
// than the others leave free; 0 if none became free within the context's
// wait limit x 60
int64_t ledger_grant(gs_ctx* c, int per_sm, int64_t want, int64_t target);
}  // namespace gs

struct gs_ctx {
    int dims[4];
    int64_t V = 0;
    double m0 = 0.0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    bool have_gauge = false;
    double2* U_abi = nullptr;          // private copy of the caller's field, [V][4][9]
    std::vector<gs::Plan*> plans;      // plans[0] = identity
    gs::InnerWork inner;
    gs::OuterWork outer;
    double2* full_a = nullptr;         // [V][12] label-ordered scratch
    double2* full_b = nullptr;
    double2* full_c = nullptr;
    double* scal_dev = nullptr;        // small device scratch for norms
    double* scal_host = nullptr;       // pinned
    gs::RedScratch red;
    long long launches = 0;
    long long stencil_sites = 0;
    gs::Profiler prof;
    void* mixed = nullptr;             // mixed-precision state (mixed.cu)
    int opt_stencil_variant = 0;       // 0 = autotune, 1/3/4 = site (4/6/8 blocks), 2 = direction
    int opt_inner_kernel = 0;          // 0 = persistent cooperative BiCGStab, 1 = one launch per phase
    int opt_net_kernel = 0;            // 0 = tensor-core network kernels (C = 24), 1 = CUDA cores only
    int opt_multi_batch = 0;           // 0 = by rest-set size, 1 = sources together, 2 = one at a time
    unsigned long long wait_ns = 1000000000ull;  // bound on every device-side wait (GS_OPT_WAIT_LIMIT_US)
    int opt_coop_blocks = 0;           // blocks of this context's cooperative grids in a batched solve (0 = by share)
    void* persist = nullptr;           // persistent-solver scratch (persistent.cu)
    void* multi = nullptr;             // multi-RHS workspaces (multi.cu)
    int coop_block_cap = 0;            // cap on cooperative grids (0 = whole GPU; batched solves)
    // batched solves: the block ledger of the schur_solve_batched call this
    // context is running an item of (null outside such a call)
    gs::BlockLedger* ledger = nullptr;
    int opt_batch_lanes = 0;           // concurrent solves of schur_solve_batched (0 = the library's choice)
    std::vector<gs_ctx*> lanes;        // extra contexts on the same lattice for schur_solve_batched
    cudaStream_t own_stream = nullptr; // a stream the library created for this context (lane contexts)
    unsigned gauge_gen = 0;            // counts gs_set_gauge calls
    unsigned lane_gauge_gen = 0;       // (lane contexts) the parent's gauge_gen their field was copied at
    struct gs_net* net = nullptr;      // learned preconditioner attached with gs_set_net (net.cu)
    bool net_links_fresh = false;      // the network's FP32 link copy matches U_abi
    float2 *fg_V = nullptr, *fg_Z = nullptr, *fg_w = nullptr;  // FGMRES-net vectors (FP32 stencil layout)
    int64_t fg_cap = 0;
    int fg_m = 0;
    double2* fg_h = nullptr;           // device H column (2 (m+2) + 1)
    double2* fg_h_host = nullptr;
    double2* fg_y = nullptr;
    double2* fg_y_host = nullptr;
    gs::RedScratch fg_red;
    int tuned_variant = 0;             // the variant the autotuner picked last
    std::string err;
};

namespace gs {

// largest rest set on which one source leaves the GPU latency bound (GB300:
// sources that share launches win on 8^4, not from 16^4 up)
constexpr int64_t kBatchMaxRestSites = 16384;

// Blocks of a cooperative grid whose kernel fits per_sm blocks on an SM, for
// a set of rest_sites sites: the whole GPU, or inside schur_solve_batched the
// share of one of the solves running at that moment -- all co-resident
// blocks on large sets (HBM bound: more loads in flight), two per SM on small
// ones (latency bound: fewer, fuller blocks and cheaper barriers; measured on
// 8^4: 76 blocks per solve beat 114 with four solves at once).  An explicit
// cap (GS_OPT_COOP_BLOCKS in a batched call) takes precedence.
inline int64_t coop_blocks(const gs_ctx* c, int per_sm, int64_t rest_sites) {
    int64_t g = (int64_t)per_sm * c->num_sms;
    if (c->coop_block_cap > 0) return g < c->coop_block_cap ? g : c->coop_block_cap;
    if (c->ledger) {
        int n = c->ledger->running.load(std::memory_order_relaxed);
        if (n < 1) n = 1;
        const int64_t per = (rest_sites <= kBatchMaxRestSites && per_sm > 2) ? 2 : per_sm;
        g = per * c->num_sms / n;
        if (g < 1) g = 1;
    }
    return g;
}

// error helpers --------------------------------------------------------------
gs_status set_err(gs_ctx* c, gs_status s, const char* fmt, ...);
#define GS_CUDA(ctx, call)                                                       \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess)                                                   \
            return gs::set_err((ctx), GS_ECUDA, "%s failed: %s (%s:%d)", #call,  \
                               cudaGetErrorString(e_), __FILE__, __LINE__);      \
    } while (0)
#define GS_CHECK_LAUNCH(ctx) GS_CUDA(ctx, cudaGetLastError())

// lattice / permutation (lattice.cu) ------------------------------------------
gs_status get_plan(gs_ctx* c, int type, int dir, int inverse, Plan** out);
gs_status pack_plan_links(gs_ctx* c, Plan* p);
void free_plan(Plan* p);
gs_status launch_gather(gs_ctx* c, const int32_t* perm, const double2* x, double2* y, int64_t n);
gs_status build_labels(gs_ctx* c, const int dims[4], int type, int dir, int inverse,
                       int32_t* perm_dev, int32_t* label_dev, int64_t* nb_out);
gs_status launch_scatter(gs_ctx* c, const int32_t* perm, const double2* x, double2* y, int64_t n);

// stencil (dslash_f64.cu) -------------------------------------------------------
// out[k] for labels o0+k, k < n_out:
//   out = [addend] + sign * ( diag * self + sum_hops U' in )
// where the input vector is split in two label segments: [a0, a1) read from
// inA + (l - a0)*12 and [a1, b1) read from inB + (l - a1)*12 (b1 == a1: no B).
// self is the input at the output label when it lies in [a0, b1).
enum StencilEpi { EPI_NONE = 0, EPI_DOT_RHAT_V = 1, EPI_DOT_TS = 2, EPI_DOT_TSR = 3 };
struct StencilArgs {
    double2* out;
    int64_t o0, n_out;
    const double2* inA;
    int64_t a0, a1;
    const double2* inB;
    int64_t b1;
    const double2* addend;   // may be null
    double diag;             // m0 + 4
    int negate;              // sign = -1 if set
    const Plan* plan;        // host-side plan (work counting only; never read on the device)
    const int2* nbr;         // plan->nbr (device)
    const double2* links;    // plan->links (device)
    // epilogue for the fused inner-solver kernels
    int epi;
    const double2* epi_vec;  // rhat (EPI_DOT_RHAT_V) or s (EPI_DOT_TS, EPI_DOT_TSR), same indexing as out
    const double2* epi_vec2; // rhat (EPI_DOT_TSR: also <rhat, t>)
    BicgState* st;
    RedScratch red;
    int* ran;                // profiling: set to 1 if the launch did work, 0 if it exited early
};
gs_status launch_stencil_f64(gs_ctx* c, const StencilArgs& a);
gs_status launch_stencil_f64_on(const StencilArgs& a, cudaStream_t stream);
// profiling (api.cu): work counted for one stencil launch on plan p
void stencil_work(const gs_ctx* c, const Plan* p, const StencilArgs& a, long long* hops,
                  double* flops, double* bytes);
gs_status prof_begin(gs_ctx* c, int* slot);
gs_status prof_end(gs_ctx* c, int slot, const Plan* p, const StencilArgs& a);
gs_status prof_end_work(gs_ctx* c, int slot, int prec, long long sites, long long hops,
                        double flops, double bytes);
gs_status prof_harvest(gs_ctx* c);

// BLAS-1 and Krylov kernels (blas.cu) ------------------------------------------
gs_status launch_bicg_init(gs_ctx* c, InnerWork& w, const double2* b, double2* x, int64_t n,
                           double tol);
gs_status launch_bicg_s_update(gs_ctx* c, InnerWork& w, double2* x, int64_t n);
gs_status launch_bicg_xr_update(gs_ctx* c, InnerWork& w, double2* x, int64_t n);
gs_status launch_bicg_p_update(gs_ctx* c, InnerWork& w, int64_t n);
// result[k] = <x_k, y> for k < nvec (x_k = X + k*ld), written to dev_out (complex)
gs_status launch_multidot(gs_ctx* c, RedScratch red, const double2* X, int64_t ld, int nvec,
                          const double2* y, int64_t n, double2* dev_out, int accumulate);
// y -= sum_k coef[k] x_k   (coef on the device); or y += if sign > 0
gs_status launch_multiaxpy(gs_ctx* c, const double2* X, int64_t ld, int nvec, const double2* coef,
                           double2* y, int64_t n, int sign);
// dev_out[0] = ||x||^2 (double)
gs_status launch_norm2(gs_ctx* c, RedScratch red, const double2* x, int64_t n, double* dev_out);
// y = a*x (a on host)
gs_status launch_scale_copy(gs_ctx* c, const double2* x, double2* y, int64_t n, double a);
gs_status launch_axpby(gs_ctx* c, double2 a, const double2* x, double2 b, double2* y, int64_t n);

// solvers (solver.cu) ---------------------------------------------------------
gs_status ensure_inner(gs_ctx* c, int64_t sites);
gs_status ensure_outer(gs_ctx* c, int64_t sites, int m);
// z = D_rr^-1 t for plan p (vectors of n_r = V - nb sites in label order r),
// dispatched on o.inner_prec to the FP64 BiCGStab or the mixed solve.
gs_status inner_solve(gs_ctx* c, const Plan* p, const double2* t, double2* z,
                      const gs_solve_opts& o, gs_solve_stats& st);
gs_status inner_solve_f64(gs_ctx* c, const Plan* p, const double2* t, double2* z,
                          const gs_solve_opts& o, gs_solve_stats& st);
gs_status inner_solve_mixed(gs_ctx* c, const Plan* p, const double2* t, double2* z,
                            const gs_solve_opts& o, gs_solve_stats& st);
void free_mixed(gs_ctx* c);
// low-precision tables of a set (compact neighbour table, 12-real links)
struct LowpTables {
    const int2* nbr;
    const void* links;
    int64_t n, nb;
    long long hops;
};
gs_status lowp_tables(gs_ctx* c, const Plan* p, int prec, LowpTables* out);
void free_multi(gs_ctx* c);
void free_net_ctx(gs_ctx* c);
gs_status lp_rr_apply_f32(gs_ctx* c, const Plan* p, const void* x, void* y);
size_t net_tc_weight_elems();
size_t net_phi_weight_elems();
size_t net_l1_weight_elems();
gs_status net_l1_pack(gs_ctx* c, const float2* WT, __nv_bfloat16* Bw);
gs_status net_l1_tc(gs_ctx* c, const float2* in, __nv_bfloat162* out, const __nv_bfloat16* Bw, const float2* U32,
                    const int2* nbr, int64_t V, int* err);
gs_status net_phi_pack(gs_ctx* c, const float2* WT, __nv_bfloat16* Bw);
gs_status net_phi_tc(gs_ctx* c, const float2* in, float2* phi, const __nv_bfloat16* Bw, int64_t V, int* err);
gs_status net_tc_pack(gs_ctx* c, const float2* WT, __nv_bfloat16* Bw);
gs_status net_conv_tc(gs_ctx* c, const __nv_bfloat162* in, float2* out, const __nv_bfloat16* Bw, const float2* U32,
                      const int2* nbr, int64_t V, int* err);
gs_status inner_fgmres_net(gs_ctx* c, const Plan* p, const double2* r, double2* e, double tol,
                           int m, int* iters_out);
void free_persist(gs_ctx* c);
gs_status persistent_bicg_f64(gs_ctx* c, const StencilArgs& A, const StencilArgs& C,
                              const double2* b, double2* x, InnerWork& w, int64_t n, double tol,
                              int maxit);
void invalidate_mixed_links(gs_ctx* c);
gs_status schur_apply_internal(gs_ctx* c, const Plan* p, const double2* xb, double2* yb,
                               const gs_solve_opts& o, gs_solve_stats& st);
gs_status outer_solve(gs_ctx* c, const Plan* p, const double2* wb, double2* xb,
                      const gs_solve_opts& o, gs_solve_stats& st);

int grid_for(int64_t n, int block, int max_blocks);

// failure-detection self-tests (persistent.cu, net_tc.cu): a bounded wait made
// to run out on purpose
gs_status selftest_grid_timeout(gs_ctx* c, gs_status* result);
gs_status selftest_mbar_timeout(gs_ctx* c, int* err_dev);

}  // namespace gs
