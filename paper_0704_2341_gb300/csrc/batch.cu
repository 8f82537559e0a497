// Several problems -- lattices, permutations, sources -- solved at once.
//
// Every source of every problem is one work item, a single-source
// schur_solve (Section 1 of the paper: S_bb x_b = f_b - D_br D_rr^-1 f_r, then
// the back-substitution).  Items are handed out largest lattice first to a
// few lanes (host threads); a lane solves one item at a time on a context of
// the item's lattice, either the problem's own or a lane context that shares
// nothing with it but a copy of the gauge field (created on first need, kept
// for later calls, the field copied again when the problem's changes).
//
// GB300 design: one persistent cooperative solve on a large lattice streams
// at ~0.6 of HBM bandwidth and spends the rest waiting at its grid barriers;
// a few solves side by side fill those gaps (24^3 x 48, FP32 inner: 5.87 s per
// solve alone, 5.49 / 5.31 / 5.26 / 5.32 s with 2 / 3 / 4 / 6 at once, so four
// lanes by default).  The cooperative grids of the running solves are drawn
// from one block ledger (BlockLedger): every persistent solver kernel has the
// same block footprint (128 threads, 168 registers), a grid is granted only
// from blocks no other solve holds, so all of them stay co-resident, and the
// blocks a finished solve frees go to the next launches of the others.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "gs_internal.cuh"

using namespace gs;

namespace {

constexpr int kBatchLanes = 4;

// the k-th lane context of parent (k >= 1), created or brought up to date:
// same lattice, mass and options, the parent's current field, its own stream
gs_status lane_context(gs_ctx* parent, size_t k, gs_ctx** out, std::string* msg) {
    while (parent->lanes.size() < k) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            *msg = "creating a lane stream failed";
            return GS_ECUDA;
        }
        gs_ctx* ch = nullptr;
        const gs_status s = gs_create(&ch, parent->dims, parent->m0, st);
        if (s != GS_OK) {
            cudaStreamDestroy(st);
            *msg = "creating a lane context failed";
            return s;
        }
        ch->own_stream = st;
        parent->lanes.push_back(ch);
    }
    if (!parent->have_gauge) {
        *msg = "no gauge field set";
        return GS_ENOGAUGE;
    }
    gs_ctx* ch = parent->lanes[k - 1];
    if (ch->opt_stencil_variant != parent->opt_stencil_variant)
        gs_set_option(ch, GS_OPT_STENCIL_VARIANT, parent->opt_stencil_variant);
    ch->opt_inner_kernel = parent->opt_inner_kernel;
    ch->opt_net_kernel = parent->opt_net_kernel;
    ch->opt_multi_batch = parent->opt_multi_batch;
    ch->wait_ns = parent->wait_ns;
    if (!ch->have_gauge || ch->lane_gauge_gen != parent->gauge_gen) {
        const gs_status s = gs_set_gauge(ch, parent->U_abi);
        if (s != GS_OK) {
            *msg = "copying the field to a lane context failed: " + ch->err;
            return s;
        }
        ch->lane_gauge_gen = parent->gauge_gen;
    }
    *out = ch;
    return GS_OK;
}

void merge_stats(gs_solve_stats& a, const gs_solve_stats& b) {
    a.outer_iters = std::max(a.outer_iters, b.outer_iters);
    a.inner_solves += b.inner_solves;
    a.inner_iters += b.inner_iters;
    a.inner_max_seen = std::max(a.inner_max_seen, b.inner_max_seen);
    a.outer_residual = std::max(a.outer_residual, b.outer_residual);
    a.true_residual = std::max(a.true_residual, b.true_residual);
    a.inner_residual = std::max(a.inner_residual, b.inner_residual);
    a.stencil_sites += b.stencil_sites;
    a.kernel_launches += b.kernel_launches;
    a.lowp_cycles += b.lowp_cycles;
    a.lowp_fallbacks += b.lowp_fallbacks;
}

gs_status worse(gs_status a, gs_status b) {
    return (b != GS_OK && (a == GS_OK || a == GS_MAXITER)) ? b : a;
}

}  // namespace

namespace gs {

void ledger_enter(BlockLedger* L, const gs_ctx* c) {
    std::lock_guard<std::mutex> lk(L->mu);
    L->held.push_back({c, 0, false});
    L->running.fetch_add(1);
}

void ledger_leave(BlockLedger* L, const gs_ctx* c) {
    {
        std::lock_guard<std::mutex> lk(L->mu);
        for (size_t k = 0; k < L->held.size(); ++k)
            if (L->held[k].ctx == c) {
                L->held.erase(L->held.begin() + (long)k);
                break;
            }
        L->running.fetch_sub(1);
    }
    L->cv.notify_all();
}

int64_t ledger_grant(gs_ctx* c, int per_sm, int64_t want, int64_t target) {
    BlockLedger* L = c->ledger;
    const int64_t capacity = (int64_t)per_sm * c->num_sms;
    int64_t limit = want < target ? want : target;
    if (limit < 1) limit = 1;
    std::unique_lock<std::mutex> lk(L->mu);
    BlockLedger::Entry* mine = nullptr;
    for (auto& e : L->held)
        if (e.ctx == c) mine = &e;
    if (!mine) return 0;
    const auto t0 = std::chrono::steady_clock::now();
    const auto bound = std::chrono::nanoseconds((long long)(c->wait_ns > 0 ? c->wait_ns : 1000000000ull) * 60);
    for (;;) {
        // held: blocks that may be in flight now; claimed: the same with
        // every solve that has not launched yet counted at the reserve
        int64_t held = 0, claimed = 0;
        for (const auto& e : L->held)
            if (e.ctx != c) {
                held += e.blocks;
                claimed += e.launched ? e.blocks : (e.blocks > L->reserve ? e.blocks : L->reserve);
            }
        int64_t g = limit < capacity - claimed ? limit : capacity - claimed;
        if (g < 1) g = limit < capacity - held ? limit : capacity - held;
        if (g >= 1) {
            mine->blocks = g;
            mine->launched = true;
            L->cv.notify_all();   // a solve waiting for blocks may find some now
            return g;
        }
        // every block is held by the others' kernels in flight: one of them
        // ends or shrinks at its next launch
        if (std::chrono::steady_clock::now() - t0 > bound) return 0;
        L->cv.wait_for(lk, std::chrono::milliseconds(1));
        for (auto& e : L->held)
            if (e.ctx == c) mine = &e;
    }
}

}  // namespace gs

extern "C" {

gs_status schur_solve_batched(int nprob, gs_ctx* const* ctxs, const int* type, const int* dir,
                              const int* inverse, const int* nrhs, const void* const* f_dev,
                              void* const* x_dev, const gs_solve_opts* opts, gs_solve_stats* stats) {
    if (nprob < 1 || !ctxs || !type || !dir || !inverse || !nrhs || !f_dev || !x_dev) return GS_EINVAL;
    for (int i = 0; i < nprob; ++i) {
        if (!ctxs[i]) return GS_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return set_err(ctxs[i], GS_EINVAL, "schur_solve_batched: problems %d and %d "
                                                                       "share a context", j, i);
        if (nrhs[i] < 1) return set_err(ctxs[i], GS_EINVAL, "schur_solve_batched: nrhs %d < 1", nrhs[i]);
        if (!f_dev[i] || !x_dev[i]) return set_err(ctxs[i], GS_EINVAL, "schur_solve_batched: null vector");
    }
    struct Item {
        int prob, src;
    };
    std::vector<Item> items;
    for (int i = 0; i < nprob; ++i)
        for (int j = 0; j < nrhs[i]; ++j) items.push_back({i, j});
    std::stable_sort(items.begin(), items.end(),
                     [&](const Item& a, const Item& b) { return ctxs[a.prob]->V > ctxs[b.prob]->V; });
    int lanes = ctxs[0]->opt_batch_lanes > 0 ? ctxs[0]->opt_batch_lanes : kBatchLanes;
    if (lanes > (int)items.size()) lanes = (int)items.size();
    // the network preconditioner is attached to the problem's own context only
    const bool net = opts && opts->inner_solver == GS_INNER_FGMRES_NET;
    const int per_prob = net ? 1 : lanes;
    // lane contexts read the inputs and the field on their own streams: drain
    // the callers' streams first
    for (int i = 0; i < nprob; ++i)
        if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) {
            const cudaError_t e = cudaGetLastError();
            return set_err(ctxs[i], GS_ECUDA, "schur_solve_batched: %s", cudaGetErrorString(e));
        }

    std::mutex mu;
    std::condition_variable cv;
    std::vector<char> taken(items.size(), 0);
    std::vector<std::vector<char>> busy(nprob, std::vector<char>(per_prob, 0));
    std::vector<gs_status> res(nprob, GS_OK);
    std::vector<gs_solve_stats> sts(nprob);
    for (auto& s : sts) memset(&s, 0, sizeof s);
    std::vector<std::string> msg(nprob);
    BlockLedger ledger;
    // a solve that has not launched yet is counted at a third of an even
    // share of the co-resident blocks (one block per SM share at 3 per SM)
    ledger.reserve = std::max(1, ctxs[0]->num_sms / std::max(1, lanes));
    size_t left = items.size();

    auto lane = [&]() {
        for (;;) {
            size_t it = items.size();
            int slot = -1;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (left == 0) return;
                    for (size_t q = 0; q < items.size() && it == items.size(); ++q) {
                        if (taken[q]) continue;
                        auto& b = busy[items[q].prob];
                        for (int k = 0; k < per_prob; ++k)
                            if (!b[k]) {
                                it = q;
                                slot = k;
                                break;
                            }
                    }
                    if (it < items.size()) break;
                    cv.wait(lk);
                }
                taken[it] = 1;
                --left;
                busy[items[it].prob][slot] = 1;
            }
            const int i = items[it].prob, j = items[it].src;
            gs_ctx* c = ctxs[i];
            gs_status s = GS_OK;
            std::string m;
            if (slot > 0) {
                std::lock_guard<std::mutex> lk(mu);   // lane contexts of a problem are created one at a time
                s = lane_context(ctxs[i], (size_t)slot, &c, &m);
            }
            gs_solve_stats sj;
            memset(&sj, 0, sizeof sj);
            if (s == GS_OK) {
                const size_t off = (size_t)j * ctxs[i]->V * kSiteC;
                const int old_cap = c->coop_block_cap;
                c->coop_block_cap = ctxs[i]->opt_coop_blocks;
                if (lanes > 1) {
                    ledger_enter(&ledger, c);
                    c->ledger = &ledger;
                }
                s = schur_solve(c, type[i], dir[i], inverse[i], (const double2*)f_dev[i] + off,
                                (double2*)x_dev[i] + off, opts, &sj);
                if (cudaStreamSynchronize(c->stream) != cudaSuccess && s == GS_OK) {
                    const cudaError_t e = cudaGetLastError();
                    s = set_err(c, GS_ECUDA, "schur_solve_batched: %s", cudaGetErrorString(e));
                }
                if (lanes > 1) {
                    c->ledger = nullptr;
                    ledger_leave(&ledger, c);
                }
                c->coop_block_cap = old_cap;
                if (s != GS_OK && s != GS_MAXITER && c != ctxs[i]) m = c->err;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                busy[i][slot] = 0;
                merge_stats(sts[i], sj);
                if (s != GS_OK && s != GS_MAXITER && msg[i].empty()) msg[i] = m.empty() ? "-" : m;
                res[i] = worse(res[i], s);
            }
            cv.notify_all();
        }
    };
    std::vector<std::thread> th;
    for (int l = 0; l < lanes; ++l) th.emplace_back(lane);
    for (auto& t : th) t.join();

    gs_status worst = GS_OK;
    for (int i = 0; i < nprob; ++i) {
        sts[i].status = res[i];
        if (stats) stats[i] = sts[i];
        // an error met on a lane context is reported on the problem's own
        if (!msg[i].empty() && msg[i] != "-") set_err(ctxs[i], res[i], "%s", msg[i].c_str());
        worst = worse(worst, res[i]);
    }
    return worst;
}

}  // extern "C"
