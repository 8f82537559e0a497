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
#include "dslash_f64.cuh"

namespace gs {

namespace {

template <int EPI>
__global__ void __launch_bounds__(kThreads) k_dslash_f64(StencilArgs a) {
    const bool skip = a.st != nullptr && a.st->done;
    if (a.ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.ran = skip ? 0 : 1;
    if (skip) return;
    __shared__ double red[4][24][kSitesPerBlock];
    __shared__ double bred[4][kMaxRedVals];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    double e[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // epilogue partial sums

    for (int64_t base = (int64_t)blockIdx.x * kSitesPerBlock; base < a.n_out;
         base += (int64_t)gridDim.x * kSitesPerBlock)
        f64_tile<EPI>(a, base, kSitesPerBlock, red, e);
    double e0 = e[0], e1 = e[1], e2 = e[2];

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
