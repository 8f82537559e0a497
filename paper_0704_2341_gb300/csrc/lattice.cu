// Site permutations (Section 2 of the paper: "Permutation_block", coarse sites
// labelled first; Type I / Type II and their inverses), neighbour tables in
// label order, label-ordered link packing and the gather / scatter kernels that
// apply P and P^T to spinor fields.
#include <stdarg.h>

#include "gs_internal.cuh"

namespace gs {

gs_status set_err(gs_ctx* c, gs_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

int grid_for(int64_t n, int block, int max_blocks) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

struct Dims {
    int L[4];
};

__device__ __forceinline__ void site_coords(int64_t s, const Dims& d, int x[4]) {
    x[0] = (int)(s % d.L[0]);
    s /= d.L[0];
    x[1] = (int)(s % d.L[1]);
    s /= d.L[1];
    x[2] = (int)(s % d.L[2]);
    x[3] = (int)(s / d.L[2]);
}

__device__ __forceinline__ int64_t site_index(const int x[4], const Dims& d) {
    return x[0] + (int64_t)d.L[0] * (x[1] + (int64_t)d.L[1] * (x[2] + (int64_t)d.L[2] * x[3]));
}

// Label of site s in the stable coarse-first order p of the given type.
//   Type I : b = { every coordinate even }.  The number of b sites before s
//            in site order is counted digit by digit from the slowest
//            coordinate (x3) down, E(x) = (x + 1) / 2 even values below x.
//   Type II: b = { x_dir even }.  With s = a + Llo*(x_dir + L_dir*c), the b
//            sites before s are c*Llo*L_dir/2 + E(x_dir)*Llo (+ a if x_dir even).
// r sites keep their site order after the n_b coarse labels.
__global__ void k_build_labels(Dims d, int type, int dir, int64_t V, int64_t nb,
                               int32_t* __restrict__ perm, int32_t* __restrict__ label) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V;
         s += (int64_t)gridDim.x * blockDim.x) {
        int x[4];
        site_coords(s, d, x);
        int64_t lab;
        if (type == 0) {
            lab = s;
        } else {
            int64_t before;
            bool is_b;
            if (type == GS_TYPE_I) {
                const int64_t H0 = d.L[0] / 2, H1 = d.L[1] / 2, H2 = d.L[2] / 2;
                before = (int64_t)((x[3] + 1) / 2) * H2 * H1 * H0;
                if ((x[3] & 1) == 0) {
                    before += (int64_t)((x[2] + 1) / 2) * H1 * H0;
                    if ((x[2] & 1) == 0) {
                        before += (int64_t)((x[1] + 1) / 2) * H0;
                        if ((x[1] & 1) == 0) before += (x[0] + 1) / 2;
                    }
                }
                is_b = ((x[0] | x[1] | x[2] | x[3]) & 1) == 0;
            } else {
                int64_t Llo = 1;
                for (int nu = 0; nu < dir; ++nu) Llo *= d.L[nu];
                const int64_t Ld = d.L[dir];
                const int64_t a = s % Llo;
                const int64_t cblk = s / (Llo * Ld);
                const int xd = x[dir];
                before = cblk * Llo * (Ld / 2) + (int64_t)((xd + 1) / 2) * Llo;
                is_b = (xd & 1) == 0;
                if (is_b) before += a;
            }
            lab = is_b ? before : nb + (s - before);
        }
        label[s] = (int32_t)lab;
        if (lab >= 0 && lab < V) perm[lab] = (int32_t)s;  // guard: a wrong label never writes out of bounds
    }
}

// nbr[j][mu] = (label of perm[j] + mu, label of perm[j] - mu), periodic.
__global__ void k_build_nbr(Dims d, int64_t V, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ label, int2* __restrict__ nbr) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < V;
         j += (int64_t)gridDim.x * blockDim.x) {
        int x[4];
        const int32_t sj = perm[j];
        site_coords((sj >= 0 && sj < V) ? sj : 0, d, x);
        for (int mu = 0; mu < 4; ++mu) {
            int y[4] = {x[0], x[1], x[2], x[3]};
            y[mu] = (x[mu] + 1 == d.L[mu]) ? 0 : x[mu] + 1;
            const int32_t f = label[site_index(y, d)];
            y[mu] = (x[mu] == 0) ? d.L[mu] - 1 : x[mu] - 1;
            const int32_t b = label[site_index(y, d)];
            nbr[j * 4 + mu] = make_int2(f, b);
        }
    }
}

// hops[o][i] += number of (j, direction) with j in set o and its neighbour in
// set i (0 = b = labels below nb, 1 = r): the work counter of gs_profile.
__global__ void k_count_hops(int64_t V, int64_t nb, const int2* __restrict__ nbr,
                             unsigned long long* __restrict__ hops) {
    unsigned long long loc[4] = {0, 0, 0, 0};
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < V;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int o = j < nb ? 0 : 1;
        for (int mu = 0; mu < 4; ++mu) {
            const int2 n = nbr[j * 4 + mu];
            loc[o * 2 + (n.x < nb ? 0 : 1)] += 1;
            loc[o * 2 + (n.y < nb ? 0 : 1)] += 1;
        }
    }
    for (int q = 0; q < 4; ++q)
        if (loc[q]) atomicAdd(hops + q, loc[q]);
}

// links[j][mu][k] = -1/2 * U[perm[j]][mu][k]  (the factor is exact in binary)
__global__ void k_pack_links(int64_t V, const int32_t* __restrict__ perm,
                             const double2* __restrict__ U, double2* __restrict__ links) {
    const int64_t n = V * 36;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / 36;
        const int k = (int)(i % 36);
        const double2 u = U[(int64_t)perm[j] * 36 + k];
        links[i] = make_double2(-0.5 * u.x, -0.5 * u.y);
    }
}

// y[i] = x[perm[i]] per site (12 complex), and the transpose.
__global__ void k_gather(const int32_t* __restrict__ perm, const double2* __restrict__ x,
                         double2* __restrict__ y, int64_t nsites) {
    const int64_t n = nsites * kSiteC;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t site = i / kSiteC;
        const int c = (int)(i - site * kSiteC);
        y[i] = x[(int64_t)perm[site] * kSiteC + c];
    }
}

__global__ void k_scatter(const int32_t* __restrict__ perm, const double2* __restrict__ x,
                          double2* __restrict__ y, int64_t nsites) {
    const int64_t n = nsites * kSiteC;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t site = i / kSiteC;
        const int c = (int)(i - site * kSiteC);
        y[(int64_t)perm[site] * kSiteC + c] = x[i];
    }
}

static int64_t coarse_count(const int L[4], int type) {
    int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    if (type == GS_TYPE_I) return V / 16;
    if (type == GS_TYPE_II) return V / 2;
    return V;
}

void free_plan(Plan* p) {
    if (!p) return;
    cudaFree(p->perm);
    cudaFree(p->label);
    cudaFree(p->nbr);
    cudaFree(p->links);
    cudaFree(p->dtinv);
    delete p;
}

gs_status pack_plan_links(gs_ctx* c, Plan* p) {
    if (!c->have_gauge) return GS_OK;
    const int64_t n = c->V * 36;
    k_pack_links<<<grid_for(n, 256, c->num_sms * 16), 256, 0, c->stream>>>(c->V, p->perm, c->U_abi,
                                                                          p->links);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    p->links_ready = true;
    p->dtinv_ready = false;   // the Reusken block inverses depend on the links
    return GS_OK;
}

gs_status get_plan(gs_ctx* c, int type, int dir, int inverse, Plan** out) {
    if (type != 0 && type != GS_TYPE_I && type != GS_TYPE_II)
        return set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (type != GS_TYPE_II) dir = 0;
    if (type == 0) inverse = 0;
    inverse = inverse ? 1 : 0;
    if (type == GS_TYPE_II && (dir < 0 || dir > 3))
        return set_err(c, GS_EINVAL, "Type II direction %d not in 0..3", dir);
    if (type == GS_TYPE_I) {
        for (int mu = 0; mu < 4; ++mu)
            if (c->dims[mu] % 2)
                return set_err(c, GS_EINVAL, "Type I blocking needs even extents (L%d = %d)", mu,
                               c->dims[mu]);
    }
    if (type == GS_TYPE_II && c->dims[dir] % 2)
        return set_err(c, GS_EINVAL, "Type II blocking along %d needs an even extent (%d)", dir,
                       c->dims[dir]);
    for (Plan* p : c->plans)
        if (p->type == type && p->dir == dir && p->inverse == inverse) {
            *out = p;
            return GS_OK;
        }
    Plan* p = new Plan();
    p->type = type;
    p->dir = dir;
    p->inverse = inverse;
    p->nb = coarse_count(c->dims, type);
    const int64_t V = c->V;
    if (cudaMalloc(&p->perm, V * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&p->label, V * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&p->nbr, V * 4 * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&p->links, V * 36 * sizeof(double2)) != cudaSuccess) {
        free_plan(p);
        cudaGetLastError();
        return set_err(c, GS_ENOMEM, "allocating a permutation plan for V = %lld failed",
                       (long long)V);
    }
    Dims d;
    for (int mu = 0; mu < 4; ++mu) d.L[mu] = c->dims[mu];
    const int g = grid_for(V, 256, c->num_sms * 8);
    // zero the tables first: every entry is a valid site even if a label were missed
    if (cudaMemsetAsync(p->perm, 0, V * sizeof(int32_t), c->stream) != cudaSuccess ||
        cudaMemsetAsync(p->label, 0, V * sizeof(int32_t), c->stream) != cudaSuccess) {
        free_plan(p);
        cudaGetLastError();
        return set_err(c, GS_ECUDA, "clearing the permutation tables failed");
    }
    // the inverse order q = p^-1 is the label array of p, and vice versa
    int32_t* pp = inverse ? p->label : p->perm;
    int32_t* ll = inverse ? p->perm : p->label;
    k_build_labels<<<g, 256, 0, c->stream>>>(d, type, dir, V, p->nb, pp, ll);
    c->launches++;
    k_build_nbr<<<g, 256, 0, c->stream>>>(d, V, p->perm, p->label, p->nbr);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        free_plan(p);
        return set_err(c, GS_ECUDA, "building the permutation plan: %s", cudaGetErrorString(e));
    }
    {
        unsigned long long* dh = nullptr;
        unsigned long long hh[4] = {0, 0, 0, 0};
        if (cudaMalloc(&dh, sizeof hh) != cudaSuccess) {
            cudaGetLastError();
            free_plan(p);
            return set_err(c, GS_ENOMEM, "allocating the hop counters failed");
        }
        cudaMemsetAsync(dh, 0, sizeof hh, c->stream);
        k_count_hops<<<g, 256, 0, c->stream>>>(V, p->nb, p->nbr, dh);
        c->launches++;
        cudaMemcpyAsync(hh, dh, sizeof hh, cudaMemcpyDeviceToHost, c->stream);
        cudaError_t e2 = cudaStreamSynchronize(c->stream);
        cudaFree(dh);
        if (e2 != cudaSuccess) {
            free_plan(p);
            return set_err(c, GS_ECUDA, "counting hops: %s", cudaGetErrorString(e2));
        }
        for (int q = 0; q < 4; ++q) p->hops[q / 2][q % 2] = (long long)hh[q];
    }
    c->plans.push_back(p);
    gs_status s = pack_plan_links(c, p);
    if (s != GS_OK) return s;
    *out = p;
    return GS_OK;
}

// The same label order for a lattice of any extents (the coarse "lattices"
// of the V-cycle's lower levels): perm_dev / label_dev (int32 [V], device)
// receive p (or q = p^-1 when inverse) and its inverse, *nb_out the coarse
// count.  The extents blocked by the type must be even.
gs_status build_labels(gs_ctx* c, const int dims[4], int type, int dir, int inverse,
                       int32_t* perm_dev, int32_t* label_dev, int64_t* nb_out) {
    if (type != GS_TYPE_I && type != GS_TYPE_II)
        return set_err(c, GS_EINVAL, "unknown permutation type %d", type);
    if (type == GS_TYPE_I) {
        dir = 0;
        for (int mu = 0; mu < 4; ++mu)
            if (dims[mu] % 2)
                return set_err(c, GS_EINVAL, "Type I blocking needs even extents (L%d = %d)", mu, dims[mu]);
    } else {
        if (dir < 0 || dir > 3) return set_err(c, GS_EINVAL, "Type II direction %d not in 0..3", dir);
        if (dims[dir] % 2)
            return set_err(c, GS_EINVAL, "Type II blocking along %d needs an even extent (%d)", dir,
                           dims[dir]);
    }
    Dims d;
    for (int mu = 0; mu < 4; ++mu) d.L[mu] = dims[mu];
    const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    const int64_t nb = coarse_count(dims, type);
    GS_CUDA(c, cudaMemsetAsync(perm_dev, 0, V * sizeof(int32_t), c->stream));
    GS_CUDA(c, cudaMemsetAsync(label_dev, 0, V * sizeof(int32_t), c->stream));
    int32_t* pp = inverse ? label_dev : perm_dev;
    int32_t* ll = inverse ? perm_dev : label_dev;
    k_build_labels<<<grid_for(V, 256, c->num_sms * 8), 256, 0, c->stream>>>(d, type, dir, V, nb, pp, ll);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    *nb_out = nb;
    return GS_OK;
}

gs_status launch_gather(gs_ctx* c, const int32_t* perm, const double2* x, double2* y,
                        int64_t n) {
    if (n <= 0) return GS_OK;
    k_gather<<<grid_for(n * kSiteC, 256, c->num_sms * 16), 256, 0, c->stream>>>(perm, x, y, n);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

gs_status launch_scatter(gs_ctx* c, const int32_t* perm, const double2* x, double2* y,
                         int64_t n) {
    if (n <= 0) return GS_OK;
    k_scatter<<<grid_for(n * kSiteC, 256, c->num_sms * 16), 256, 0, c->stream>>>(perm, x, y, n);
    c->launches++;
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

}  // namespace gs
