/*
 * gschur.h -- C ABI of the GB300 library for the gauged renormalisation-group
 * step of lattice Wilson fermions: the Schur complement
 *
 *     S_bb = D_bb - D_br D_rr^-1 D_rb
 *
 * of the SU(3) Wilson-Dirac operator D after a site permutation puts the
 * coarse sites b first (Boric, "On Gauged Renormalisation Group
 * Transformations of Lattice Fermions", Section 1: the 2x2 partition, the
 * Schur complement and its block UL factorisation; Section 2: the Type I /
 * Type II permutations and their inverses).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: extents dims[4] = {L0, L1, L2, L3}, periodic; site index
 *   s = x0 + L0*(x1 + L1*(x2 + L2*x3))   (x0 fastest).
 * Gauge field: complex128 (interleaved re, im doubles) [V][4][3][3];
 *   element [s][mu][a][b] is row a, column b of U_mu(x), the link from s to
 *   s + mu-hat.
 * Spinors: complex128 [n_sites][4][3] ([site][spin][colour]), 192 bytes a
 *   site.  "Site order" = the lattice order above; "label order" = the order
 *   of the permuted operator P D P^T, entry i being the site perm[i].
 *   Vectors on the coarse set b are the first n_b labels; vectors on the rest
 *   r are labels n_b .. V-1.
 * Operator (Wilson parameter r = 1, gamma matrices in the DeGrand-Rossi
 *   chiral basis, gamma_5 = diag(1, 1, -1, -1), direction mu <-> gamma_{mu+1}):
 *   (D psi)(x) = (m0 + 4) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                   + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ].
 * Permutations (p lists the label order; (P x)_i = x_{p(i)}):
 *   GS_TYPE_I : b = sites with every coordinate even (n_b = V/16), stable.
 *   GS_TYPE_II: b = sites with x_dir even (n_b = V/2), stable; one
 *               direction per renormalisation step.
 *   inverse != 0 uses q = p^-1 (operator P^T) with the same n_b.
 *
 * Memory: every pointer argument named *_dev is a device pointer owned by
 * the caller (any allocator, e.g. PyTorch); the library never frees it and
 * does not keep it past the call.  The library owns the context's own device
 * memory (index tables, packed links, solver workspaces).
 * Streams: all work is enqueued on the stream given to gs_create (a
 * cudaStream_t passed as void*; NULL = the legacy default stream).  Calls
 * that return solver statistics synchronise that stream; the others are
 * asynchronous.
 * Errors: every call returns a gs_status; GS_OK is 0.  On failure
 * gs_last_error() describes the cause.  No call aborts the process.
 * A context is not thread-safe; use one context per host thread.
 */
#ifndef GSCHUR_H
#define GSCHUR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_ctx gs_ctx;

typedef enum {
    GS_OK = 0,
    GS_EINVAL = 1,     /* bad argument (sizes, type, null pointer, odd extent) */
    GS_ENOMEM = 2,     /* device or host allocation failed */
    GS_MAXITER = 3,    /* solver stopped at its iteration limit; result = last iterate */
    GS_BREAKDOWN = 4,  /* Krylov breakdown (a zero inner product) */
    GS_NONFINITE = 5,  /* NaN or Inf met in a solver scalar */
    GS_TIMEOUT = 6,    /* a bounded device-side wait gave up */
    GS_ECUDA = 7,      /* a CUDA runtime call failed */
    GS_ENOGAUGE = 8,   /* no gauge field set yet */
    GS_ETOOLARGE = 9   /* lattice larger than wilson_apply_noalloc's static scratch */
} gs_status;

enum { GS_TYPE_I = 1, GS_TYPE_II = 2 };
enum { GS_F64 = 0, GS_F32 = 1, GS_BF16 = 2 };
enum { GS_GMRES = 0, GS_BICGSTAB = 1 };
enum { GS_INNER_BICGSTAB = 0, GS_INNER_FGMRES_NET = 1 };

/* Options of schur_apply / schur_solve.  gs_default_opts fills the defaults
 * in brackets. */
typedef struct {
    double tol;            /* outer: relative residual ||w_b - S_bb x_b|| / ||w_b|| [1e-10] */
    int    max_iter;       /* outer: Arnoldi / BiCGStab steps in total [3000] */
    int    restart;        /* GMRES(m) restart length m, 1..64 [30] */
    int    outer_solver;   /* GS_GMRES or GS_BICGSTAB [GS_GMRES] */
    double inner_tol;      /* inner: ||t - D_rr z|| / ||t|| for each D_rr^-1 [1e-12] */
    int    inner_max_iter; /* inner: BiCGStab iterations per solve [5000] */
    int    inner_prec;     /* inner D_rr solve: GS_F64 (plain BiCGStab), or GS_F32 /
                            * GS_BF16: FP64 defect correction around a BiCGStab with
                            * FP32 arithmetic and FP32 / BF16 storage (12-real links);
                            * the result meets inner_tol in FP64 either way [GS_F64] */
    int    check_every;    /* inner iterations queued ahead of the convergence read-back, 1..4 [2] */
    double lowp_tol;       /* relative tolerance of each low-precision solve; 0 = 1e-5
                            * for GS_F32, 3e-2 for GS_BF16 [0] */
    int    inner_relax;    /* outer GMRES: relax the inner tolerance of Arnoldi step j to
                            * inner_tol * ||w_b|| / ||r_j|| (at most relax_cap), accepting
                            * the solve only on a tightly recomputed true residual [1] */
    double relax_cap;      /* largest relaxed inner tolerance [1e-4] */
    int    inner_solver;   /* low-precision stage of the mixed inner solve: GS_INNER_BICGSTAB,
                            * or GS_INNER_FGMRES_NET = flexible GMRES(inner_restart) with the
                            * network attached by gs_set_net as right preconditioner, run in
                            * FP32 (basis vectors, D_rr stencil, products; dot-product sums
                            * in FP64); each pass reduces the residual by lowp_tol and the
                            * FP64 true residual is recomputed after it
                            * [GS_INNER_BICGSTAB] */
    int    inner_restart;  /* Krylov steps of one FGMRES-with-network pass, 1..64 [16] */
} gs_solve_opts;

/* Statistics written by schur_apply / schur_solve (may be NULL). */
typedef struct {
    int       status;          /* gs_status of the call */
    int       outer_iters;     /* Arnoldi (or BiCGStab) steps of the outer solve */
    int       inner_solves;    /* number of D_rr^-1 applications */
    long long inner_iters;     /* BiCGStab iterations summed over inner solves */
    int       inner_max_seen;  /* largest single inner iteration count */
    double    outer_residual;  /* final ||w_b - S_bb x_b|| / ||w_b|| (recursive estimate) */
    double    true_residual;   /* schur_solve: ||f - D x|| / ||f|| recomputed in FP64 */
    double    inner_residual;  /* largest final inner relative residual seen */
    long long stencil_sites;   /* output sites of all stencil launches (work counter) */
    long long kernel_launches; /* kernels enqueued by the call */
    long long lowp_cycles;     /* defect-correction cycles of the mixed inner solves */
    long long lowp_fallbacks;  /* mixed inner solves finished by the FP64 BiCGStab */
} gs_solve_stats;

/* Create a context for a dims[0] x dims[1] x dims[2] x dims[3] periodic
 * lattice with bare mass m0 (kappa = 1/(2 m0 + 8)).  Every extent must be
 * >= 2; V must be < 2^31 / 12.  stream: a cudaStream_t or NULL. */
gs_status gs_create(gs_ctx** ctx_out, const int dims[4], double m0, void* stream);

/* Release every device and host resource of the context (NULL is a no-op). */
gs_status gs_destroy(gs_ctx* ctx);

/* Copy the gauge field U_dev (complex128 [V][4][3][3], site order) into the
 * context's packed link arrays.  U_dev is read during the call only.  Any
 * permutation plan built before is repacked. */
gs_status gs_set_gauge(gs_ctx* ctx, const void* U_dev);

/* Context options.
 * GS_OPT_STENCIL_VARIANT selects the low-precision stencil kernel: 0 = chosen
 * by the library's autotuner per set and precision (the default: every
 * variant is timed with CUDA events when a set is first used), 1 = one
 * thread per site (all eight hops in registers), 3 / 4 = the same with a
 * register budget for 6 / 8 blocks of 128 threads per SM, 2 = one warp per
 * direction (four partial sums combined in shared memory), 5 / 6 = one thread
 * per site with the next direction's operands loaded while the current one
 * is computed (register budget for 3 / 4 blocks per SM).  gs_get_option
 * returns the forced value, or under autotuning the variant chosen most
 * recently. */
enum { GS_OPT_STENCIL_VARIANT = 1, GS_OPT_INNER_KERNEL = 2, GS_OPT_NET_KERNEL = 3, GS_OPT_MULTI_BATCH = 4,
       GS_OPT_WAIT_LIMIT_US = 5, GS_OPT_COOP_BLOCKS = 6, GS_OPT_BATCH_LANES = 7 };
/* GS_OPT_INNER_KERNEL: 0 = each inner BiCGStab solve runs as one persistent
 * cooperative kernel (grid barriers with bounded waits between its phases;
 * the default), 1 = five kernel launches per iteration with the convergence
 * flag read back while iterations are queued.
 * GS_OPT_NET_KERNEL: 0 = the contractions of a 24-channel network (1 -> C,
 * C -> C, and the weights-first half of C -> 1) run on the tensor cores
 * (tcgen05.mma, BF16 operands: the transported activations are rounded to
 * BF16 as well as the weights; FP32 accumulation; the default), 1 = every
 * layer on the CUDA cores (FP32 activations, BF16 weights).
 * GS_OPT_MULTI_BATCH: how schur_solve_multi (and schur_solve_batched per
 * problem) shapes its work: 0 = the sources of a problem share every launch
 * when the rest set has at most 16384 sites, where one source leaves the GPU
 * latency bound, else they are solved one at a time by the single-source
 * solver (the default); 1 = always together; 2 = always one at a time.
 * GS_OPT_WAIT_LIMIT_US: the bound, in microseconds (1 .. 60000000), on every
 * device-side wait of the context's kernels -- the grid barriers of the
 * persistent solvers and the mbarrier waits of the tensor-core network
 * kernels [1000000, i.e. 1 s].  A wait that runs out makes its kernel stop,
 * release what it holds (tensor memory) and report GS_TIMEOUT; the context
 * stays usable.
 * GS_OPT_COOP_BLOCKS: the number of blocks the persistent (cooperative)
 * solver kernels of this problem use while schur_solve_batched runs several
 * solves at once (the caller then keeps their sum within what the GPU holds
 * at once); 0 = granted at each launch by the call's block ledger (the
 * default): on rest sets of at most 16384 sites one pass over the set (FP64:
 * one round of 32-site tiles; FP32 / BF16: about 96 sites per block), above
 * that an even share of the co-resident blocks among the running solves,
 * never more than the other solves leave free.
 * GS_OPT_BATCH_LANES (read from the first problem's context): how many solves
 * schur_solve_batched runs at once, 1 .. 64; 0 = four (the default). */
gs_status gs_set_option(gs_ctx* ctx, int option, int value);
gs_status gs_get_option(gs_ctx* ctx, int option, int* value);

/* Failure-detection self-test of the bounded device waits (the paper has no
 * counterpart).  which = 0: a two-block cooperative kernel in which one block
 * never arrives at the persistent solvers' grid barrier; which = 1: one
 * thread waits on an mbarrier that nothing arrives at.  Either wait runs out
 * after the context's GS_OPT_WAIT_LIMIT_US, the kernel returns, and the call
 * returns GS_TIMEOUT (the intended outcome; gs_last_error says so).  No fault
 * and no hang: every wait involved is bounded.  Synchronises the stream. */
gs_status gs_selftest_wait(gs_ctx* ctx, int which);

/* Fill opts with the defaults listed in gs_solve_opts. */
void gs_default_opts(gs_solve_opts* opts);

/* y = D x on the full lattice, site order (the Wilson-Dirac operator above,
 * the operator the paper blocks).  x_dev, y_dev: complex128 [V][4][3]; must
 * not overlap.  Asynchronous. */
gs_status wilson_apply(gs_ctx* ctx, const void* x_dev, void* y_dev);

/* Site permutation of Section 2 ("Permutation_block": P(p) exchanges the
 * rows of D, coarse sites labelled first).
 *   transpose == 0: y = P x,   y[i] = x[perm[i]]   (site order -> label order)
 *   transpose != 0: y = P^T x, y[perm[i]] = x[i]   (label order -> site order)
 * perm is p (inverse == 0) or q = p^-1 (inverse != 0) of the given type and
 * direction (dir is used by GS_TYPE_II only, 0..3).  x_dev, y_dev: complex128
 * [V][4][3], not overlapping.  *n_b_out (may be NULL) receives n_b.
 * Asynchronous. */
gs_status permute_sites(gs_ctx* ctx, int type, int dir, int inverse, int transpose,
                        const void* x_dev, void* y_dev, int64_t* n_b_out);

/* The label order itself: perm_dev (int32 [V], device) receives perm, i.e.
 * perm_dev[i] = the site at label i.  *n_b_out (may be NULL) receives n_b.
 * Asynchronous. */
gs_status gs_get_permutation(gs_ctx* ctx, int type, int dir, int inverse,
                             int32_t* perm_dev, int64_t* n_b_out);

/* y_b = S_bb x_b = D_bb x_b - D_br D_rr^-1 D_rb x_b (Section 1), with the
 * inner D_rr^-1 taken by BiCGStab to opts->inner_tol.  xb_dev, yb_dev:
 * complex128 [n_b][4][3] in label order, not overlapping.  Synchronises the
 * stream (inner convergence).  Returns GS_MAXITER if the inner solve did not
 * converge (y_b then uses its last iterate). */
gs_status schur_apply(gs_ctx* ctx, int type, int dir, int inverse,
                      const void* xb_dev, void* yb_dev,
                      const gs_solve_opts* opts, gs_solve_stats* stats);

/* Solve D x = f through the block UL factorisation of Section 1:
 *   w_b = f_b - D_br D_rr^-1 f_r,   S_bb x_b = w_b (outer GMRES(m) or
 *   BiCGStab),   x_r = D_rr^-1 (f_r - D_rb x_b).
 * f_dev, x_dev: complex128 [V][4][3] in site order, not overlapping; x_dev
 * receives the solution.  stats->true_residual is ||f - D x|| / ||f|| in
 * FP64.  Synchronises the stream. */
gs_status schur_solve(gs_ctx* ctx, int type, int dir, int inverse,
                      const void* f_dev, void* x_dev,
                      const gs_solve_opts* opts, gs_solve_stats* stats);

/* y = D x on the full lattice, like wilson_apply, for callers that cannot
 * allocate device memory: a service whose device memory is all handed out by
 * its own pool allocator, or one that cannot afford the device-wide
 * synchronisation cudaFree implies.  It needs no context and allocates
 * nothing.  The paper has no counterpart; it is the same operator and the
 * same stencil kernel as wilson_apply.
 *
 * U_dev: complex128 [V][4][3][3] (site order), x_dev, y_dev: complex128
 * [V][4][3] (site order, not overlapping), all caller-owned device memory;
 * stream: a cudaStream_t or NULL.  Asynchronous.
 *
 * Scratch: the stencil's neighbour table and packed links are written into
 * one static device array of 4.75 MiB (room for V <= 8192 sites, e.g. 8^4),
 * which every GPU that loads the library holds until the process exits.
 * Larger lattices return GS_ETOOLARGE.  Every call overwrites the whole
 * table it uses, so no state carries over between calls; but all calls on a
 * device share the one array, so calls whose GPU work overlaps (e.g. on two
 * streams at once) race.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) in the current device's context; the first call on a
 * device also loads the library's module there, so make that first call
 * before any stream capture.  Undersized buffers are not detected here: the
 * caller guarantees the sizes above (the Python binding checks them). */
gs_status wilson_apply_noalloc(const int dims[4], double m0, const void* U_dev,
                               const void* x_dev, void* y_dev, void* stream);

/* Live timing of the Wilson stencil kernels (the dominant kernels of every
 * entry point above).  While enabled, each stencil launch is bracketed by two
 * CUDA events on the context's stream and its algorithmic work is counted:
 *   hops  = neighbour terms whose input site lies in the launch's input range,
 *   flops = 168 per hop (spin projection 12, two SU(3) x colour-vector
 *           products 132, reconstruction 24) + 48 per site with a diagonal
 *           (m0 + 4) term (FP64 flops, an FMA counting 2),
 *   bytes = 192 per output site + 192 per input site of the ranges read
 *           + 144 per link used (hops / 2 when both ends are outputs, else
 *           one per hop) + 192 per output site of an addend, each datum once.
 * gs_profile(ctx, 1) resets the counters and starts timing; gs_profile(ctx, 0)
 * stops it.  gs_profile_read synchronises the stream and returns the totals. */
typedef struct {
    long long launches;  /* stencil launches timed */
    double    ms;        /* summed event-to-event durations of those launches */
    long long sites;     /* output sites */
    long long hops;      /* in-range neighbour terms */
    double    flops;     /* algorithmic flops as defined above */
    double    bytes;     /* algorithmic bytes as defined above */
} gs_kernel_profile;

gs_status gs_profile(gs_ctx* ctx, int enable);
/* family: GS_PROF_STENCIL_F64 (k_dslash_f64), GS_PROF_STENCIL_F32 /
 * GS_PROF_STENCIL_BF16 (the low-precision stencil; bytes use 96 / 48 B per
 * spinor and 48 / 24 B per 12-real link), GS_PROF_SOLVER_F64 /
 * GS_PROF_SOLVER_LP (the persistent BiCGStab kernels: per launch, two D_rr
 * applications and 84 flop per complex entry of vector updates per
 * iteration; "sites" counts stencil output sites). */
enum { GS_PROF_STENCIL_F64 = 0, GS_PROF_STENCIL_F32 = 1, GS_PROF_STENCIL_BF16 = 2,
       GS_PROF_SOLVER_F64 = 3, GS_PROF_SOLVER_LP = 4 };
gs_status gs_profile_read(gs_ctx* ctx, int family, gs_kernel_profile* out);
/* The timed launches of a family as intervals: out[2 i], out[2 i + 1] = start
 * and end of launch i, in ms since a per-device origin common to every
 * context of the process (so the intervals of concurrent contexts can be
 * merged); up to cap doubles are written, *n_out receives the number of
 * launches recorded since profiling was enabled.  Synchronises the stream. */
gs_status gs_profile_timeline(gs_ctx* ctx, int family, double* out, int cap, int* n_out);
/* SM clock cycles that block 0 of the persistent FP64 BiCGStab spent in each
 * phase of its iterations while profiling was on (summed over launches):
 * out[3 s + 0] = work of step s (s = 0: v = D p and <rhat, v>; 1: s = r - a v
 * and ||s||^2; 2: t = D s, <t, s>, <t, t>, <rhat, t>; 3: the x, r and p
 * updates and ||r||^2; 4: unused, 0), out[3 s + 1] = its grid barrier,
 * out[3 s + 2] = the reduction of the per-block partials and the scalar
 * algebra after it.  n >= 15.  A diagnostic of where an iteration's time
 * goes; synchronises. */
gs_status gs_profile_phases(gs_ctx* ctx, double* out, int n);

/* The FP64 peak of this GPU as measured here (the denominator of the FP64
 * rooflines): a kernel of 8 independent FMA chains per thread on 8 blocks of
 * 256 threads per SM, timed with CUDA events on the context's stream, the
 * fastest of 5 launches after one warm-up; *tflops_out = 2 x FMAs / time, in
 * TFLOP/s.  Synchronises the stream. */
gs_status gs_fp64_peak(gs_ctx* ctx, double* tflops_out);

/* Low-precision vectors and stencil: the arithmetic of the mixed inner solve
 * (GS_F32 / GS_BF16 storage, FP32 arithmetic, links stored as two rows of
 * -1/2 U with the third row rebuilt as the SU(3) cross product).
 * Set: type == 0 is the whole lattice in site order (n = V, operator D);
 * GS_TYPE_I / GS_TYPE_II (with dir, inverse) is the rest set r of that
 * permutation in label order (n = V - n_b, operator D_rr of Section 1).
 * A low-precision vector of n sites holds each site's 24 reals
 * ([spin][colour][re, im]) component-major in 16-byte groups:
 *   GS_F32 : float  [6][n][4]  (group g holds reals 4g .. 4g+3), n x 96 bytes;
 *   GS_BF16: bf16   [3][n][8]  (group g holds reals 8g .. 8g+7), n x 48 bytes.
 * gs_lowp_pack rounds a complex128 [n][4][3] vector to that layout,
 * gs_lowp_unpack widens it back; wilson_apply_lowp computes y = D x (or
 * D_rr x) in FP32 arithmetic.  Caller-owned device buffers, not overlapping.
 * Asynchronous. */
gs_status gs_lowp_pack(gs_ctx* ctx, int type, int dir, int inverse, int prec,
                       const void* x_dev, void* x_lp_dev);
gs_status gs_lowp_unpack(gs_ctx* ctx, int type, int dir, int inverse, int prec,
                         const void* x_lp_dev, void* x_dev);
gs_status wilson_apply_lowp(gs_ctx* ctx, int type, int dir, int inverse, int prec,
                            const void* x_lp_dev, void* y_lp_dev);

/* Several sources on one lattice (nrhs = 1..32), solved together: the
 * block UL solve of schur_solve for every source, with the inner D_rr solves
 * of all sources in one persistent low-precision kernel (opts->inner_prec
 * must be GS_F32 or GS_BF16; FP64 defect correction as in schur_solve) and the
 * outer GMRES(m) systems advanced in lock step (one batched S_bb
 * application per Arnoldi step).  f_dev, x_dev: complex128
 * [nrhs][V][4][3], site order.  stats (may be NULL) aggregates: iterations
 * summed, true_residual and outer_residual the worst over the sources.
 * Whether the sources actually share launches is set by GS_OPT_MULTI_BATCH
 * (by default only on rest sets of at most 16384 sites; larger problems are
 * solved one source at a time with the same options and results to the same
 * tolerance).  Synchronises the stream. */
gs_status schur_solve_multi(gs_ctx* ctx, int type, int dir, int inverse, int nrhs,
                            const void* f_dev, void* x_dev, const gs_solve_opts* opts,
                            gs_solve_stats* stats);

/* Several problems -- lattices with their own contexts, permutations and
 * source counts -- solved at once (Section 1 of the paper for each source).
 * Problem i solves D x = f for the nrhs[i] sources f_dev[i] (complex128
 * [nrhs[i]][V][4][3], site order) into x_dev[i] through S_bb of permutation
 * (type[i], dir[i], inverse[i]) on the lattice of ctxs[i], with opts (any
 * inner precision).  Every source is one schur_solve; the solves go largest
 * lattice first to GS_OPT_BATCH_LANES concurrent lanes, each on a context of
 * the source's lattice: the problem's own, or a lane context the library
 * creates with its own stream and a copy of the problem's field (kept with
 * the problem's context and released by gs_destroy; several GB on large
 * lattices; its field is copied again after gs_set_gauge).  With the
 * network inner solver (GS_INNER_FGMRES_NET) a problem's sources run on its
 * own context only.  The running solves' persistent kernels draw their
 * blocks from one ledger, so their cooperative grids always fit on the GPU
 * together (GS_OPT_COOP_BLOCKS).  The callers' streams are
 * synchronised before the first solve, every lane stream before return.  The
 * contexts must be distinct (they may hold the same lattice and field).
 * stats (may be NULL): nprob entries, each aggregating its problem's sources
 * (iterations summed, residuals the worst).  Returns the worst status; an
 * error met on a lane context is reported on the problem's own. */
gs_status schur_solve_batched(int nprob, gs_ctx* const* ctxs, const int* type, const int* dir,
                              const int* inverse, const int* nrhs, const void* const* f_dev,
                              void* const* x_dev, const gs_solve_opts* opts,
                              gs_solve_stats* stats);

/* Low-precision vectors of nrhs sources (1..32) with the sources interleaved
 * inside each site: GS_F32 float [6][n][nrhs][4], GS_BF16 bf16
 * [3][n][nrhs][8] (n as for gs_lowp_pack); the complex128 side is
 * [nrhs][n][4][3].  wilson_apply_lowp_multi applies D (type 0) or D_rr to all
 * sources at once, reading each site's links once per launch.  Asynchronous. */
gs_status gs_lowp_pack_multi(gs_ctx* ctx, int type, int dir, int inverse, int prec, int nrhs,
                             const void* x_dev, void* x_lp_dev);
gs_status gs_lowp_unpack_multi(gs_ctx* ctx, int type, int dir, int inverse, int prec, int nrhs,
                               const void* x_lp_dev, void* x_dev);
gs_status wilson_apply_lowp_multi(gs_ctx* ctx, int type, int dir, int inverse, int prec,
                                  int nrhs, const void* x_lp_dev, void* y_lp_dev);

/* y_b = S~_bb x_b: the second-order Schur-complement approximation of
 * Section 3 of the paper,
 *   S~_bb = D_bb - D_br (d^-1 + d~^-1 - d^-1 D_rr d~^-1) D_rb,
 * d the diagonal and d~ the row sums of D_rr, both read as 12 x 12 blocks per
 * rest site (spin x colour).  No inner solve: three stencil launches and one
 * 12 x 12 block product per rest site; the block inverses of d~ are built on
 * the first call per permutation and gauge field (GS_NONFINITE if one is
 * singular).  xb_dev, yb_dev: complex128 [n_b][4][3] in label order, as for
 * schur_apply.  Uses the context's inner-solve workspace; asynchronous
 * except for that first call. */
gs_status schur_apply_reusken(gs_ctx* ctx, int type, int dir, int inverse, const void* xb_dev,
                              void* yb_dev);

/* y_b = S~_bb x_b with the approximation of the given order (Section 3):
 * order 2 is schur_apply_reusken; order 1 is the cruder approximation that
 * Section 3 cites as earlier work, which ignores the couplings inside D_rr:
 * D_rr is replaced by its diagonal d = (m0 + 4) 1, so
 *   S~_bb = D_bb - D_br D_rb / (m0 + 4)
 * (two stencil launches and a scaling; no set-up).  Vectors and workspace as
 * for schur_apply_reusken; asynchronous (order 2: except its first call). */
gs_status schur_apply_approx(gs_ctx* ctx, int type, int dir, int inverse, int order,
                             const void* xb_dev, void* yb_dev);

/* z = D_rr^-1 t on the rest set of (type, dir, inverse): the inner solve of
 * S_bb on its own (opts->inner_tol, inner_prec, inner_solver as for
 * schur_solve).  t_dev, z_dev: complex128 [n_r][4][3] in label order (labels
 * n_b .. V-1).  Used, for example, to make the training pairs of the learned
 * preconditioner.  stats->true_residual = ||t - D_rr z|| / ||t|| recomputed
 * in FP64, inner_iters the Krylov steps taken.  Synchronises the stream. */
gs_status gs_solve_rr(gs_ctx* ctx, int type, int dir, int inverse, const void* t_dev, void* z_dev,
                      const gs_solve_opts* opts, gs_solve_stats* stats);

/* The learned preconditioner: a gauge-equivariant linear convolutional
 * network M ~ D_rr^-1 with three layers, 1 -> C -> C -> 1 channels (C = 2,
 * 4, 8 or 24).  Layer l maps activations psi(x) (channel, spin, colour) to
 *   out(x)[R, a] = sum_{d=0..8} sum_k W_d[R, k] (U_d(x) psi(x + d))[k, a],
 * d = 0: identity, d = 1 + mu: U_mu(x) psi(x + mu), d = 5 + mu:
 * U_mu(x - mu)^dag psi(x - mu); R and k index (channel, spin).  The input is
 * the rest-set vector embedded in the lattice (zero on the coarse sites); the
 * output is read on the rest set.  The paper has no learned component; its
 * own preconditioner is a hand-made approximation of the Schur complement
 * (Section 3, Section 4): this one is fitted to pairs (t, D_rr^-1 t) that
 * gs_solve_rr produces (or t = D_rr z for a given z).  Training: FP32
 * arithmetic and FP32 master weights.  Inference: BF16 weights; with C = 24
 * and GS_OPT_NET_KERNEL = 0 the contractions of all three layers run on the
 * tensor cores (tcgen05.mma, BF16 operands including the transported
 * activations, FP32 accumulation), otherwise on the CUDA cores with FP32
 * activations.  A network is not tied to a context: it uses the links of the
 * context it is called with. */
typedef struct gs_net gs_net;
gs_status gs_net_create(gs_net** net_out, int channels);
gs_status gs_net_destroy(gs_net* net);
/* w_host: complex64 [9][4 C_out][4 C_in] = W_d[R][k] of layer 0, 1 or 2 (host
 * memory; resets the optimiser state). */
gs_status gs_net_set_weights(gs_net* net, int layer, const void* w_host);
/* what = 0: the FP32 weights, 1: the weight gradients of the last training
 * step; same layout as gs_net_set_weights (host memory). */
gs_status gs_net_get(gs_net* net, int what, int layer, void* host_out);
/* y = M t on the rest set; t_dev, y_dev complex128 [n_r][4][3] (label order).
 * BF16 weights; kernels as GS_OPT_NET_KERNEL selects.  Synchronises the
 * stream; GS_TIMEOUT if a tensor-core kernel gave up on a wait (each wait is
 * bounded by one second). */
gs_status gs_net_apply(gs_ctx* ctx, gs_net* net, int type, int dir, int inverse,
                       const void* t_dev, void* y_dev);
/* One training step on `batch` pairs: t_dev, z_dev complex64 [batch][n_r][4][3]
 * with z = D_rr^-1 t.  Loss = mean over the batch of ||M t - z||^2 / ||z||^2
 * (*loss_out); gradients by the backward kernels; with update != 0 one Adam
 * step (lr; beta1 0.9, beta2 0.999, eps 1e-8).  Synchronises the stream. */
gs_status gs_net_train_step(gs_ctx* ctx, gs_net* net, int type, int dir, int inverse, int batch,
                            const void* t_dev, const void* z_dev, float lr, int update,
                            float* loss_out);
/* Attach (or with NULL detach) the network used by GS_INNER_FGMRES_NET. */
gs_status gs_set_net(gs_ctx* ctx, gs_net* net);

/* The cyclic-reduction V-cycle preconditioner of Section 4 (the "3-level
 * V-cycle" of Table 1 is nsteps = 2).  Level 0 is D on the context's
 * lattice; level l + 1 is the Section 3 approximation S~ (order 2; order 1:
 * D_rr's couplings ignored) of level l's operator on its coarse set, indexed
 * by level l's coarse labels in order; coarsening step l uses the
 * permutation type[l], dir[l] (Type II only), inverse[l], applied at levels
 * >= 1 to the coarse labels as a lattice of the coarse extents (Type I halves
 * every extent, Type II(dir) halves L_dir; the blocked extents must be
 * even).  The coarsest level (at most 1024 sites) is inverted exactly (a
 * dense inverse); every rest-set inverse A_rr^-1 is BiCGStab to rest_tol
 * (the paper: 1e-2), at most rest_max_iter steps (the last iterate is used
 * beyond).  One application x = V(f) is the block UL solve of Section 1 with
 * the Schur complement replaced by the next level:
 *   w_b = F_b - A_br A_rr^-1 F_r,  x_b = V_next(w_b),  x_r = A_rr^-1 (F_r - A_rb x_b).
 * The lower levels' operators are assembled once, here: S~ is applied to
 * probe vectors (one per colour of a column colouring of its pattern and
 * spin-colour component) and the results fill a block-sparse matrix.  The V-cycle belongs to the context and
 * must be destroyed before it; a new gauge field needs a new V-cycle.
 * Synchronises the stream. */
typedef struct gs_vcycle gs_vcycle;
gs_status gs_vcycle_create(gs_ctx* ctx, int nsteps, const int* type, const int* dir,
                           const int* inverse, int order, double rest_tol, int rest_max_iter,
                           gs_vcycle** vc_out);
gs_status gs_vcycle_destroy(gs_vcycle* vc);
/* x = V(f): f_dev, x_dev complex128 [V][4][3], site order, not overlapping.
 * stats (may be NULL): inner_solves / inner_iters / inner_max_seen count the
 * rest-set BiCGStab solves of all levels, lowp_fallbacks those stopped at
 * rest_max_iter.  Synchronises the stream. */
gs_status gs_vcycle_apply(gs_vcycle* vc, const void* f_dev, void* x_dev, gs_solve_stats* stats);
/* Level l's extents, sites, stored blocks (12 x 12; 0 for level 0, which is
 * the stencil) and the number of probe colours used to assemble level l + 1
 * (0 for the coarsest). */
gs_status gs_vcycle_level(const gs_vcycle* vc, int level, int dims_out[4], int64_t* sites,
                          int64_t* blocks, int* colours);
/* y = A_level x for level >= 1, in the level's natural order (level l - 1's
 * coarse labels): the assembled coarse operator.  complex128 [sites][4][3]. */
gs_status gs_vcycle_operator_apply(gs_vcycle* vc, int level, const void* x_dev, void* y_dev);

/* BiCGStab (van der Vorst) on the whole system D x = f, to tol in the
 * recursively updated residual, right-preconditioned by one V-cycle per
 * application when vc != NULL (Section 4's preconditioned solver; x is
 * accumulated from the preconditioned directions actually applied, so an
 * inexact V-cycle still gives the x whose residual the recursion tracks),
 * plain when vc == NULL.  f_dev, x_dev complex128 [V][4][3], site order.
 * stats: outer_iters = steps, true_residual = ||f - D x|| / ||f|| recomputed
 * in FP64, outer_residual = the recursive one, rest-set counts as for
 * gs_vcycle_apply.  *rate_out (may be NULL) = Section 4's average
 * convergence rate R = (||r_n|| / ||r_0||)^(1/n) over the n steps taken;
 * history (may be NULL) receives ||r_0||, ||r_1||, ... (-1 past the end),
 * history_cap entries at most.  GS_MAXITER after max_iter steps (x = the last
 * iterate).  Synchronises the stream. */
gs_status gs_solve_bicgstab(gs_ctx* ctx, gs_vcycle* vc, const void* f_dev, void* x_dev, double tol,
                            int max_iter, gs_solve_stats* stats, double* rate_out, double* history,
                            int history_cap);

/* Extreme parts of the spectrum of the context's Wilson operator D (Table 1's
 * second row, the estimated condition number, read as the 2-norm condition
 * number sigma_max / sigma_min of D; the eigenvalues nearest the origin
 * behind the convergence rates of Section 4).
 *
 * gs_condition_number: Lanczos (no reorthogonalisation) on the Hermitian
 * D^H D = gamma_5 D gamma_5 D from start_dev (complex128 [V][4][3], not
 * zero; the caller draws it); every 20 steps the extreme eigenvalues of the
 * tridiagonal matrix are found by bisection and their residual estimates
 * beta_j |last component of the Ritz vector| compared with tol x the
 * eigenvalue; stops when both meet it (GS_OK) or after max_steps steps
 * (GS_MAXITER, the last estimates returned).  *kappa_out = sigma_max /
 * sigma_min, sigma = sqrt(eigenvalue of D^H D); *steps_out (may be NULL)
 * = steps taken.  Synchronises the stream.
 *
 * gs_leftmost_eigenvalues: m steps of Arnoldi (classical Gram-Schmidt twice)
 * on D from start_dev; the eigenvalues of the m x m Hessenberg matrix (shifted
 * QR on the host) sorted by real part, then imaginary part; the first
 * min(k, steps) are written to re_out / im_out, *found_out (may be NULL) =
 * how many.  An invariant Krylov space ends the iteration early with exact
 * eigenvalues.  m <= 4096 (the basis takes (m + 1) V x 192 bytes).
 * Synchronises the stream. */
gs_status gs_condition_number(gs_ctx* ctx, const void* start_dev, int max_steps, double tol,
                              double* kappa_out, double* sigma_min_out, double* sigma_max_out,
                              int* steps_out);
gs_status gs_leftmost_eigenvalues(gs_ctx* ctx, const void* start_dev, int m, int k, double* re_out,
                                  double* im_out, int* found_out);

/* Text of the last error on this context ("" if none).  The pointer stays
 * valid until the next call on the context. */
const char* gs_last_error(const gs_ctx* ctx);

/* Library version string. */
const char* gs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSCHUR_H */
