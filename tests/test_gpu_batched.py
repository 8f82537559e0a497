"""Several sources and several lattices solved together (multi-source
stencil, persistent multi-source inner solves, lock-step outer GMRES,
concurrent solves on lanes), through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import lattice_inputs as li
from oracle import dirac, permute, schur
from tests.gpu_util import close, lib, maxrel, rel, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


def _ctx(gs, torch, dims, m0, U, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    ctx = gs.Context(dims, m0, s)
    ctx.set_gauge(to_dev(U, torch))
    return ctx


@pytest.mark.parametrize("prec,tol", [("f32", 4e-6), ("bf16", 3e-2)])
@pytest.mark.parametrize("nrhs", [1, 3, 12])
@pytest.mark.parametrize("t", [0, 1])
def test_multi_source_stencil(env, prec, tol, nrhs, t):
    torch, gs = env
    dims = (4, 4, 2, 4)
    U = li.random_gauge(dims, 0.35, 4)
    ctx = _ctx(gs, torch, dims, 0.05, U)
    D = dirac.wilson_matrix(U, dims, 0.05)
    if t == 0:
        n = li.volume(dims)
        A = D
    else:
        perm, nb = permute.permutation(dims, 1)
        A = schur.partition(D, perm, nb)[3]
        n = li.volume(dims) - nb
    p = gs.GS_F32 if prec == "f32" else gs.GS_BF16
    x = li.gaussian_source(dims, 9, n_src=max(nrhs, 2))[:nrhs].reshape(nrhs, -1, 12)[:, :n]
    xd = to_dev(np.ascontiguousarray(x), torch)
    xl = torch.empty(gs.lowp_bytes(n * nrhs, p), dtype=torch.uint8, device="cuda:0")
    yl = torch.empty_like(xl)
    yd = torch.empty_like(xd)
    ctx.lowp_pack_multi(t, 0, 0, p, nrhs, xd, xl)
    ctx.wilson_apply_lowp_multi(t, 0, 0, p, nrhs, xl, yl)
    ctx.lowp_unpack_multi(t, 0, 0, p, nrhs, yl, yd)
    got = yd.cpu().numpy().reshape(nrhs, -1)
    for j in range(nrhs):
        ref = A @ x[j].ravel()
        assert np.abs(got[j] - ref).max() <= tol * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("t,mu,inv", [(1, 0, False), (2, 0, False), (1, 0, True), (2, 1, True)])
def test_schur_solve_multi_matches_direct(env, prec, t, mu, inv):
    torch, gs = env
    dims, m0 = (4, 4, 4, 4), 0.2
    U = li.random_gauge(dims, 0.3, 0)
    ctx = _ctx(gs, torch, dims, m0, U)
    N = 3
    f = li.gaussian_source(dims, 21, n_src=N)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    p = gs.GS_F32 if prec == "f32" else gs.GS_BF16
    st = ctx.schur_solve_multi(t, mu, int(inv), N, fd, xd, gs.gs_default_opts(inner_prec=p))
    D = dirac.wilson_matrix(U, dims, m0).tocsc()
    x = xd.cpu().numpy().reshape(N, -1)
    for j in range(N):
        xs = sla.spsolve(D, f[j].ravel())
        assert close(x[j], xs, 1e-9)
    assert st.true_residual <= 1e-10
    ctx.close()


def test_schur_solve_multi_8x4_heatbath(env):
    torch, gs = env
    dims, U = li.workload_gauge("8^4 heatbath b5.4")
    ctx = _ctx(gs, torch, dims, -0.4, U)
    N = 4
    f = li.gaussian_source(dims, 31, n_src=N)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    st = ctx.schur_solve_multi(1, 0, 0, N, fd, xd, gs.gs_default_opts(inner_prec=gs.GS_F32))
    D = dirac.wilson_matrix(U, dims, -0.4)
    x = xd.cpu().numpy().reshape(N, -1)
    for j in range(N):
        assert np.linalg.norm(f[j].ravel() - D @ x[j]) <= 1e-10 * np.linalg.norm(f[j])
    assert st.true_residual <= 1e-10
    ctx.close()


def test_schur_solve_batched_concurrent_problems(env):
    """Three problems of different lattices, permutations and source counts
    on three contexts and streams at once, each against a direct solve."""
    torch, gs = env
    specs = [((4, 4, 4, 4), 0.2, 0.3, 0, 1, 0, 0, 2),
             ((2, 2, 6, 2), 0.1, 0.4, 9, 2, 0, 1, 3),
             ((4, 2, 4, 4), -0.1, 0.3, 5, 2, 2, 0, 1)]
    ctxs, probs, refs, keep = [], [], [], []
    for dims, m0, eps, seed, t, mu, inv, N in specs:
        U = li.random_gauge(dims, eps, seed)
        s = torch.cuda.Stream()
        ctx = _ctx(gs, torch, dims, m0, U, s.cuda_stream)
        f = li.gaussian_source(dims, seed + 50, n_src=max(N, 2))[:N]
        fd = to_dev(np.ascontiguousarray(f), torch)
        xd = torch.zeros_like(fd)
        probs.append(dict(ctx=ctx.handle, type=t, dir=mu, inverse=inv, nrhs=N, f=fd, x=xd))
        refs.append((dirac.wilson_matrix(U, dims, m0).tocsc(), f))
        ctxs.append(ctx)
        keep.append(s)
    torch.cuda.synchronize()
    status, stats = gs.schur_solve_batched(probs, gs.gs_default_opts(inner_prec=gs.GS_F32))
    torch.cuda.synchronize()
    assert status == gs.GS_OK
    for (D, f), pr, st in zip(refs, probs, stats):
        x = pr["x"].cpu().numpy().reshape(pr["nrhs"], -1)
        for j in range(pr["nrhs"]):
            assert close(x[j], sla.spsolve(D, f[j].ravel()), 1e-9)
        assert st.true_residual <= 1e-10
    for c in ctxs:
        c.close()


def test_multi_rejects_bad_arguments(env):
    torch, gs = env
    dims = (4, 4, 2, 2)
    ctx = _ctx(gs, torch, dims, 0.1, li.random_gauge(dims, 0.3, 2))
    z = torch.zeros(li.volume(dims) * 12, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(gs.GschurError):
        ctx.schur_solve_multi(1, 0, 0, 33, z, z.clone())
    with pytest.raises(gs.GschurError):   # the multi-source solve runs low-precision inner solves
        ctx.schur_solve_multi(1, 0, 0, 1, z, z.clone(), gs.gs_default_opts(inner_prec=gs.GS_F64))
    ctx.close()


def test_batch_shape_option_gives_the_same_solutions(env):
    """GS_OPT_MULTI_BATCH: sources together (1) or one at a time (2) solve to
    the same 1e-10 residual and agree to the solver tolerance; the default (0)
    shares launches on this 8^4-like rest set and reports 0."""
    torch, gs = env
    dims = (8, 8, 4, 8)
    U = li.random_gauge(dims, 0.3, 4)
    ctx = _ctx(gs, torch, dims, -0.1, U)
    assert ctx.get_option(gs.GS_OPT_MULTI_BATCH) == 0
    f = to_dev(np.ascontiguousarray(li.gaussian_source(dims, 31, n_src=3)), torch)
    o = gs.gs_default_opts(inner_prec=gs.GS_F32)
    xs = []
    for mode in (1, 2):
        ctx.set_option(gs.GS_OPT_MULTI_BATCH, mode)
        x = torch.zeros_like(f)
        st = ctx.schur_solve_multi(1, 0, 0, 3, f, x, o)
        assert st.true_residual <= 1e-10
        xs.append(x.cpu().numpy())
    assert close(xs[0], xs[1], 1e-8)
    with pytest.raises(gs.GschurError):
        ctx.set_option(gs.GS_OPT_MULTI_BATCH, 3)
    ctx.close()


def test_batched_plain_f64_four_permutations_match_one_at_a_time(env):
    """The benchmark's form: the four permutations of one 8^4 system solved
    at once by schur_solve_batched with plain FP64 inner solves (one context
    and stream each, the persistent kernels on SM shares), against the same
    solves one at a time, and against the oracle's D."""
    torch, gs = env
    from oracle import dirac
    dims, U = li.workload_gauge("8^4 heatbath b5.4")
    D = dirac.wilson_matrix(U, dims, -0.4)
    perms = [(1, 0, 0), (2, 0, 0), (1, 0, 1), (2, 0, 1)]
    streams = [torch.cuda.Stream() for _ in perms]
    ctxs = [_ctx(gs, torch, dims, -0.4, U, s.cuda_stream) for s in streams]
    f = to_dev(li.gaussian_source(dims, 100), torch)
    xs = [torch.empty_like(f) for _ in perms]
    probs = [dict(ctx=c.handle, type=t, dir=mu, inverse=inv, nrhs=1, f=f, x=x)
             for c, (t, mu, inv), x in zip(ctxs, perms, xs)]
    o = gs.gs_default_opts()
    status, sts = gs.schur_solve_batched(probs, o)
    torch.cuda.synchronize()
    assert status == gs.GS_OK
    fh = f.cpu().numpy().ravel()
    for (t, mu, inv), c, x, st in zip(perms, ctxs, xs, sts):
        assert st.true_residual <= 1e-10
        xb = x.cpu().numpy().ravel()
        assert np.linalg.norm(fh - D @ xb) <= 1e-10 * np.linalg.norm(fh)
        x1 = torch.empty_like(f)
        c.schur_solve(t, mu, inv, f, x1, o)
        assert close(xb, x1.cpu().numpy(), 1e-8)
    status, _ = gs.schur_solve_batched([probs[0], probs[0]], o)   # one context twice
    assert status == gs.GS_EINVAL
    status, _ = gs.schur_solve_batched([dict(probs[0], nrhs=0)], o)
    assert status == gs.GS_EINVAL
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_sources_on_lane_contexts(env, prec):
    """More sources than problems: the library spreads them over lane
    contexts of the same lattice (its own streams and field copies); every
    solution against a direct sparse solve, and the aggregated statistics
    against the same sources solved one at a time."""
    torch, gs = env
    specs = [((4, 4, 4, 4), 0.2, 0.3, 0, 1, 0, 0, 5),
             ((4, 2, 4, 4), -0.1, 0.3, 5, 2, 2, 1, 3)]
    p = gs.GS_F64 if prec == "f64" else gs.GS_F32
    o = gs.gs_default_opts(inner_prec=p)
    ctxs, probs, refs, keep = [], [], [], []
    for dims, m0, eps, seed, t, mu, inv, N in specs:
        U = li.random_gauge(dims, eps, seed)
        s = torch.cuda.Stream()
        ctx = _ctx(gs, torch, dims, m0, U, s.cuda_stream)
        f = li.gaussian_source(dims, seed + 70, n_src=N)
        fd = to_dev(np.ascontiguousarray(f), torch)
        probs.append(dict(ctx=ctx.handle, type=t, dir=mu, inverse=inv, nrhs=N, f=fd, x=torch.zeros_like(fd)))
        refs.append((dirac.wilson_matrix(U, dims, m0).tocsc(), f))
        ctxs.append(ctx)
        keep.append(s)
    ctxs[0].set_option(gs.GS_OPT_BATCH_LANES, 3)
    assert ctxs[0].get_option(gs.GS_OPT_BATCH_LANES) == 3
    torch.cuda.synchronize()
    status, stats = gs.schur_solve_batched(probs, o)
    assert status == gs.GS_OK
    for (D, f), pr, st, c, spec in zip(refs, probs, stats, ctxs, specs):
        t, mu, inv, N = spec[4:]
        x = pr["x"].cpu().numpy().reshape(N, -1)
        inner = 0
        for j in range(N):
            assert close(x[j], sla.spsolve(D, f[j].ravel()), 1e-9)
            x1 = torch.zeros_like(pr["f"][j])
            inner += c.schur_solve(t, mu, inv, pr["f"][j], x1, o).inner_solves
        assert st.true_residual <= 1e-10
        # the same work, up to an outer iteration or two where the grid sizes
        # (and so the rounding of the reductions) differ
        assert abs(st.inner_solves - inner) <= max(2 * N, inner // 10)
    for c in ctxs:
        c.close()


def test_batched_lane_contexts_follow_a_new_field(env):
    """Lane contexts keep a copy of the problem's field: after gs_set_gauge
    on the problem's context the next batched call solves with the new one."""
    torch, gs = env
    dims, m0, N = (4, 4, 4, 4), 0.1, 4
    U1, U2 = li.random_gauge(dims, 0.3, 11), li.random_gauge(dims, 0.4, 12)
    ctx = _ctx(gs, torch, dims, m0, U1)
    ctx.set_option(gs.GS_OPT_BATCH_LANES, 4)
    f = li.gaussian_source(dims, 13, n_src=N)
    fd = to_dev(np.ascontiguousarray(f), torch)
    o = gs.gs_default_opts()
    for U in (U1, U2):
        ctx.set_gauge(to_dev(U, torch))
        pr = dict(ctx=ctx.handle, type=1, dir=0, inverse=0, nrhs=N, f=fd, x=torch.zeros_like(fd))
        status, (st,) = gs.schur_solve_batched([pr], o)
        assert status == gs.GS_OK and st.true_residual <= 1e-10
        D = dirac.wilson_matrix(U, dims, m0).tocsc()
        x = pr["x"].cpu().numpy().reshape(N, -1)
        for j in range(N):
            assert close(x[j], sla.spsolve(D, f[j].ravel()), 1e-9)
    with pytest.raises(gs.GschurError):
        ctx.set_option(gs.GS_OPT_BATCH_LANES, 65)
    ctx.close()


def test_batched_one_lane_is_the_sequential_solve(env):
    """GS_OPT_BATCH_LANES = 1: the sources one after another on the problem's
    own context, with whole-GPU grids -- bit for bit the single-source calls."""
    torch, gs = env
    dims, m0, N = (4, 4, 4, 8), 0.0, 3
    U = li.random_gauge(dims, 0.35, 21)
    ctx = _ctx(gs, torch, dims, m0, U)
    ctx.set_option(gs.GS_OPT_BATCH_LANES, 1)
    fd = to_dev(np.ascontiguousarray(li.gaussian_source(dims, 22, n_src=N)), torch)
    o = gs.gs_default_opts(inner_prec=gs.GS_F32)
    pr = dict(ctx=ctx.handle, type=2, dir=3, inverse=0, nrhs=N, f=fd, x=torch.zeros_like(fd))
    status, _ = gs.schur_solve_batched([pr], o)
    assert status == gs.GS_OK
    for j in range(N):
        x1 = torch.zeros_like(fd[j])
        ctx.schur_solve(2, 3, 0, fd[j], x1, o)
        assert torch.equal(x1, pr["x"][j])
    ctx.close()


def test_batched_block_ledger_under_contention(env):
    """Six FP64 solves at once on 8^4 Type I rest sets (3840 sites): each
    asks the block ledger for one round of 32-site tiles, 120 blocks, 720 in
    all against 456 co-resident, so later launches get what the others leave
    (or wait for it).  Every solve still converges and equals its
    one-at-a-time result."""
    torch, gs = env
    dims, m0 = (8, 8, 8, 8), -0.1
    U = li.random_gauge(dims, 0.3, 31)
    streams = [torch.cuda.Stream() for _ in range(6)]
    ctxs = [_ctx(gs, torch, dims, m0, U, s.cuda_stream) for s in streams]
    ctxs[0].set_option(gs.GS_OPT_BATCH_LANES, 6)
    fs = [to_dev(li.gaussian_source(dims, 40 + k), torch) for k in range(6)]
    perms = [(1, 0, 0), (1, 0, 1), (1, 0, 0), (1, 0, 1), (1, 0, 0), (1, 0, 1)]
    probs = [dict(ctx=c.handle, type=t, dir=mu, inverse=inv, nrhs=1, f=f, x=torch.zeros_like(f))
             for c, (t, mu, inv), f in zip(ctxs, perms, fs)]
    o = gs.gs_default_opts()
    for _ in range(2):
        status, stats = gs.schur_solve_batched(probs, o)
        assert status == gs.GS_OK
        assert max(st.true_residual for st in stats) <= 1e-10
    for c, (t, mu, inv), pr in zip(ctxs, perms, probs):
        x1 = torch.zeros_like(pr["f"])
        c.schur_solve(t, mu, inv, pr["f"], x1, o)
        assert close(pr["x"].cpu().numpy(), x1.cpu().numpy(), 1e-8)
    for c in ctxs:
        c.close()
