"""Failure detection through the C ABI, in forms that fault no GPU: a
non-finite input is reported as GS_NONFINITE; a learned preconditioner whose
output is not finite is discarded and the plain FP64 solver finishes the solve
to the same tolerance; a bounded device wait that is made to run out (one
block never arrives at a grid barrier, or nothing arrives at an mbarrier)
returns GS_TIMEOUT after the context's wait limit, and the context stays
usable."""
import time

import numpy as np
import pytest

import lattice_inputs as li
from oracle import dirac, permute, schur
from tests.gpu_util import close, lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu
DIMS, M0 = (4, 4, 4, 4), 0.2


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


def _ctx(gs, torch):
    U = li.random_gauge(DIMS, 0.3, 0)
    ctx = gs.Context(DIMS, M0, torch.cuda.current_stream().cuda_stream)
    ctx.set_gauge(to_dev(U, torch))
    return ctx, U


def _apply_matches_oracle(gs, torch, ctx, U):
    perm, nb = permute.permutation(DIMS, 1)
    xb = li.gaussian_source(DIMS, 100).reshape(-1, 12)[perm[:nb]].ravel()
    xbd = to_dev(xb, torch)
    ybd = torch.empty_like(xbd)
    ctx.schur_apply(1, 0, 0, xbd, ybd, gs.gs_default_opts(inner_tol=1e-14))
    ref = schur.SchurOperator(dirac.wilson_matrix(U, DIMS, M0), perm, nb, inner="direct")(xb)
    return close(ybd.cpu().numpy(), ref, 1e-12)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("where", ["coarse", "rest"])
def test_nan_source_is_reported_and_the_context_stays_usable(env, prec, where):
    torch, gs = env
    ctx, U = _ctx(gs, torch)
    perm, nb = permute.permutation(DIMS, 1)
    f = li.gaussian_source(DIMS, 3).reshape(-1, 12)
    site = perm[0] if where == "coarse" else perm[nb + 5]
    f[site, 4] = np.nan
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    with pytest.raises(gs.GschurError) as e:
        ctx.schur_solve(1, 0, 0, fd, xd, gs.gs_default_opts(inner_prec=prec))
    assert e.value.status == gs.GS_NONFINITE
    xb = torch.full((nb * 12,), float("nan"), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(gs.GschurError) as e:
        ctx.schur_apply(1, 0, 0, xb, torch.empty_like(xb), gs.gs_default_opts(inner_prec=prec))
    assert e.value.status == gs.GS_NONFINITE
    assert _apply_matches_oracle(gs, torch, ctx, U)
    ctx.close()


def test_nonfinite_network_falls_back_to_the_plain_solver(env):
    """A network with NaN weights gives a non-finite correction in the first
    FGMRES pass; the pass is discarded and the FP64 BiCGStab finishes: the
    solve still meets 1e-10 and matches a direct solve."""
    import scipy.sparse.linalg as sla
    from paper_0704_2341_gb300 import learned
    torch, gs = env
    ctx, U = _ctx(gs, torch)
    nt = gs.Net(8)
    for layer, w in enumerate(learned.identity_like_weights(8, M0, 3)):
        w = np.array(w, dtype=np.complex64)
        if layer == 1:
            w[0, 0, 0] = np.nan
        nt.set_weights(layer, w)
    ctx.set_net(nt)
    f = li.gaussian_source(DIMS, 100)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    st = ctx.schur_solve(1, 0, 0, fd, xd, learned.fgmres_net_opts())
    xs = sla.spsolve(dirac.wilson_matrix(U, DIMS, M0).tocsc(), f.ravel())
    assert st.true_residual <= 1e-10
    assert st.lowp_fallbacks >= 1
    assert close(xd.cpu().numpy(), xs, 1e-9)
    ctx.set_net(None)
    nt.close()
    ctx.close()


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_runs_out_and_reports_timeout(env, which):
    torch, gs = env
    ctx, U = _ctx(gs, torch)
    assert ctx.get_option(gs.GS_OPT_WAIT_LIMIT_US) == 1000000
    ctx.set_option(gs.GS_OPT_WAIT_LIMIT_US, 20000)           # 20 ms
    assert ctx.get_option(gs.GS_OPT_WAIT_LIMIT_US) == 20000
    t0 = time.perf_counter()
    status = ctx.selftest_wait(which)
    dt = time.perf_counter() - t0
    assert status == gs.GS_TIMEOUT
    assert "ran out" in gs.gs_last_error(ctx.handle)
    assert dt < 0.9                                          # the short limit, not the 1 s default
    # the context (and the persistent solvers that share the barrier words)
    # still work, with the short limit and after restoring the default
    assert _apply_matches_oracle(gs, torch, ctx, U)
    ctx.set_option(gs.GS_OPT_WAIT_LIMIT_US, 1000000)
    assert _apply_matches_oracle(gs, torch, ctx, U)
    for bad in (0, -5, 60000001):
        with pytest.raises(gs.GschurError):
            ctx.set_option(gs.GS_OPT_WAIT_LIMIT_US, bad)
    ctx.close()
