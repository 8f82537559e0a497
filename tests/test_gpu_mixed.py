"""Mixed-precision inner solves (FP32 and BF16 storage, FP32 arithmetic, FP64
defect correction) against the FP64 oracle through the C ABI.

The low-precision iterations only precondition: every result must meet the
same FP64 tolerances as the plain FP64 path.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import lattice_inputs as li
from oracle import dirac, permute, schur
from tests.gpu_util import lib, rel, to_dev, torch_cuda

pytestmark = pytest.mark.gpu
TYPES = [(1, 0, False), (2, 0, False), (1, 0, True), (2, 0, True)]


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


def _ctx(gs, torch, dims, m0, U):
    ctx = gs.Context(dims, m0, torch.cuda.current_stream().cuda_stream)
    ctx.set_gauge(to_dev(U, torch))
    return ctx


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("t,mu,inv", TYPES)
def test_mixed_schur_apply_matches_oracle(env, prec, t, mu, inv):
    torch, gs = env
    dims, m0 = (4, 4, 4, 4), 0.2
    U = li.random_gauge(dims, 0.3, 0)
    ctx = _ctx(gs, torch, dims, m0, U)
    perm, nb = permute.permutation(dims, t, mu, inv)
    xb = li.gaussian_source(dims, 100).reshape(-1, 12)[perm[:nb]].ravel()
    xbd = to_dev(xb, torch)
    ybd = torch.empty_like(xbd)
    p = gs.GS_F32 if prec == "f32" else gs.GS_BF16
    st = ctx.schur_apply(t, mu, int(inv), xbd, ybd,
                         gs.gs_default_opts(inner_prec=p, inner_tol=1e-13))
    ref = schur.SchurOperator(dirac.wilson_matrix(U, dims, m0), perm, nb, inner="direct")(xb)
    assert rel(ybd.cpu().numpy(), ref) <= 1e-11
    assert st.lowp_cycles >= 2 and st.inner_residual <= 1e-13
    ctx.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_mixed_schur_solve_ragged_and_direct(env, prec):
    torch, gs = env
    dims, m0 = (2, 2, 6, 2), 0.1
    U = li.random_gauge(dims, 0.4, 9)
    ctx = _ctx(gs, torch, dims, m0, U)
    f = li.gaussian_source(dims, 11)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    D = dirac.wilson_matrix(U, dims, m0)
    xs = sla.spsolve(D.tocsc(), f.ravel())
    p = gs.GS_F32 if prec == "f32" else gs.GS_BF16
    for t, mu, inv in TYPES:
        st = ctx.schur_solve(t, mu, int(inv), fd, xd, gs.gs_default_opts(inner_prec=p))
        assert rel(xd.cpu().numpy(), xs) <= 1e-9
        assert st.true_residual <= 1e-10
    ctx.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("t,mu,inv", TYPES)
def test_mixed_solve_8x4_heatbath(env, prec, t, mu, inv):
    """The benchmark workload with the mixed inner solve: same 1e-10 bar,
    checked with the oracle's D."""
    torch, gs = env
    dims, U = li.workload_gauge("8^4 heatbath b5.4")
    ctx = _ctx(gs, torch, dims, -0.4, U)
    f = li.gaussian_source(dims, 100)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    p = gs.GS_F32 if prec == "f32" else gs.GS_BF16
    st = ctx.schur_solve(t, mu, int(inv), fd, xd, gs.gs_default_opts(inner_prec=p))
    D = dirac.wilson_matrix(U, dims, -0.4)
    x = xd.cpu().numpy().ravel()
    assert np.linalg.norm(f.ravel() - D @ x) <= 1e-10 * np.linalg.norm(f)
    assert st.true_residual <= 1e-10
    ctx.close()


def test_mixed_solve_16x32_type_II_sampled(env):
    """16^3 x 32, exp(i 0.25 H) + 5 APE steps, m0 = -0.3, Type II, one
    Gaussian source (the mixed-precision workload): FP64 true residual from
    the library and, on 64 sampled sites, f - D x from the oracle's rows."""
    torch, gs = env
    dims, U = li.workload_gauge("16^3x32 eps0.25 ape5")
    m0 = -0.3
    ctx = _ctx(gs, torch, dims, m0, U)
    f = li.gaussian_source(dims, 100)
    fd = to_dev(f, torch)
    for prec in (gs.GS_F32, gs.GS_BF16):
        xd = torch.empty_like(fd)
        st = ctx.schur_solve(2, 0, 0, fd, xd, gs.gs_default_opts(inner_prec=prec))
        assert st.true_residual <= 1e-10
        x = xd.cpu().numpy().ravel()
        sites = np.random.default_rng(4).choice(li.volume(dims), 64, replace=False)
        Ds = dirac.wilson_matrix(U, dims, m0, rows_of=sites)
        fs = f.reshape(-1, 12)[sites].ravel()
        r = fs - Ds @ x
        assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(fs)
    ctx.close()


def test_lowp_tol_validation(env):
    torch, gs = env
    dims = (4, 4, 2, 2)
    ctx = _ctx(gs, torch, dims, 0.1, li.random_gauge(dims, 0.3, 2))
    z = torch.zeros(li.volume(dims) * 12, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(gs.GschurError):
        ctx.schur_solve(1, 0, 0, z, z.clone(), gs.gs_default_opts(inner_prec=1, lowp_tol=2.0))
    with pytest.raises(gs.GschurError):
        ctx.schur_solve(1, 0, 0, z, z.clone(), gs.gs_default_opts(inner_prec=7))
    ctx.close()
