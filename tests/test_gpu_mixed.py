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
from tests.gpu_util import close, lib, maxrel, rel, to_dev, torch_cuda

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


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("t,mu,inv", TYPES)
def test_mixed_schur_apply_matches_oracle(env, prec, t, mu, inv, kernel):
    torch, gs = env
    dims, m0 = (4, 4, 4, 4), 0.2
    U = li.random_gauge(dims, 0.3, 0)
    ctx = _ctx(gs, torch, dims, m0, U)
    ctx.set_option(gs.GS_OPT_INNER_KERNEL, kernel)
    perm, nb = permute.permutation(dims, t, mu, inv)
    xb = li.gaussian_source(dims, 100).reshape(-1, 12)[perm[:nb]].ravel()
    xbd = to_dev(xb, torch)
    ybd = torch.empty_like(xbd)
    p = gs.GS_F32 if prec == "f32" else gs.GS_BF16
    st = ctx.schur_apply(t, mu, int(inv), xbd, ybd,
                         gs.gs_default_opts(inner_prec=p, inner_tol=1e-13))
    ref = schur.SchurOperator(dirac.wilson_matrix(U, dims, m0), perm, nb, inner="direct")(xb)
    assert close(ybd.cpu().numpy(), ref, 1e-11)
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
        assert close(xd.cpu().numpy(), xs, 1e-9)
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


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("prec,tol", [("f32", 4e-6), ("bf16", 3e-2)])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (3, 4, 2, 5), (12, 10, 6, 14)])
def test_lowp_stencil_full_lattice(env, prec, tol, dims, variant):
    """wilson_apply_lowp (type 0, whole lattice) against the oracle's D in
    FP64, to the rounding of the storage format (FP32: 2^-24, BF16: 2^-9 per
    input, about 100 terms per output).  On the whole lattice the kernels
    compute the neighbours from the site index (odd extents, L = 2 and a
    10080-site lattice over many blocks check that arithmetic)."""
    torch, gs = env
    U = li.random_gauge(dims, 0.4, 3)
    ctx = _ctx(gs, torch, dims, -0.2, U)
    ctx.set_option(gs.GS_OPT_STENCIL_VARIANT, variant)
    V = li.volume(dims)
    p = gs.GS_F32 if prec == "f32" else gs.GS_BF16
    x = li.gaussian_source(dims, 5)
    xd = to_dev(x, torch)
    xl = torch.empty(gs.lowp_bytes(V, p), dtype=torch.uint8, device="cuda:0")
    yl = torch.empty_like(xl)
    yd = torch.empty_like(xd)
    ctx.lowp_pack(0, 0, 0, p, xd, xl)
    ctx.wilson_apply_lowp(0, 0, 0, p, xl, yl)
    ctx.lowp_unpack(0, 0, 0, p, yl, yd)
    ref = (dirac.wilson_matrix(U, dims, -0.2) @ x.ravel()).reshape(x.shape)
    got = yd.cpu().numpy()
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # pack / unpack round trip is exact up to the storage rounding
    back = torch.empty_like(xd)
    ctx.lowp_unpack(0, 0, 0, p, xl, back)
    assert np.abs(back.cpu().numpy() - x).max() <= (2 ** -8 if prec == "bf16" else 2 ** -23) * np.abs(x).max()
    ctx.close()


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("prec,tol", [("f32", 4e-6), ("bf16", 3e-2)])
@pytest.mark.parametrize("t,mu,inv", TYPES + [(2, 2, True)])
def test_lowp_stencil_rest_set(env, prec, tol, t, mu, inv, variant):
    """wilson_apply_lowp on the rest set r: D_rr of P D P^T (Section 1)."""
    torch, gs = env
    dims = (4, 4, 4, 4)
    U = li.random_gauge(dims, 0.3, 6)
    ctx = _ctx(gs, torch, dims, 0.1, U)
    ctx.set_option(gs.GS_OPT_STENCIL_VARIANT, variant)
    perm, nb = permute.permutation(dims, t, mu, inv)
    _, _, _, Drr = schur.partition(dirac.wilson_matrix(U, dims, 0.1), perm, nb)
    n = li.volume(dims) - nb
    p = gs.GS_F32 if prec == "f32" else gs.GS_BF16
    z = li.gaussian_source(dims, 8).reshape(-1, 12)[:n].ravel()
    zd = to_dev(z, torch)
    zl = torch.empty(gs.lowp_bytes(n, p), dtype=torch.uint8, device="cuda:0")
    yl = torch.empty_like(zl)
    yd = torch.empty_like(zd)
    ctx.lowp_pack(t, mu, int(inv), p, zd, zl)
    ctx.wilson_apply_lowp(t, mu, int(inv), p, zl, yl)
    ctx.lowp_unpack(t, mu, int(inv), p, yl, yd)
    ref = Drr @ z
    assert np.abs(yd.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    ctx.close()


def test_autotuner_picks_a_variant_and_options_validate(env):
    torch, gs = env
    dims = (8, 8, 4, 4)
    ctx = _ctx(gs, torch, dims, 0.1, li.random_gauge(dims, 0.3, 2))
    V = li.volume(dims)
    x = to_dev(li.gaussian_source(dims, 1), torch)
    xl = torch.empty(gs.lowp_bytes(V, gs.GS_F32), dtype=torch.uint8, device="cuda:0")
    ctx.lowp_pack(0, 0, 0, gs.GS_F32, x, xl)
    assert ctx.get_option(gs.GS_OPT_STENCIL_VARIANT) in (1, 2, 3, 4, 5, 6)
    with pytest.raises(gs.GschurError):
        ctx.set_option(gs.GS_OPT_STENCIL_VARIANT, 7)
    with pytest.raises(gs.GschurError):
        ctx.set_option(99, 0)
    ctx.close()
