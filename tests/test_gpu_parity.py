"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (FP64 throughout): the stencil and the permutations differ from the
oracle only by rounding order (<= 1e-13 relative; indices bit-exact); every
result that goes through an inner Krylov solve is compared at a tolerance set
by that solve's stopping criterion.
"""
import numpy as np
import pytest

import lattice_inputs as li
from oracle import dirac, permute, schur
from tests.gpu_util import close, lib, maxrel, rel, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TYPES = [(1, 0, False), (2, 0, False), (1, 0, True), (2, 0, True)]


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    gs = lib()
    return torch, gs


def _ctx(gs, torch, dims, m0, U):
    ctx = gs.Context(dims, m0, torch.cuda.current_stream().cuda_stream)
    ctx.set_gauge(to_dev(U, torch))
    return ctx


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 2, 8), (2, 2, 2, 2),
                                  (16, 16, 16, 32)])
def test_permutation_bit_exact(env, dims):
    torch, gs = env
    ctx = gs.Context(dims, 0.0, torch.cuda.current_stream().cuda_stream)
    V = li.volume(dims)
    out = torch.empty(V, dtype=torch.int32, device="cuda:0")
    cases = [(1, 0, inv) for inv in (0, 1)] + [(2, mu, inv) for mu in range(4) for inv in (0, 1)]
    for t, mu, inv in cases:
        nb = ctx.get_permutation(t, mu, inv, out)
        ref, nb_ref = permute.permutation(dims, t, mu, bool(inv))
        assert nb == nb_ref
        assert np.array_equal(out.cpu().numpy().astype(np.int64), ref), (t, mu, inv)
    ctx.close()


def test_permute_sites_gather_scatter_bit_exact(env):
    torch, gs = env
    dims = (6, 4, 2, 8)
    V = li.volume(dims)
    ctx = gs.Context(dims, 0.0, torch.cuda.current_stream().cuda_stream)
    x = li.gaussian_source(dims, 7)
    xd = to_dev(x, torch)
    y = torch.empty_like(xd)
    z = torch.empty_like(xd)
    for t, mu, inv in [(1, 0, 0), (1, 0, 1), (2, 1, 0), (2, 3, 1)]:
        perm, nb = permute.permutation(dims, t, mu, bool(inv))
        assert ctx.permute_sites(t, mu, inv, 0, xd, y) == nb
        assert np.array_equal(y.cpu().numpy(), x[perm])          # (P x)_i = x_{p(i)}
        ctx.permute_sites(t, mu, inv, 1, y, z)
        assert np.array_equal(z.cpu().numpy(), x)                 # P^T P = 1
    ctx.close()


@pytest.mark.parametrize("dims,eps,m0", [((4, 4, 4, 4), 0.3, 0.2), ((2, 2, 2, 2), 0.5, -0.3),
                                         ((3, 4, 2, 5), 0.4, 0.1), ((6, 4, 4, 8), 0.3, -0.4),
                                         ((8, 8, 8, 8), 0.2, -0.38)])
def test_wilson_apply_matches_oracle(env, dims, eps, m0):
    torch, gs = env
    U = li.random_gauge(dims, eps, 1)
    ctx = _ctx(gs, torch, dims, m0, U)
    x = li.gaussian_source(dims, 3)
    xd = to_dev(x, torch)
    yd = torch.empty_like(xd)
    ctx.wilson_apply(xd, yd)
    torch.cuda.synchronize()
    ref = (dirac.wilson_matrix(U, dims, m0) @ x.ravel()).reshape(x.shape)
    got = yd.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("t,mu,inv", TYPES + [(2, 3, False), (2, 1, True)])
def test_schur_apply_matches_oracle_4x4(env, t, mu, inv, kernel):
    """4^4, exp(i 0.3 H) seed 0, m0 = 0.2, Gaussian source seed 100 (the small
    workload), inner tolerance 1e-14: S_bb x_b within 1e-12 of the oracle
    (direct sparse LU for D_rr^-1)."""
    torch, gs = env
    dims, m0 = (4, 4, 4, 4), 0.2
    U = li.random_gauge(dims, 0.3, 0)
    ctx = _ctx(gs, torch, dims, m0, U)
    ctx.set_option(gs.GS_OPT_INNER_KERNEL, kernel)   # persistent / one launch per phase
    perm, nb = permute.permutation(dims, t, mu, inv)
    src = li.gaussian_source(dims, 100).reshape(-1, 12)
    xb = src[perm[:nb]].ravel()
    xbd = to_dev(xb, torch)
    ybd = torch.empty_like(xbd)
    st = ctx.schur_apply(t, mu, int(inv), xbd, ybd, gs.gs_default_opts(inner_tol=1e-14))
    D = dirac.wilson_matrix(U, dims, m0)
    ref = schur.SchurOperator(D, perm, nb, inner="direct")(xb)
    assert close(ybd.cpu().numpy(), ref, 1e-12)
    assert st.inner_solves == 1 and st.inner_iters > 0
    ctx.close()


def test_schur_columns_match_dense_S(env):
    """Column probes of S_bb (unit vectors) against the oracle's dense S_bb."""
    torch, gs = env
    dims, m0 = (4, 4, 2, 2), 0.3
    U = li.random_gauge(dims, 0.3, 5)
    ctx = _ctx(gs, torch, dims, m0, U)
    for t, mu, inv in [(1, 0, False), (2, 1, True)]:
        perm, nb = permute.permutation(dims, t, mu, inv)
        S = schur.schur_dense(dirac.wilson_matrix(U, dims, m0), perm, nb)
        n = 12 * nb
        for k in [0, 5, n // 2, n - 1]:
            e = np.zeros(n, complex)
            e[k] = 1.0
            ed = to_dev(e, torch)
            yd = torch.empty_like(ed)
            ctx.schur_apply(t, mu, int(inv), ed, yd, gs.gs_default_opts(inner_tol=1e-14))
            assert close(yd.cpu().numpy(), S[:, k], 1e-12)
    ctx.close()


@pytest.mark.parametrize("t,mu,inv", TYPES)
def test_schur_solve_matches_direct_solve_4x4(env, t, mu, inv):
    import scipy.sparse.linalg as sla
    torch, gs = env
    dims, m0 = (4, 4, 4, 4), 0.2
    U = li.random_gauge(dims, 0.3, 0)
    ctx = _ctx(gs, torch, dims, m0, U)
    f = li.gaussian_source(dims, 100)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    st = ctx.schur_solve(t, mu, int(inv), fd, xd, gs.gs_default_opts(tol=1e-11, inner_tol=1e-13))
    D = dirac.wilson_matrix(U, dims, m0)
    x = xd.cpu().numpy().ravel()
    xs = sla.spsolve(D.tocsc(), f.ravel())
    assert np.linalg.norm(f.ravel() - D @ x) <= 1e-10 * np.linalg.norm(f)
    assert close(x, xs, 1e-9)
    assert st.true_residual <= 1e-10
    ctx.close()


@pytest.mark.parametrize("outer", ["gmres", "bicgstab"])
def test_schur_solve_outer_solvers_ragged_lattice(env, outer):
    """V = 2*2*6*2 = 48 sites (not a multiple of the 32-site tile), n_b = 3."""
    import scipy.sparse.linalg as sla
    torch, gs = env
    dims, m0 = (2, 2, 6, 2), 0.1
    U = li.random_gauge(dims, 0.4, 9)
    ctx = _ctx(gs, torch, dims, m0, U)
    f = li.gaussian_source(dims, 11)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    solver = gs.GS_GMRES if outer == "gmres" else gs.GS_BICGSTAB
    for t, mu, inv in TYPES:
        st = ctx.schur_solve(t, mu, int(inv), fd, xd,
                             gs.gs_default_opts(outer_solver=solver, inner_tol=1e-13))
        D = dirac.wilson_matrix(U, dims, m0)
        xs = sla.spsolve(D.tocsc(), f.ravel())
        assert close(xd.cpu().numpy(), xs, 1e-9)
        assert st.true_residual <= 1e-10
    ctx.close()


def test_zero_source_and_errors(env):
    torch, gs = env
    dims = (4, 4, 2, 2)
    U = li.random_gauge(dims, 0.3, 2)
    ctx = gs.Context(dims, 0.1, torch.cuda.current_stream().cuda_stream)
    z = torch.zeros(li.volume(dims) * 12, dtype=torch.complex128, device="cuda:0")
    x = torch.full_like(z, 3.0)
    with pytest.raises(gs.GschurError) as e:
        ctx.schur_solve(1, 0, 0, z, x)
    assert e.value.status == gs._binding.GS_ENOGAUGE
    ctx.set_gauge(to_dev(U, torch))
    st = ctx.schur_solve(1, 0, 0, z, x)
    assert st.status == 0 and torch.count_nonzero(x).item() == 0
    with pytest.raises(gs.GschurError) as e:
        ctx.schur_solve(3, 0, 0, z, x)
    assert e.value.status == gs._binding.GS_EINVAL
    with pytest.raises(gs.GschurError):
        ctx.schur_solve(2, 4, 0, z, x)
    f = to_dev(li.gaussian_source(dims, 1), torch)
    st = ctx.schur_solve(1, 0, 0, f, x, gs.gs_default_opts(inner_max_iter=1),
                         allow=(gs.GS_OK, gs.GS_MAXITER))
    assert st.status == gs.GS_MAXITER
    ctx.close()
    odd = gs.Context((3, 4, 4, 4), 0.1, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(gs.GschurError):
        odd.get_permutation(1, 0, 0, torch.empty(192, dtype=torch.int32, device="cuda:0"))
    odd.close()


_CFG1 = {}


def _cfg1_field():
    if not _CFG1:
        dims, U = li.workload_gauge("8^4 heatbath b5.4")
        _CFG1["dims"], _CFG1["U"] = dims, U
        _CFG1["D"] = dirac.wilson_matrix(U, dims, -0.4)
    return _CFG1["dims"], _CFG1["U"], _CFG1["D"]


_SREF = {}


def _schur_ref(D, dims, t, mu, inv, seed):
    """The oracle's S_bb x_b on a Gaussian x_b (inner BiCGStab to 1e-14; a
    sparse LU of D_rr is out of reach at these sizes), cached per case."""
    key = (dims, t, mu, inv, seed)
    if key not in _SREF:
        perm, nb = permute.permutation(dims, t, mu, inv)
        rng = np.random.default_rng(seed)
        xb = rng.standard_normal(nb * 12) + 1j * rng.standard_normal(nb * 12)
        op = schur.SchurOperator(D, perm, nb, inner="bicgstab", inner_tol=1e-14)
        _SREF[key] = (xb, op(xb))
    return _SREF[key]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("t,mu,inv", TYPES)
def test_schur_apply_elementwise_8x4(env, t, mu, inv, kernel, prec):
    """S_bb x_b (Section 1) on the 8^4 benchmark field (beta = 5.4 heatbath,
    m0 = -0.4), element by element against the oracle, for the four
    permutations, both inner kernels and the FP64 and mixed FP32 inner solves.
    Type I's rest set is 3840 sites: the persistent solver's grid barrier
    spans 120 tiles, the one-launch-per-phase path 120 blocks."""
    torch, gs = env
    dims, U, D = _cfg1_field()
    xb, ref = _schur_ref(D, dims, t, mu, inv, 31)
    ctx = _ctx(gs, torch, dims, -0.4, U)
    ctx.set_option(gs.GS_OPT_INNER_KERNEL, kernel)
    xbd = to_dev(xb, torch)
    ybd = torch.empty_like(xbd)
    o = gs.gs_default_opts(inner_tol=1e-14, inner_prec=gs.GS_F64 if prec == "f64" else gs.GS_F32)
    st = ctx.schur_apply(t, mu, int(inv), xbd, ybd, o)
    got = ybd.cpu().numpy()
    assert close(got, ref, 1e-11), (rel(got, ref), maxrel(got, ref))
    assert st.inner_solves == 1 and st.inner_residual <= 1e-14
    ctx.close()


def test_schur_apply_elementwise_16x32_type_II(env):
    """16^3 x 32, exp(i 0.25 H) + 5 APE steps, m0 = -0.3, Type II along x0:
    S_bb x_b on all 65536 coarse sites, element by element against the
    oracle (inner BiCGStab to 1e-14), with both inner kernels and the FP64
    and mixed FP32 inner solves.  The rest set is 65536 sites, so every
    block of the persistent grid runs many tiles."""
    torch, gs = env
    dims, U = li.workload_gauge("16^3x32 eps0.25 ape5")
    m0 = -0.3
    xb, ref = _schur_ref(dirac.wilson_matrix(U, dims, m0), dims, 2, 0, False, 32)
    ctx = _ctx(gs, torch, dims, m0, U)
    xbd = to_dev(xb, torch)
    for kernel in (0, 1):
        ctx.set_option(gs.GS_OPT_INNER_KERNEL, kernel)
        for prec in (gs.GS_F64, gs.GS_F32):
            ybd = torch.empty_like(xbd)
            st = ctx.schur_apply(2, 0, 0, xbd, ybd, gs.gs_default_opts(inner_tol=1e-14,
                                                                      inner_prec=prec))
            got = ybd.cpu().numpy()
            assert close(got, ref, 1e-11), (kernel, prec, rel(got, ref), maxrel(got, ref))
            assert st.inner_residual <= 1e-14
    ctx.close()


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("t,mu,inv", TYPES)
def test_schur_solve_8x4_heatbath_residual(env, t, mu, inv, kernel):
    """The benchmark workload: 8^4 plaquette-action field at beta = 5.4,
    m0 = -0.4, GMRES(30) to 1e-10 with back-substitution.  The GPU solution
    must solve the oracle's own D: ||f - D x|| / ||f|| <= 1e-10."""
    torch, gs = env
    dims, U, D = _cfg1_field()
    ctx = _ctx(gs, torch, dims, -0.4, U)
    ctx.set_option(gs.GS_OPT_INNER_KERNEL, kernel)
    f = li.gaussian_source(dims, 100)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    st = ctx.schur_solve(t, mu, int(inv), fd, xd)
    x = xd.cpu().numpy().ravel()
    assert np.linalg.norm(f.ravel() - D @ x) <= 1e-10 * np.linalg.norm(f)
    assert st.true_residual <= 1e-10
    ctx.close()


def test_schur_solve_8x4_matches_oracle_solution(env):
    """Type I on the benchmark workload against the oracle's own
    outer GMRES(30) / inner BiCGStab solve (both to 1e-10 / 1e-12)."""
    torch, gs = env
    dims, U, D = _cfg1_field()
    ctx = _ctx(gs, torch, dims, -0.4, U)
    f = li.gaussian_source(dims, 100)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    ctx.schur_solve(1, 0, 0, fd, xd)
    perm, nb = permute.permutation(dims, 1)
    xo, info = schur.schur_solve(D, perm, nb, f.ravel(), tol=1e-10, inner="bicgstab",
                                 inner_tol=1e-12)
    # both residuals <= 1e-10: the solutions agree to kappa(D) * 2e-10
    assert close(xd.cpu().numpy(), xo, 1e-7)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_relaxed_inner_tolerance_same_solution_fewer_iterations(env, prec):
    """Inexact Krylov on the 8^4 workload: relaxing the inner tolerance of
    later Arnoldi steps keeps the 1e-10 true residual (checked with the
    oracle's D) and the solution, with fewer inner iterations."""
    torch, gs = env
    dims, U, D = _cfg1_field()
    ctx = _ctx(gs, torch, dims, -0.4, U)
    f = li.gaussian_source(dims, 100)
    fd = to_dev(f, torch)
    xs = []
    its = []
    for relax in (0, 1):
        xd = torch.empty_like(fd)
        st = ctx.schur_solve(2, 0, 1, fd, xd,
                             gs.gs_default_opts(inner_relax=relax, inner_prec=prec))
        x = xd.cpu().numpy().ravel()
        assert np.linalg.norm(f.ravel() - D @ x) <= 1e-10 * np.linalg.norm(f)
        xs.append(x)
        its.append(st.inner_iters)
    assert close(xs[1], xs[0], 1e-7)
    assert its[1] < its[0]
    ctx.close()


def test_profile_phases_of_the_persistent_solver(env):
    """gs_profile_phases: while profiling, block 0 of the persistent FP64
    BiCGStab counts cycles per phase; the counts are non-negative, the two
    stencil phases are the largest work phases, and they are cleared when
    profiling restarts."""
    torch, gs = env
    dims = (8, 8, 4, 4)
    U = li.random_gauge(dims, 0.3, 5)
    ctx = gs.Context(dims, 0.1, torch.cuda.current_stream().cuda_stream)
    ctx.set_gauge(to_dev(U, torch))
    f = to_dev(li.gaussian_source(dims, 7), torch)
    x = torch.empty_like(f)
    ctx.schur_solve(1, 0, 0, f, x)
    ctx.profile(True)
    ctx.schur_solve(1, 0, 0, f, x)
    ph = ctx.profile_phases()
    ctx.profile(False)
    assert len(ph) == 15 and all(v >= 0 for v in ph)
    assert ph[0] > 0 and ph[6] > 0                  # v = D p and t = D s
    work = [ph[3 * s] for s in range(5)]
    assert max(work) in (ph[0], ph[6])
    ctx.profile(True)
    assert sum(ctx.profile_phases()) == 0.0
    ctx.profile(False)
    ctx.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 4)])
@pytest.mark.parametrize("t,mu,inv", [(1, 0, False), (2, 0, False), (2, 2, False), (1, 0, True),
                                      (2, 0, True), (2, 3, True)])
def test_reusken_apply_matches_oracle(env, dims, t, mu, inv):
    """S~_bb x_b (Section 3, site-block diagonal and row sums) against the
    oracle's ReuskenOperator, every permutation type."""
    from oracle import reusken
    torch, gs = env
    m0 = 0.1
    U = li.random_gauge(dims, 0.4, 9)
    ctx = gs.Context(dims, m0, torch.cuda.current_stream().cuda_stream)
    ctx.set_gauge(to_dev(U, torch))
    perm, nb = permute.permutation(dims, t, mu, inv)
    op = reusken.ReuskenOperator(dirac.wilson_matrix(U, dims, m0), perm, nb)
    rng = np.random.default_rng(3)
    xb = rng.standard_normal(nb * 12) + 1j * rng.standard_normal(nb * 12)
    xd = torch.from_numpy(xb).to("cuda:0")
    yd = torch.empty_like(xd)
    ctx.schur_apply_reusken(t, mu, inv, xd, yd)
    torch.cuda.synchronize()
    assert close(yd.cpu().numpy(), op(xb), 1e-12)
    ctx.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 4)])
@pytest.mark.parametrize("t,mu,inv", [(1, 0, False), (2, 0, False), (2, 2, False), (1, 0, True),
                                      (2, 0, True), (2, 3, True)])
def test_first_order_approximation_matches_oracle(env, dims, t, mu, inv):
    """The first-order approximation of Section 3 (D_rr's couplings ignored,
    M = d^-1) against the oracle's ReuskenOperator(order=1); order 2 through
    the same entry point is the Reusken apply itself, bit for bit."""
    from oracle import reusken
    torch, gs = env
    m0 = 0.1
    U = li.random_gauge(dims, 0.4, 9)
    ctx = _ctx(gs, torch, dims, m0, U)
    perm, nb = permute.permutation(dims, t, mu, inv)
    op = reusken.ReuskenOperator(dirac.wilson_matrix(U, dims, m0), perm, nb, order=1)
    rng = np.random.default_rng(4)
    xb = rng.standard_normal(nb * 12) + 1j * rng.standard_normal(nb * 12)
    xd = to_dev(xb, torch)
    y1, y2, y2r = torch.empty_like(xd), torch.empty_like(xd), torch.empty_like(xd)
    ctx.schur_apply_approx(t, mu, inv, 1, xd, y1)
    ctx.schur_apply_approx(t, mu, inv, 2, xd, y2)
    ctx.schur_apply_reusken(t, mu, inv, xd, y2r)
    torch.cuda.synchronize()
    assert close(y1.cpu().numpy(), op(xb), 1e-13)
    assert torch.equal(y2, y2r)
    with pytest.raises(gs.GschurError):
        ctx.schur_apply_approx(t, mu, inv, 3, xd, y1)
    ctx.close()
