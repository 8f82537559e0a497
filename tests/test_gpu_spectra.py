"""The GPU condition number (Lanczos on D^H D) and leftmost eigenvalues
(Arnoldi on D) through the C ABI: exact against dense linear algebra on tiny
lattices, and against the oracle (oracle.spectra, restarted Lanczos /
Arnoldi) on the beta = 5.4 stand-in field of Table 1 (8^4, kappa = 1/6)."""
import time

import numpy as np
import pytest

import lattice_inputs as li
from oracle import dirac, spectra
from tests.gpu_util import lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


def _ctx(gs, torch, dims, m0, U):
    ctx = gs.Context(dims, m0, torch.cuda.current_stream().cuda_stream)
    ctx.set_gauge(to_dev(U, torch))
    return ctx


@pytest.mark.parametrize("dims,m0", [((2, 2, 2, 2), -0.5), ((4, 2, 2, 2), -0.9)])
def test_condition_number_matches_dense_svd(env, dims, m0):
    torch, gs = env
    U = li.random_gauge(dims, 0.5, 7)
    D = dirac.wilson_matrix(U, dims, m0).toarray()
    sv = np.linalg.svd(D, compute_uv=False)
    ctx = _ctx(gs, torch, dims, m0, U)
    start = to_dev(li.gaussian_source(dims, 12), torch)
    kappa, smin, smax, steps = ctx.condition_number(start, max_steps=4000, tol=1e-10)
    assert abs(smax - sv[0]) <= 1e-8 * sv[0]
    assert abs(smin - sv[-1]) <= 1e-8 * sv[0]
    assert abs(kappa - sv[0] / sv[-1]) <= 1e-6 * kappa
    assert 20 <= steps <= 4000
    ctx.close()


@pytest.mark.parametrize("dims,m0", [((2, 2, 2, 2), -0.5), ((4, 2, 2, 2), -0.9)])
def test_arnoldi_on_the_whole_space_gives_the_dense_spectrum(env, dims, m0):
    """m = N Arnoldi steps span the whole space: the Ritz values are the
    eigenvalues, which checks the Hessenberg QR iteration as well."""
    torch, gs = env
    U = li.random_gauge(dims, 0.5, 8)
    D = dirac.wilson_matrix(U, dims, m0).toarray()
    dense = np.linalg.eigvals(D)
    N = D.shape[0]
    ctx = _ctx(gs, torch, dims, m0, U)
    start = to_dev(li.gaussian_source(dims, 13), torch)
    got = np.array(ctx.leftmost_eigenvalues(start, m=N, k=8))
    want = dense[np.lexsort((dense.imag, dense.real))][:8]
    assert np.all(np.diff(got.real) >= -1e-12)
    assert np.allclose(got.real, want.real, atol=1e-9)
    for z in got:                                   # each one an eigenvalue of D
        assert np.abs(dense - z).min() < 1e-9
    ctx.close()


def test_table1_condition_number_and_leftmost_eigenvalue_match_oracle(env):
    """beta = 5.4 stand-in field, kappa = 1/6: the condition number from GPU
    Lanczos (tolerance 1e-6) against the oracle's restarted Lanczos, and the
    eigenvalues of smallest real part from 1200 Arnoldi steps against the
    oracle's restarted Arnoldi."""
    torch, gs = env
    dims, U = li.coupling_gauge(5.4, 0)
    D = dirac.wilson_matrix(U, dims, -1.0).tocsr()
    t0 = time.time()
    kappa_o, smin_o, smax_o = spectra.condition_number(D, tol=1e-6)
    ev_o = spectra.leftmost_eigenvalues(D, k=2, tol=1e-6)
    oracle_s = time.time() - t0
    ctx = _ctx(gs, torch, dims, -1.0, U)
    start = to_dev(li.gaussian_source(dims, 14), torch)
    t0 = time.time()
    kappa, smin, smax, steps = ctx.condition_number(start, max_steps=20000, tol=1e-6)
    ev = ctx.leftmost_eigenvalues(start, m=1200, k=2)
    gpu_s = time.time() - t0
    assert abs(kappa - kappa_o) <= 1e-4 * kappa_o, (kappa, kappa_o)
    assert abs(smin - smin_o) <= 1e-4 * smin_o and abs(smax - smax_o) <= 1e-4 * smax_o
    # gamma_5-hermiticity: D's eigenvalues come in complex-conjugate pairs, so
    # a converged leftmost pair is symmetric
    assert abs(ev[0] - np.conj(ev[1])) <= 2e-6, ev
    assert abs(ev[0].real - ev_o[0].real) <= 2e-6, (ev, ev_o)
    assert abs(abs(ev[0].imag) - abs(ev_o[0].imag)) <= 2e-6
    print("\ncondition number %.4f (oracle %.4f), %d Lanczos steps; leftmost %s (oracle %s); "
          "GPU %.2f s, oracle %.1f s" % (kappa, kappa_o, steps, ev[0], ev_o[0], gpu_s, oracle_s))
    ctx.close()


def test_spectra_argument_errors(env):
    torch, gs = env
    dims = (2, 2, 2, 2)
    ctx = _ctx(gs, torch, dims, 0.1, li.random_gauge(dims, 0.3, 1))
    z = torch.zeros(li.volume(dims) * 12, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(gs.GschurError):
        ctx.condition_number(z)                           # zero start vector
    s = to_dev(li.gaussian_source(dims, 1), torch)
    for m, k in ((1, 1), (500, 1), (10, 11)):
        with pytest.raises(gs.GschurError):
            ctx.leftmost_eigenvalues(s, m=m, k=k)
    ctx.close()
