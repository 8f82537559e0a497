"""Pins of the oracle's Krylov solvers against a direct sparse solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle import krylov


def _system(n=400, seed=1):
    rng = np.random.default_rng(seed)
    A = (sp.random(n, n, density=0.02, random_state=seed) * (1 + 0.7j)
         + sp.diags(3.0 + rng.random(n))).tocsr()
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b, sla.spsolve(A.tocsc(), b)


@pytest.mark.parametrize("solver", ["bicgstab", "gmres30", "gmres4"])
def test_solver_matches_direct(solver):
    A, b, xd = _system()
    if solver == "bicgstab":
        x, info = krylov.bicgstab(lambda v: A @ v, b, tol=1e-12)
    else:
        m = int(solver[5:])
        x, info = krylov.gmres(lambda v: A @ v, b, m=m, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 1.0001
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_gmres_exact_in_n_steps():
    """Without restart GMRES on an n x n system terminates in <= n steps."""
    A, b, xd = _system(n=25, seed=4)
    x, info = krylov.gmres(lambda v: A @ v, b, m=25, tol=1e-14)
    assert info["iters"] <= 25
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_zero_rhs_and_maxiter():
    A, b, _ = _system(n=50)
    x, info = krylov.bicgstab(lambda v: A @ v, np.zeros(50, complex))
    assert info["converged"] and not np.any(x)
    x, info = krylov.gmres(lambda v: A @ v, b, m=3, tol=1e-14, maxiter=2)
    assert not info["converged"] and info["iters"] == 2


def test_convergence_rate_geometric():
    h = [1.0 * 0.5 ** k for k in range(11)]
    assert krylov.convergence_rate(h) == pytest.approx(0.5)


def test_bicgstab_iterates_match_an_independent_implementation():
    """The first iterates of van der Vorst's recurrence are fixed by the
    algorithm (x0 = 0, shadow residual r0): they must equal SciPy's
    independent implementation step by step (a wrong conjugation in alpha or
    omega still converges, but along a different path)."""
    A, b, _ = _system()
    ref = []
    sla.bicgstab(A, b, rtol=1e-12, atol=0.0, callback=lambda xk: ref.append(xk.copy()))
    for k in range(1, 6):
        x, _ = krylov.bicgstab(lambda v: A @ v, b, tol=1e-30, maxiter=k)
        assert np.linalg.norm(x - ref[k - 1]) <= 1e-13 * np.linalg.norm(x)


def test_gmres_first_cycle_minimises_residual():
    """After k Arnoldi steps GMRES returns the minimiser of ||b - A x|| over
    the Krylov space K_k(A, b); compare with a dense least-squares solve."""
    A, b, _ = _system(n=60, seed=2)
    Ad = A.toarray()
    for k in (1, 3, 7):
        x, _ = krylov.gmres(lambda v: A @ v, b, m=k, tol=1e-30, maxiter=k)
        K = np.stack([np.linalg.matrix_power(Ad, i) @ b for i in range(k)], 1)
        c = np.linalg.lstsq(Ad @ K, b, rcond=None)[0]
        assert np.linalg.norm(x - K @ c) <= 1e-9 * np.linalg.norm(x)


def test_mean_ratio_against_geometric_rate():
    """Arithmetic mean of successive ratios: equals the geometric rate on a
    geometric sequence and exceeds it otherwise (AM-GM); worked example
    1, 0.5, 0.05: ratios 0.5 and 0.1, mean 0.3, geometric sqrt(0.05)."""
    h = [1.0 * 0.3 ** k for k in range(8)]
    assert krylov.mean_ratio(h) == pytest.approx(0.3)
    assert krylov.convergence_rate(h) == pytest.approx(0.3)
    h = [1.0, 0.5, 0.05]
    assert krylov.mean_ratio(h) == pytest.approx(0.3)
    assert krylov.convergence_rate(h) == pytest.approx(0.05 ** 0.5)
    assert krylov.mean_ratio([2.0]) == 0.0
