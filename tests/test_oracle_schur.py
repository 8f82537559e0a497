"""Pins of the oracle's Schur complement, apply and solve (Section 1).

Each pin is an identity the paper states or that follows from the algebra it
uses, checked with arithmetic that does not go through ``schur_dense``'s
formula: determinants by dense LU, the general Gaussian-integration form,
inverse blocks of D, direct sparse solves and the quotient property.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import lattice_inputs as li
from oracle import dirac, permute, schur
from oracle.permute import TYPE_I, TYPE_II, expand_sites

FOUR = [(TYPE_I, 0, False), (TYPE_II, 0, False), (TYPE_I, 0, True), (TYPE_II, 0, True)]


def _field(dims, eps=0.3, seed=0):
    return li.random_gauge(dims, eps, seed)


@pytest.mark.parametrize("t,mu,inv", FOUR + [(TYPE_II, 3, False), (TYPE_II, 2, True)])
def test_det_factorisation_2x4(t, mu, inv):
    """det D = det S_bb det D_rr (Section 1, item ii), dense LU on 2^4."""
    dims = (2, 2, 2, 2)
    D = dirac.wilson_matrix(_field(dims), dims, 0.2)
    perm, nb = permute.permutation(dims, t, mu, inv)
    S = schur.schur_dense(D, perm, nb)
    _, _, _, Drr = schur.partition(D, perm, nb)
    sD, lD = np.linalg.slogdet(D.toarray())
    sS, lS = np.linalg.slogdet(S)
    sR, lR = np.linalg.slogdet(Drr.toarray())
    assert abs(lD - (lS + lR)) <= 1e-12 * abs(lD)
    assert abs(sD - sS * sR) < 1e-12


@pytest.mark.parametrize("t,mu,inv", [(TYPE_II, 0, False), (TYPE_II, 1, True), (TYPE_I, 0, True)])
def test_gaussian_form_and_det_Dtilde(t, mu, inv):
    """With B = (0, D_bb^-1 D_br), B-bar = (0; D_rb D_bb^-1) and
    D~ = D + B-bar D_bb B, the Gaussian-integration form
    S = D_bb - D_bb B D~^-1 B-bar D_bb equals D_bb - D_br D_rr^-1 D_rb, and
    det D~ = det D_bb det D_rr (Section 1, the three displayed identities)."""
    dims = (2, 2, 2, 4)
    D = dirac.wilson_matrix(_field(dims, 0.35, 7), dims, 0.25)
    perm, nb = permute.permutation(dims, t, mu, inv)
    P = permute.perm_matrix(perm, 12)
    Dp = (P @ D @ P.T).toarray()           # coarse block first
    n = 12 * nb
    Dbb, Dbr, Drb, Drr = Dp[:n, :n], Dp[:n, n:], Dp[n:, :n], Dp[n:, n:]
    N = Dp.shape[0]
    Dbb_inv = np.linalg.inv(Dbb)
    B = np.zeros((n, N), dtype=complex)
    B[:, n:] = Dbb_inv @ Dbr
    Bbar = np.zeros((N, n), dtype=complex)
    Bbar[n:, :] = Drb @ Dbb_inv
    Dt = Dp + Bbar @ Dbb @ B
    S_gauss = Dbb - Dbb @ B @ np.linalg.solve(Dt, Bbar @ Dbb)
    S = schur.schur_dense(D, perm, nb)
    assert np.abs(S_gauss - S).max() <= 1e-12 * np.abs(S).max()
    lt = np.linalg.slogdet(Dt)[1]
    assert abs(lt - (np.linalg.slogdet(Dbb)[1] + np.linalg.slogdet(Drr)[1])) <= 1e-12 * abs(lt)


@pytest.mark.parametrize("t,mu,inv", FOUR)
def test_schur_inverse_is_block_of_inverse(t, mu, inv):
    """S_bb^-1 = (D^-1)_bb: the coarse block of the inverse of P D P^T."""
    dims = (2, 2, 4, 2)
    D = dirac.wilson_matrix(_field(dims, 0.3, 1), dims, 0.2)
    perm, nb = permute.permutation(dims, t, mu, inv)
    S = schur.schur_dense(D, perm, nb)
    bi = expand_sites(perm[:nb])
    Dinv = np.linalg.inv(D.toarray())
    assert np.abs(np.linalg.inv(S) - Dinv[np.ix_(bi, bi)]).max() < 1e-12 * np.abs(Dinv).max()


@pytest.mark.parametrize("t,mu,inv", FOUR)
def test_gamma5_hermiticity_of_S(t, mu, inv):
    """gamma_5 is site-local, so S_bb^dag = G5 S_bb G5 on the coarse set."""
    dims = (4, 2, 2, 2)
    D = dirac.wilson_matrix(_field(dims, 0.4, 2), dims, -0.2)
    perm, nb = permute.permutation(dims, t, mu, inv)
    S = schur.schur_dense(D, perm, nb)
    G5 = np.kron(np.eye(nb), np.kron(dirac.GAMMA5, np.eye(3)))
    assert np.abs(S.conj().T - G5 @ S @ G5).max() < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("t,mu,inv", FOUR)
def test_gauge_covariance_of_S(t, mu, inv):
    """S_bb[U^g] = G_b S_bb[U] G_b^dag, G_b = diag over b of 1_4 (x) g(x)."""
    dims = (2, 4, 2, 2)
    V = li.volume(dims)
    U = _field(dims, 0.4, 8)
    g = li.random_su3((V,), 9)
    Ug = np.empty_like(U)
    for m in range(4):
        fwd = dirac.neighbour(dims, m, +1)
        Ug[:, m] = g @ U[:, m] @ np.conj(np.swapaxes(g[fwd], -1, -2))
    perm, nb = permute.permutation(dims, t, mu, inv)
    S = schur.schur_dense(dirac.wilson_matrix(U, dims, 0.3), perm, nb)
    Sg = schur.schur_dense(dirac.wilson_matrix(Ug, dims, 0.3), perm, nb)
    Gb = scipy.linalg.block_diag(*[np.kron(np.eye(4), g[s]) for s in perm[:nb]])
    assert np.abs(Sg - Gb @ S @ Gb.conj().T).max() < 1e-12 * np.abs(S).max()


def test_quotient_property_type_II_steps_equal_type_I():
    """Four exact one-direction steps (mu = 0, 1, 2, 3, each on the coarse
    lattice of the step before) give the Type I Schur complement on 4^4."""
    dims = [4, 4, 4, 4]
    D = dirac.wilson_matrix(_field(tuple(dims), 0.3, 0), tuple(dims), 0.2)
    pI, nbI = permute.permutation(tuple(dims), TYPE_I)
    S_I = schur.schur_dense(D, pI, nbI)
    A = D.toarray()
    cur = list(dims)
    for mu in range(4):
        perm, nb = permute.permutation(tuple(cur), TYPE_II, mu)
        bi = expand_sites(perm[:nb])
        ri = expand_sites(perm[nb:])
        A = A[np.ix_(bi, bi)] - A[np.ix_(bi, ri)] @ np.linalg.solve(
            A[np.ix_(ri, ri)], A[np.ix_(ri, bi)])
        cur[mu] //= 2
    assert np.abs(A - S_I).max() < 1e-11 * np.abs(S_I).max()


@pytest.mark.parametrize("t,mu,inv", FOUR)
def test_solve_through_S_equals_direct_solve(t, mu, inv):
    """Coarse solve + back-substitution (the block UL factorisation)
    reproduces the direct sparse solve of D x = f on 4^4."""
    dims = (4, 4, 4, 4)
    D = dirac.wilson_matrix(_field(dims), dims, 0.2)
    f = li.gaussian_source(dims, 100).ravel()
    perm, nb = permute.permutation(dims, t, mu, inv)
    x, info = schur.schur_solve(D, perm, nb, f, tol=1e-12, inner="direct")
    xd = sla.spsolve(D.tocsc(), f)
    assert info["converged"]
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert np.linalg.norm(f - D @ x) <= 1e-11 * np.linalg.norm(f)


def test_iterative_inner_matches_direct_and_known_solution():
    dims = (4, 4, 4, 4)
    D = dirac.wilson_matrix(_field(dims), dims, 0.2)
    perm, nb = permute.permutation(dims, TYPE_I)
    rng = np.random.default_rng(3)
    xb = rng.standard_normal(12 * nb) + 1j * rng.standard_normal(12 * nb)
    Sd = schur.SchurOperator(D, perm, nb, inner="direct")
    Si = schur.SchurOperator(D, perm, nb, inner="bicgstab", inner_tol=1e-14)
    y1, y2 = Sd(xb), Si(xb)
    assert np.linalg.norm(y1 - y2) <= 1e-12 * np.linalg.norm(y1)
    # known solution: x random, f = D x
    x = rng.standard_normal(D.shape[0]) + 1j * rng.standard_normal(D.shape[0])
    f = D @ x
    xs, info = schur.schur_solve(D, perm, nb, f, tol=1e-11, inner="bicgstab",
                                 inner_tol=1e-13)
    assert np.linalg.norm(xs - x) <= 1e-9 * np.linalg.norm(x)


def test_type_I_coarse_block_is_diagonal():
    """Type I coarse sites have no coarse neighbours: D_bb = (m0 + 4) 1."""
    dims = (4, 4, 4, 4)
    m0 = -0.4
    D = dirac.wilson_matrix(_field(dims), dims, m0)
    perm, nb = permute.permutation(dims, TYPE_I)
    Dbb, _, _, _ = schur.partition(D, perm, nb)
    assert abs(Dbb - (m0 + 4) * sp.eye(12 * nb)).max() < 1e-15
