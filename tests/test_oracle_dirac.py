"""Pins of the oracle's Wilson-Dirac matrix against facts the operator must obey.

None of these retypes the oracle's formula: they test the Clifford algebra,
the textbook momentum-space form at U = 1, the free spectrum, gamma_5-
hermiticity and gauge covariance, each of which a dropped term, a wrong sign,
a wrong link index or a missing dagger would break.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linear_sum_assignment

import lattice_inputs as li
from oracle import dirac


def test_gamma_clifford_and_hermitian():
    G = dirac.GAMMA
    for a in range(4):
        assert np.allclose(G[a], G[a].conj().T)
        for b in range(4):
            acomm = G[a] @ G[b] + G[b] @ G[a]
            assert np.allclose(acomm, 2.0 * (a == b) * np.eye(4), atol=0)
    # chiral basis: gamma_5 = g1 g2 g3 g4 is diagonal (+1, +1, -1, -1)
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))


def _unit_gauge(dims):
    V = li.volume(dims)
    return np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()


@pytest.mark.parametrize("dims", [(4, 3, 2, 5), (2, 2, 2, 2), (6, 4, 4, 2)])
def test_plane_wave_closed_form(dims):
    """At U = 1, psi(x) = exp(i p.x) u is mapped to D(p) psi with
    D(p) = m0 + r sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu."""
    m0 = -0.37
    D = dirac.wilson_matrix(_unit_gauge(dims), dims, m0)
    x = dirac.coords(dims)
    rng = np.random.default_rng(5)
    for trial in range(4):
        n = np.array([rng.integers(0, L) for L in dims])
        p = 2 * np.pi * n / np.array(dims)
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (x @ p))
        psi = (phase[:, None, None] * u[None]).ravel()
        Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(
            dirac.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
        expect = (phase[:, None, None] * (Dp @ u)[None]).ravel()
        assert np.allclose(D @ psi, expect, atol=1e-13, rtol=0)


def test_free_field_spectrum():
    """Eigenvalues at U = 1: m0 + r sum(1 - cos p) +- i sqrt(sum sin^2 p), each 6-fold."""
    dims = (4, 4, 2, 3)
    m0 = 0.15
    D = dirac.wilson_matrix(_unit_gauge(dims), dims, m0).toarray()
    ev = np.linalg.eigvals(D)
    expect = []
    for n0 in range(dims[0]):
        for n1 in range(dims[1]):
            for n2 in range(dims[2]):
                for n3 in range(dims[3]):
                    p = 2 * np.pi * np.array([n0, n1, n2, n3]) / np.array(dims)
                    re = m0 + np.sum(1 - np.cos(p))
                    im = np.sqrt(np.sum(np.sin(p) ** 2))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.array(expect)
    cost = np.abs(ev[:, None] - expect[None, :])
    r, c = linear_sum_assignment(cost)
    assert cost[r, c].max() < 1e-10


@pytest.mark.parametrize("dims", [(3, 4, 2, 5), (4, 4, 4, 4)])
def test_gamma5_hermiticity(dims):
    U = li.random_gauge(dims, 0.4, 11)
    D = dirac.wilson_matrix(U, dims, -0.3)
    V = li.volume(dims)
    G5 = sp.kron(sp.eye(V), sp.kron(dirac.GAMMA5, sp.eye(3))).tocsr()
    assert abs(D.conj().T - G5 @ D @ G5).max() < 1e-15


@pytest.mark.parametrize("dims", [(3, 4, 2, 5), (2, 2, 2, 2)])
def test_gauge_covariance(dims):
    """D[U^g] (G psi) = G D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    V = li.volume(dims)
    U = li.random_gauge(dims, 0.5, 3)
    g = li.random_su3((V,), 4)
    Ug = np.empty_like(U)
    for mu in range(4):
        fwd = dirac.neighbour(dims, mu, +1)
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[fwd], -1, -2))
    m0 = 0.1
    D = dirac.wilson_matrix(U, dims, m0)
    Dg = dirac.wilson_matrix(Ug, dims, m0)
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    Gpsi = np.einsum("sij,saj->sai", g, psi)
    lhs = (Dg @ Gpsi.ravel()).reshape(V, 4, 3)
    rhs = np.einsum("sij,saj->sai", g, (D @ psi.ravel()).reshape(V, 4, 3))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_hopping_parameter_relation():
    assert dirac.kappa_to_m0(1.0 / 6.0) == pytest.approx(-1.0)
    assert dirac.kappa_to_m0(1.0 / 8.0) == pytest.approx(0.0)


def test_two_site_extent_adds_both_hops():
    """On L_mu = 2 the forward and backward neighbours coincide; the block to
    that neighbour must be the sum of both hopping terms: at U = 1 it is
    -1/2 [(1 - g) + (1 + g)] (x) 1_3 = -1 (x) 1_3."""
    dims = (2, 3, 3, 3)
    D = dirac.wilson_matrix(_unit_gauge(dims), dims, 0.0).toarray()
    s, t = 0, 1  # sites (0,0,0,0) and (1,0,0,0)
    blk = D[12 * s:12 * s + 12, 12 * t:12 * t + 12]
    assert np.allclose(blk, -np.eye(12))


def test_sampled_rows_equal_full_matrix_rows():
    dims = (3, 4, 2, 4)
    U = li.random_gauge(dims, 0.4, 12)
    D = dirac.wilson_matrix(U, dims, 0.1)
    sites = np.array([0, 5, 17, 95])
    Ds = dirac.wilson_matrix(U, dims, 0.1, rows_of=sites)
    idx = (12 * sites[:, None] + np.arange(12)[None]).ravel()
    assert abs(Ds - D[idx]).max() == 0
