"""Checks of the seeded gauge-field and source generators."""
import numpy as np
import pytest

import lattice_inputs as li


def _su3_ok(U):
    I = np.eye(3)
    un = np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - I).max()
    dt = np.abs(np.linalg.det(U) - 1).max()
    return un < 1e-12 and dt < 1e-12


def test_random_gauge_su3_and_seeded():
    d = (4, 2, 2, 4)
    U = li.random_gauge(d, 0.3, 0)
    assert U.shape == (64, 4, 3, 3) and _su3_ok(U)
    assert np.array_equal(U, li.random_gauge(d, 0.3, 0))
    assert not np.array_equal(U, li.random_gauge(d, 0.3, 1))
    # eps -> 0 gives the unit field
    assert np.abs(li.random_gauge(d, 0.0, 0) - np.eye(3)).max() < 1e-14


def test_ape_smearing_is_su3_and_smooths():
    d = (4, 4, 4, 4)
    U = li.random_gauge(d, 0.3, 0)
    S = li.ape_smear(U, d, 0.5, 3)
    assert _su3_ok(S)
    assert li.average_plaquette(S, d) > li.average_plaquette(U, d)
    # a unit field is a fixed point
    I = li.random_gauge(d, 0.0, 0)
    assert np.abs(li.ape_smear(I, d, 0.5, 2) - np.eye(3)).max() < 1e-13


def test_heatbath_limits():
    """Strong coupling: <P> = beta/18 + O(beta^2); weak coupling: 1 - 2/beta."""
    d = (8, 8, 4, 4)
    U = li.heatbath_gauge(d, 0.6, 8, 3)
    assert _su3_ok(U)
    assert abs(li.average_plaquette(U, d) - 0.6 / 18) < 0.012
    d2 = (4, 4, 4, 4)
    U = li.heatbath_gauge(d2, 30.0, 15, 4)
    assert abs(li.average_plaquette(U, d2) - (1 - 2 / 30.0)) < 0.01


def test_heatbath_is_the_same_on_every_machine():
    """The heatbath chain turns a last-bit rounding difference into another
    configuration, so it uses correctly rounded float64 operations only: this
    4^4 field has the same bytes on x86-64 and on aarch64 (the digest was
    taken on both)."""
    import hashlib
    U = li.heatbath_gauge((4, 4, 4, 4), 5.4, 10, 3)
    assert _su3_ok(U)
    digest = hashlib.sha256(np.ascontiguousarray(U).tobytes()).hexdigest()
    assert digest == "bbfa43e5a479a2d7dbd2badd41e4f748a4d3a782a575a19ef70ad061d85339d5"


def test_staples_on_a_parity_equal_the_whole_lattice_sum():
    """The heatbath computes the staples of one parity's links only; they are
    the whole-lattice staple sum at those sites, bit for bit, and the staple
    closes the plaquettes: Re tr(U_mu(x) A_mu(x)) summed over x is twice the
    sum over x of the plaquettes in the planes (mu, nu != mu)."""
    d = (4, 2, 4, 2)
    U = li.random_gauge(d, 0.4, 8)
    G = li._to_grid(U, d)
    fwd, bwd = li._nbr_tables(d)
    par = li._parity_mask(d).ravel()
    for mu in range(4):
        full = li._staple_sum(G, mu).reshape(-1, 3, 3)
        for p in (0, 1):
            S = np.flatnonzero(par == p)
            part = li._staple_sites(U, mu, S, fwd, bwd)
            assert np.array_equal(part, full[S])
    mu = 1
    A = li._staple_sum(G, mu).reshape(-1, 3, 3)
    lhs = np.einsum("xab,xba->", U[:, mu], A).real
    rhs = 0.0
    for nu in range(4):
        if nu == mu:
            continue
        Um, Un = G[..., mu, :, :], G[..., nu, :, :]
        P = Um @ li._shift(Un, mu, 1) @ li._dag(li._shift(Um, nu, 1)) @ li._dag(Un)
        rhs += 2.0 * np.trace(P, axis1=-2, axis2=-1).real.sum()
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_library_helpers_of_the_heatbath():
    """The correctly rounded helpers against numpy / LAPACK: complex products,
    the SU(3) re-unitarisation, the logarithm, points on the circle."""
    rng = np.random.default_rng(5)
    A = rng.normal(size=(40, 3, 3)) + 1j * rng.normal(size=(40, 3, 3))
    B = rng.normal(size=(40, 3, 2)) + 1j * rng.normal(size=(40, 3, 2))
    assert np.abs(li._cmm(A, B) - A @ B).max() < 1e-13
    W = li._reunitarize(A)
    assert np.abs(W @ np.conj(np.swapaxes(W, -1, -2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(W) - 1).max() < 1e-14
    # Gram-Schmidt: the first row is the normalised first row of the input
    assert np.abs(W[:, 0] - A[:, 0] / np.linalg.norm(A[:, 0], axis=1)[:, None]).max() < 1e-15
    x = np.concatenate([rng.random(1000) * 5 + 1e-300, np.exp(rng.uniform(-700, 700, 1000))])
    assert np.abs(li._log(x) - np.log(x)).max() < 1e-12
    c, s = li._unit_circle(5000, rng)
    assert np.abs(c * c + s * s - 1).max() < 1e-15
    assert abs(np.mean(c * c) - 0.5) < 0.02 and abs(np.mean(c)) < 0.03


def test_sources():
    d = (2, 2, 2, 2)
    s = li.gaussian_source(d, 100)
    assert s.shape == (16, 4, 3) and s.dtype == np.complex128
    assert np.array_equal(s, li.gaussian_source(d, 100))
    P = li.point_sources(d)
    assert P.shape == (12, 16, 4, 3)
    assert np.array_equal(P.reshape(12, -1)[:, :12], np.eye(12))


def test_torch_generator_matches_numpy_recipe():
    """The torch route (Taylor exp, Newton polar factor) reproduces the numpy
    route (eigh, SVD) of the same seeded recipe to rounding."""
    torch = pytest.importorskip("torch")
    from lattice_inputs import torchgen
    dims = (4, 4, 2, 4)
    for eps in (0.2, 0.6):
        U = li.random_gauge(dims, eps, 5)
        Ut = torchgen.random_gauge_t(dims, eps, 5)
        assert np.abs(U - Ut.numpy()).max() < 1e-13
        A = li.ape_smear(U, dims, 0.5, 4)
        At = torchgen.ape_smear_t(Ut, dims, 0.5, 4).numpy()
        assert np.abs(A - At).max() < 1e-13
        # SU(3): unitary with unit determinant
        assert np.abs(At @ np.conj(np.swapaxes(At, -1, -2)) - np.eye(3)).max() < 1e-13
        assert np.abs(np.linalg.det(At) - 1).max() < 1e-13
