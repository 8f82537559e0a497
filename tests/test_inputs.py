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
