"""Pins of the oracle's gauge-equivariant network and its gradients."""
import numpy as np
import pytest

import lattice_inputs as li
from oracle import dirac, net


def _setup(dims=(4, 2, 2, 4), C=3, seed=0):
    U = li.random_gauge(dims, 0.5, seed)
    tr = net.transports(U, dims)
    Ws = net.init_weights(C, seed + 1, scale=0.3)
    return U, tr, Ws


def test_gauge_equivariance():
    dims = (4, 2, 2, 4)
    V = li.volume(dims)
    U, tr, Ws = _setup(dims)
    g = li.random_su3((V,), 7)
    Ug = np.empty_like(U)
    for mu in range(4):
        fwd = dirac.neighbour(dims, mu, +1)
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[fwd], -1, -2))
    trg = net.transports(Ug, dims)
    psi = li.gaussian_source(dims, 3)
    out = net.forward(Ws, psi, tr)[-1].reshape(V, 4, 3)
    outg = net.forward(Ws, np.einsum("vab,vsb->vsa", g, psi), trg)[-1].reshape(V, 4, 3)
    assert np.abs(outg - np.einsum("vab,vsb->vsa", g, out)).max() < 1e-12 * np.abs(out).max()


def test_linearity_and_translation():
    dims = (4, 2, 2, 4)
    V = li.volume(dims)
    U, tr, Ws = _setup(dims)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    t1, t2 = li.gaussian_source(dims, 1), li.gaussian_source(dims, 2)
    M = lambda t: net.forward(Ws, t, tr)[-1].ravel()   # noqa: E731
    assert np.abs(M(a * t1 + b * t2) - a * M(t1) - b * M(t2)).max() < 1e-12 * np.abs(M(t1)).max()
    # shift everything by one site along x3
    sh = lambda F: np.roll(F.reshape(dims[::-1] + F.shape[1:]), 1, axis=0).reshape(F.shape)  # noqa: E731
    trs = net.transports(sh(U), dims)
    out_s = net.forward(Ws, sh(t1), trs)[-1]
    assert np.abs(out_s - sh(net.forward(Ws, t1, tr)[-1])).max() < 1e-12 * np.abs(out_s).max()


def test_identity_weight_reduces_to_scaling():
    dims = (2, 2, 2, 2)
    U = li.random_gauge(dims, 0.5, 4)
    tr = net.transports(U, dims)
    W = np.zeros((9, 4, 4), complex)
    W[0] = (0.25 - 0.5j) * np.eye(4)
    psi = li.gaussian_source(dims, 6)
    out = net.layer(W, psi.reshape(-1, 1, 4, 3), tr)
    assert np.allclose(out.reshape(psi.shape), (0.25 - 0.5j) * psi, atol=1e-15)


@pytest.mark.parametrize("layer_idx", [0, 1, 2])
def test_gradients_match_finite_differences(layer_idx):
    dims = (4, 2, 2, 2)
    V = li.volume(dims)
    U, tr, Ws = _setup(dims, C=2, seed=3)
    rng = np.random.default_rng(11)
    rest = rng.random(V) < 0.8          # an arbitrary rest set
    t = li.gaussian_source(dims, 8) * rest[:, None, None]
    z = (li.gaussian_source(dims, 9) * rest[:, None, None])[rest]

    def L(ws):
        y = net.forward(ws, t, tr)[-1].reshape(V, 4, 3)[rest]
        return net.loss(y, z)

    acts = net.forward(Ws, t, tr)
    y = acts[-1].reshape(V, 4, 3)
    gy = np.zeros_like(y)
    gy[rest] = 2.0 * (y[rest] - z) / np.vdot(z, z).real
    grads = net.backward(Ws, acts, gy.reshape(V, 1, 4, 3), tr)
    E = rng.standard_normal(Ws[layer_idx].shape) + 1j * rng.standard_normal(Ws[layer_idx].shape)
    eps = 1e-6
    wp = [w.copy() for w in Ws]
    wm = [w.copy() for w in Ws]
    wp[layer_idx] += eps * E
    wm[layer_idx] -= eps * E
    fd = (L(wp) - L(wm)) / (2 * eps)
    an = np.vdot(grads[layer_idx], E).real
    assert abs(fd - an) <= 1e-6 * abs(an)
