"""Gauge-equivariant linear convolutional network (oracle).

Test infrastructure, like the rest of ``oracle/``.

The learned preconditioner M ~ D_rr^-1 used inside flexible GMRES for the
inner solve.  (The paper's own preconditioner is the Reusken approximation
and a V-cycle, Section 4; the learned one replaces the hand-made
approximation of D_rr^-1 by one fitted to pairs (t, D_rr^-1 t) that the
method itself produces.)

A layer maps C_in channels of spinor fields psi(x) in C^{C_in x 4 x 3}
(channel, spin, colour) to C_out channels:

    out(x)[o, s, a] = sum_{d = 0..8} sum_{i, r} W_d[(o, s), (i, r)] (U_d(x) psi(x + d)[i, r])[a]

with the nine parallel transports d = 0 (x itself, U = 1), d = 1 + mu
(+mu-hat: U_mu(x) psi(x + mu)) and d = 5 + mu (-mu-hat: U_mu(x - mu)^dag
psi(x - mu)).  W_d acts on channel (x) spin and the transport on colour, so
a gauge rotation psi -> g psi, U_mu(x) -> g(x) U_mu(x) g(x + mu)^dag maps
out -> g out: the layer is gauge equivariant.  It is linear (D_rr^-1 t is
linear in t), so the network is a learned polynomial in the hopping terms
with channel/spin mixing.

Network: 3 layers, channels 1 -> C -> C -> 1 (C = 24); the input is the
rest-set vector t embedded in the whole lattice (zero on the coarse sites),
the output is restricted to the rest set.  Loss of a pair (t, z):
||M(t)|_r - z||^2 / ||z||^2.

Gradients are real-pair gradients g = dL/dRe + i dL/dIm, for which y = A x
gives g_x = A^H g_y and y = W T gives g_W = g_y T^H (summed over sites and
colour).  The transport of the input gradient is the forward convolution
with weights W'_0 = W_0^H, W'_{+mu} = W_{-mu}^H, W'_{-mu} = W_{+mu}^H.

Pins (tests/test_oracle_net.py): gauge equivariance under random SU(3)
transformations, linearity, translation equivariance, the analytic
gradients against central finite differences in FP64, and a one-layer
network with only W_0 = c 1 reducing to c times the identity.
"""
from __future__ import annotations

import numpy as np

from .dirac import neighbour

__all__ = ["transports", "layer", "forward", "loss", "backward", "n_params", "init_weights"]


def transports(U, dims):
    """Neighbour index and 3x3 transport matrix of the nine terms: lists of
    (nbr[V], T[V, 3, 3]) for d = 0 .. 8."""
    V = int(np.prod(dims))
    U = np.asarray(U).reshape(V, 4, 3, 3)
    out = [(np.arange(V), np.broadcast_to(np.eye(3), (V, 3, 3)))]
    for mu in range(4):
        out.append((neighbour(dims, mu, +1), U[:, mu]))
    for mu in range(4):
        bwd = neighbour(dims, mu, -1)
        out.append((bwd, np.conj(np.swapaxes(U[bwd, mu], -1, -2))))
    return out


def layer(W, psi, tr):
    """One layer.  W: (9, 4 C_out, 4 C_in) complex; psi: (V, C_in, 4, 3).
    Returns (V, C_out, 4, 3)."""
    V, cin = psi.shape[0], psi.shape[1]
    cout = W.shape[1] // 4
    x = psi.reshape(V, 4 * cin, 3)
    out = np.zeros((V, 4 * cout, 3), dtype=np.complex128)
    for d, (nbr, T) in enumerate(tr):
        moved = np.einsum("vab,vkb->vka", T, x[nbr])      # U_d(x) psi(x + d)
        out += np.einsum("ok,vka->voa", W[d], moved)       # channel/spin mixing
    return out.reshape(V, cout, 4, 3)


def n_params(channels=24):
    return [(9, 4 * channels, 4), (9, 4 * channels, 4 * channels), (9, 4, 4 * channels)]


def init_weights(channels, seed, scale=None):
    """Random complex weights (Gaussian, seeded) for the 1 -> C -> C -> 1 net."""
    rng = np.random.default_rng(seed)
    Ws = []
    for shape in n_params(channels):
        s = scale if scale is not None else 1.0 / np.sqrt(2.0 * 9 * shape[2])
        g = rng.standard_normal((2,) + shape)
        Ws.append(s * (g[0] + 1j * g[1]))
    return Ws


def forward(Ws, t_full, tr):
    """Activations of every layer: [psi0, psi1, psi2, psi3]."""
    acts = [np.asarray(t_full, dtype=np.complex128).reshape(-1, 1, 4, 3)]
    for W in Ws:
        acts.append(layer(W, acts[-1], tr))
    return acts


def loss(y_r, z):
    z = np.asarray(z).ravel()
    return float(np.vdot(y_r.ravel() - z, y_r.ravel() - z).real / np.vdot(z, z).real)


def backward(Ws, acts, g_out, tr):
    """Real-pair gradients of the weights, given the gradient of the last
    activation g_out (V, 1, 4, 3).  Returns [g_W1, g_W2, g_W3]."""
    grads = [None] * len(Ws)
    g = np.asarray(g_out, dtype=np.complex128)
    for l in range(len(Ws) - 1, -1, -1):
        W = Ws[l]
        psi = acts[l]
        V, cin = psi.shape[0], psi.shape[1]
        cout = W.shape[1] // 4
        x = psi.reshape(V, 4 * cin, 3)
        gy = g.reshape(V, 4 * cout, 3)
        gW = np.zeros_like(W)
        for d, (nbr, T) in enumerate(tr):
            moved = np.einsum("vab,vkb->vka", T, x[nbr])
            gW[d] = np.einsum("voa,vka->ok", gy, np.conj(moved))
        grads[l] = gW
        if l > 0:
            # g_psi(y) = sum_d U_d(y - d)^H W_d^H g(y - d), scattered back
            gx = np.zeros((V, 4 * cin, 3), dtype=np.complex128)
            for d, (nbr, T) in enumerate(tr):
                back = np.einsum("ok,voa->vka", np.conj(W[d]), gy)       # W_d^H g
                back = np.einsum("vba,vkb->vka", np.conj(T), back)        # U_d^H
                np.add.at(gx, nbr, back)
            g = gx.reshape(V, cin, 4, 3)
    return grads
