"""The exp(i eps H) and APE-smeared gauge fields of this package, computed with
torch tensor operations so that large lattices (32^3 x 64: 8.4 M links) can be
made on whatever device the caller names.

Same recipes and the same seeded draws as ``random_gauge`` and ``ape_smear``;
only the way two matrix functions are evaluated differs, both exact up to
rounding:

* exp(i eps H) by scaling and squaring of a Taylor series (``random_gauge``
  goes through ``eigh``);
* the unitary polar factor by the scaled Newton iteration
  W <- (g W + W^-H / g) / 2, g = |det W|^(-1/3) (Higham, Functions of
  Matrices, Section 8.6), with W^-H from the 3x3 cofactor matrix
  (``ape_smear`` goes through the SVD).

The two routes agree to ~1e-13 (tests/test_inputs.py).  Like the rest of the
package this holds none of the method's arithmetic.
"""
from __future__ import annotations

import numpy as np

__all__ = ["random_gauge_t", "ape_smear_t", "workload_gauge_t"]


def _dag(M):
    return M.conj().transpose(-1, -2)


def _expi_taylor(X):
    """exp(i X) for Hermitian X (..., 3, 3): exp(i X / 2^s) by its Taylor
    series to order 12, squared s times, with ||X / 2^s||_F <= 1/8."""
    import torch
    nrm = torch.linalg.matrix_norm(X).max().item()
    s = max(0, int(np.ceil(np.log2(max(nrm, 1e-300) * 8.0))))
    A = (1j / 2.0 ** s) * X
    eye = torch.eye(3, dtype=X.dtype, device=X.device).expand_as(X)
    E = eye.clone()
    term = eye.clone()
    for k in range(1, 13):
        term = term @ A / k
        E = E + term
    for _ in range(s):
        E = E @ E
    return E


def random_gauge_t(dims, eps, seed, device="cpu"):
    """``random_gauge(dims, eps, seed)`` as a complex128 torch tensor (V, 4, 3, 3)."""
    import torch
    L0, L1, L2, L3 = dims
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((2, L3, L2, L1, L0, 4, 3, 3))
    A = torch.complex(torch.from_numpy(g[0]), torch.from_numpy(g[1])).to(device)
    del g
    H = 0.5 * (A + _dag(A))
    del A
    tr = H.diagonal(dim1=-2, dim2=-1).sum(-1)
    H = H - (tr / 3.0)[..., None, None] * torch.eye(3, dtype=H.dtype, device=H.device)
    U = _expi_taylor(eps * H)
    return U.reshape(L0 * L1 * L2 * L3, 4, 3, 3).contiguous()


def _cofactor(W):
    """Cofactor matrix of (..., 3, 3): inv(W) = cof(W)^T / det(W)."""
    import torch
    rows = []
    for i in range(3):
        i1, i2 = (i + 1) % 3, (i + 2) % 3
        cols = []
        for j in range(3):
            j1, j2 = (j + 1) % 3, (j + 2) % 3
            cols.append(W[..., i1, j1] * W[..., i2, j2] - W[..., i1, j2] * W[..., i2, j1])
        rows.append(torch.stack(cols, -1))
    return torch.stack(rows, -2)


def _project_su3_t(M, iters=12):
    """Unitary polar factor of M by scaled Newton, then the phase of det removed."""
    import torch
    W = M
    for _ in range(iters):
        cof = _cofactor(W)
        det = (W[..., 0, :] * cof[..., 0, :]).sum(-1)
        winvh = cof.conj() / det.conj()[..., None, None]          # W^-H
        gam = det.abs().pow(-1.0 / 3.0)[..., None, None]
        W = 0.5 * (gam * W + winvh / gam)
    cof = _cofactor(W)
    det = (W[..., 0, :] * cof[..., 0, :]).sum(-1)
    return W * torch.exp(-1j * torch.angle(det) / 3.0)[..., None, None]


def ape_smear_t(U, dims, alpha, steps):
    """``ape_smear`` on a torch tensor (V, 4, 3, 3), on U's device."""
    import torch
    L0, L1, L2, L3 = dims
    G = U.reshape(L3, L2, L1, L0, 4, 3, 3)

    def sh(F, mu, step):
        return torch.roll(F, -step, dims=3 - mu)

    for _ in range(int(steps)):
        new = torch.empty_like(G)
        for mu in range(4):
            Um = G[..., mu, :, :]
            C = torch.zeros_like(Um)
            for nu in range(4):
                if nu == mu:
                    continue
                Un = G[..., nu, :, :]
                C += Un @ sh(Um, nu, 1) @ _dag(sh(Un, mu, 1))
                Un_m = sh(Un, nu, -1)
                C += _dag(Un_m) @ sh(Um, nu, -1) @ sh(Un_m, mu, 1)
            new[..., mu, :, :] = _project_su3_t((1.0 - alpha) * Um + (alpha / 6.0) * C)
            del C
        G = new
    return G.reshape(L0 * L1 * L2 * L3, 4, 3, 3).contiguous()


def workload_gauge_t(name, device="cpu"):
    """The exp(i eps H) (+ APE) workloads of ``workload_gauge`` made with torch."""
    table = {
        "16^3x32 eps0.25 ape5": ((16, 16, 16, 32), 0.25, 2, 5),
        "24^3x48 eps0.2": ((24, 24, 24, 48), 0.2, 3, 0),
        "16^4 eps0.2": ((16, 16, 16, 16), 0.2, 4, 0),
        "8^4 eps0.2": ((8, 8, 8, 8), 0.2, 6, 0),
        "32^3x64 eps0.2 ape10": ((32, 32, 32, 64), 0.2, 5, 10),
    }
    dims, eps, seed, steps = table[name]
    U = random_gauge_t(dims, eps, seed, device)
    if steps:
        U = ape_smear_t(U, dims, 0.5, steps)
    return dims, U
