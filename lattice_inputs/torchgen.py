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

Matrices are held entry-major ([3][3][...]: entry (i, j) of every link is one
contiguous vector), so a 3x3 product is three broadcast multiply-adds of
vectors rather than millions of tiny batched GEMMs.  The two routes agree to
~1e-13 (tests/test_inputs.py).  Like the rest of the package this holds none
of the method's arithmetic.
"""
from __future__ import annotations

import numpy as np

__all__ = ["random_gauge_t", "ape_smear_t", "workload_gauge_t"]


# entry-major 3x3 helpers: M[i, j] is a tensor over the links
def _mm(A, B):
    return A[:, 0, None] * B[None, 0] + A[:, 1, None] * B[None, 1] + A[:, 2, None] * B[None, 2]


def _dag(M):
    return M.transpose(0, 1).conj()


def _eye_like(M):
    import torch
    E = torch.zeros_like(M)
    for i in range(3):
        E[i, i] = 1.0
    return E


def _to_entry(M):
    """(..., 3, 3) -> (3, 3, ...)"""
    nd = M.dim()
    return M.permute(nd - 2, nd - 1, *range(nd - 2)).contiguous()


def _from_entry(E):
    """(3, 3, ...) -> (..., 3, 3)"""
    nd = E.dim()
    return E.permute(*range(2, nd), 0, 1).contiguous()


def _expi_taylor(X):
    """exp(i X) for Hermitian X (3, 3, ...): exp(i X / 2^s) by its Taylor
    series to order 12, squared s times, with ||X / 2^s||_F <= 1/8."""
    import torch
    nrm = torch.sqrt((X.abs() ** 2).sum(dim=(0, 1))).max().item()
    s = max(0, int(np.ceil(np.log2(max(nrm, 1e-300) * 8.0))))
    A = (1j / 2.0 ** s) * X
    E = _eye_like(X)
    term = E.clone()
    for k in range(1, 13):
        term = _mm(term, A) / k
        E = E + term
    for _ in range(s):
        E = _mm(E, E)
    return E


def random_gauge_t(dims, eps, seed, device="cpu"):
    """``random_gauge(dims, eps, seed)`` as a complex128 torch tensor (V, 4, 3, 3)."""
    import torch
    L0, L1, L2, L3 = dims
    V = L0 * L1 * L2 * L3
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((2, V * 4, 3, 3))
    A = _to_entry(torch.complex(torch.from_numpy(g[0]), torch.from_numpy(g[1])).to(device))
    del g
    H = 0.5 * (A + _dag(A))
    del A
    tr = H[0, 0] + H[1, 1] + H[2, 2]
    for i in range(3):
        H[i, i] = H[i, i] - tr / 3.0
    U = _expi_taylor(eps * H)
    return _from_entry(U).reshape(V, 4, 3, 3)


def _project_su3_e(M, iters=12):
    """Unitary polar factor of the entry-major M by scaled Newton, then the
    phase of det removed."""
    import torch

    def cof_det(W):
        cof = torch.empty_like(W)
        for i in range(3):
            i1, i2 = (i + 1) % 3, (i + 2) % 3
            for j in range(3):
                j1, j2 = (j + 1) % 3, (j + 2) % 3
                cof[i, j] = W[i1, j1] * W[i2, j2] - W[i1, j2] * W[i2, j1]
        det = W[0, 0] * cof[0, 0] + W[0, 1] * cof[0, 1] + W[0, 2] * cof[0, 2]
        return cof, det

    W = M
    for _ in range(iters):
        cof, det = cof_det(W)
        winvh = cof.conj() / det.conj()                       # W^-H
        gam = det.abs().pow(-1.0 / 3.0)
        W = 0.5 * (gam * W + winvh / gam)
    _, det = cof_det(W)
    return W * torch.exp(-1j * torch.angle(det) / 3.0)


def ape_smear_t(U, dims, alpha, steps):
    """``ape_smear`` on a torch tensor (V, 4, 3, 3), on U's device."""
    import torch
    L0, L1, L2, L3 = dims
    V = L0 * L1 * L2 * L3
    # G[mu] entry-major over the lattice grid: (4, 3, 3, L3, L2, L1, L0)
    G = _to_entry(U.reshape(L3, L2, L1, L0, 4, 3, 3)).permute(6, 0, 1, 2, 3, 4, 5).contiguous()

    def sh(F, mu, step):   # F(x + step mu-hat) on (3, 3, L3, L2, L1, L0)
        return torch.roll(F, -step, dims=5 - mu)

    for _ in range(int(steps)):
        new = torch.empty_like(G)
        for mu in range(4):
            Um = G[mu]
            C = torch.zeros_like(Um)
            for nu in range(4):
                if nu == mu:
                    continue
                Un = G[nu]
                C += _mm(_mm(Un, sh(Um, nu, 1)), _dag(sh(Un, mu, 1)))
                Un_m = sh(Un, nu, -1)
                C += _mm(_mm(_dag(Un_m), sh(Um, nu, -1)), sh(Un_m, mu, 1))
            new[mu] = _project_su3_e((1.0 - alpha) * Um + (alpha / 6.0) * C)
            del C
        G = new
    # back to (V, 4, 3, 3) with the site index x0 fastest
    return G.permute(3, 4, 5, 6, 0, 1, 2).reshape(V, 4, 3, 3).contiguous()


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
