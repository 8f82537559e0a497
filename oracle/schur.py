"""Partition, Schur complement, apply and solve (oracle).

Test infrastructure, like the rest of ``oracle/``.

Section 1 of the paper: after permuting the sites so that the coarse set b
comes first, D is split into the 2x2 block operator

    D = [[D_bb, D_br],
         [D_rb, D_rr]]

and the coarse operator is the Schur complement

    S_bb = D_bb - D_br D_rr^-1 D_rb

(the second identity after the definition of the blocking kernels B, B-bar).
The block UL factorisation that follows it,

    D = [[I, D_br D_rr^-1], [0, I]] . [[S_bb, 0], [D_rb, D_rr]],

turns D x = f into the coarse solve and a back-substitution:

    w_b = f_b - D_br D_rr^-1 f_r,   S_bb x_b = w_b,   x_r = D_rr^-1 (f_r - D_rb x_b).

Vectors on b (and r) are ordered as the labels: entry i of x_b is the spinor
at site perm[i].  The inner inverse D_rr^-1 is either a direct sparse LU
(``inner="direct"``, the plain definition, for small lattices) or the
oracle's BiCGStab to a relative tolerance (``inner="bicgstab"``).

Pins (tests/test_oracle_schur.py): det D = det S_bb det D_rr (Section 1, item
ii) by dense LU on 2^4; the general Gaussian form S = D_bb - D_bb B D~^-1 B-bar
D_bb with D~ = D + B-bar D_bb B and det D~ = det D_bb det D_rr; S_bb^-1 =
(D^-1)_bb; the solve through S_bb plus back-substitution equals a direct
sparse solve of D x = f; four Type II steps equal one Type I step (quotient
property); gamma_5-hermiticity and gauge covariance carried over to S_bb.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from .permute import expand_sites
from . import krylov

__all__ = ["partition", "schur_dense", "SchurOperator", "schur_solve"]


def partition(D, perm, n_b):
    """The four blocks (D_bb, D_br, D_rb, D_rr) of P D P^T as CSR matrices."""
    perm = np.asarray(perm, dtype=np.int64)
    bi = expand_sites(perm[:n_b])
    ri = expand_sites(perm[n_b:])
    Db = D[bi]
    Dr = D[ri]
    return (Db[:, bi].tocsr(), Db[:, ri].tocsr(),
            Dr[:, bi].tocsr(), Dr[:, ri].tocsr())


def schur_dense(D, perm, n_b):
    """Dense S_bb = D_bb - D_br D_rr^-1 D_rb (tiny lattices only)."""
    Dbb, Dbr, Drb, Drr = partition(D, perm, n_b)
    X = np.linalg.solve(Drr.toarray(), Drb.toarray())
    return Dbb.toarray() - Dbr.toarray() @ X


class SchurOperator:
    """y_b = S_bb x_b applied as D_bb x_b - D_br (D_rr^-1 (D_rb x_b))."""

    def __init__(self, D, perm, n_b, inner="direct", inner_tol=1e-12,
                 inner_maxiter=100000):
        self.perm = np.asarray(perm, dtype=np.int64)
        self.n_b = int(n_b)
        self.Dbb, self.Dbr, self.Drb, self.Drr = partition(D, self.perm, self.n_b)
        self.inner = inner
        self.inner_tol = inner_tol
        self.inner_maxiter = inner_maxiter
        self.inner_iters = []
        self._lu = sla.splu(self.Drr.tocsc()) if inner == "direct" else None

    def solve_rr(self, t):
        """z = D_rr^-1 t."""
        if self._lu is not None:
            return self._lu.solve(np.asarray(t, dtype=np.complex128))
        z, info = krylov.bicgstab(lambda v: self.Drr @ v, t, tol=self.inner_tol,
                                  maxiter=self.inner_maxiter)
        self.inner_iters.append(info["iters"])
        return z

    def __call__(self, xb):
        xb = np.asarray(xb, dtype=np.complex128)
        return self.Dbb @ xb - self.Dbr @ self.solve_rr(self.Drb @ xb)


def schur_solve(D, perm, n_b, f, tol=1e-10, m=30, inner="direct",
                inner_tol=1e-12, maxiter=100000):
    """Solve D x = f through S_bb and the block UL back-substitution.

    f and the returned x are full-lattice vectors in the original site order.
    Returns (x, info) with the outer GMRES(m) info plus the inner counts.
    """
    S = SchurOperator(D, perm, n_b, inner=inner, inner_tol=inner_tol)
    f = np.asarray(f, dtype=np.complex128).ravel()
    bi = expand_sites(S.perm[:S.n_b])
    ri = expand_sites(S.perm[S.n_b:])
    fb, fr = f[bi], f[ri]
    wb = fb - S.Dbr @ S.solve_rr(fr)
    xb, info = krylov.gmres(S, wb, m=m, tol=tol, maxiter=maxiter)
    xr = S.solve_rr(fr - S.Drb @ xb)
    x = np.empty_like(f)
    x[bi] = xb
    x[ri] = xr
    info = dict(info)
    info["inner_iters"] = list(S.inner_iters)
    info["w_b"] = wb
    info["x_b"] = xb
    return x, info
