"""The cyclic-reduction V-cycle preconditioner of Section 4 (oracle).

Test infrastructure, like the rest of ``oracle/``.

Section 4 of the paper preconditions BiCGStab with a 3-level V-cycle built
from the Schur-complement approximation of Section 3: level 0 is D on the
lattice; level l + 1 is the approximation S~ of level l's operator on its
coarse set; the coarsest level is inverted exactly; the rest-set inverses
D_rr^-1 of every level are done by an inner solve (BiCGStab to 1e-2 in the
paper).  One application of the preconditioner is the block UL solve of
Section 1 with the exact Schur complement replaced by the next level:

    w_b = f_b - A_br A_rr^-1 f_r,   x_b = V_{l+1}(w_b),
    x_r = A_rr^-1 (f_r - A_rb x_b).

Readings (the paper gives the recipe, not its bookkeeping):
  * the coarse lattice of Type I halves every extent, of Type II(mu) halves
    L_mu; the inverse types have the same counts and so the same coarse
    extents;
  * the coarse operator of level l + 1 is indexed by level l's coarse labels
    in order, and level l + 1 applies its own permutation to those labels as
    a lattice of the coarse extents (the permutation routine acts on the
    coarse matrix as it stands; for Type I and II this label order is the
    coarse lattice's own site order);
  * ``schur="exact"`` uses the exact Schur complement at every level (then a
    V-cycle with exact inner solves is D^-1: the pin), ``schur="reusken"``
    the Section 3 approximation, ``schur="first"`` its first-order truncation
    M = d^-1 (the approximation that ignores D_rr's couplings, which Section
    3 cites as earlier work), a cheap baseline.

The average convergence rate R of Section 4 is ``krylov.convergence_rate``
of the (preconditioned) BiCGStab residual history.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from . import krylov, permute, reusken
from .permute import expand_sites
from .schur import partition

__all__ = ["coarse_dims", "VCycle", "preconditioned_bicgstab"]


def coarse_dims(dims, ptype, mu=0):
    d = list(dims)
    if ptype == permute.TYPE_I:
        return tuple(L // 2 for L in d)
    d[mu] //= 2
    return tuple(d)


def _approx_schur(A, perm, nb, schur):
    """Sparse (reusken) or dense (exact) coarse operator of A."""
    Abb, Abr, Arb, Arr = partition(A, perm, nb)
    if schur == "exact":
        X = np.linalg.solve(Arr.toarray(), Arb.toarray())
        return sp.csr_matrix(Abb.toarray() - Abr.toarray() @ X)
    order = {"reusken": 2, "first": 1}[schur]
    op = reusken.ReuskenOperator.from_blocks(Abb, Abr, Arb, Arr, order=order)
    n = op.n_r
    dinv = sp.bsr_matrix((op.dinv, np.arange(n), np.arange(n + 1)), shape=Arr.shape).tocsr()
    if order == 1:
        return (Abb - Abr @ dinv @ Arb).tocsr()
    dtinv = sp.bsr_matrix((op.dtinv, np.arange(n), np.arange(n + 1)), shape=Arr.shape).tocsr()
    M = dinv + dtinv - dinv @ Arr @ dtinv
    return (Abb - Abr @ M @ Arb).tocsr()


class VCycle:
    """levels: list of (ptype, mu, inv) for levels 0 .. L-2 (the last level is
    solved exactly).  inner: "direct" (sparse LU of A_rr) or a BiCGStab
    tolerance (float) for the rest-set solves, each capped at inner_maxiter
    steps (the last iterate is used if the cap is reached).  inner_log
    collects (level, steps, converged) of every iterative rest-set solve."""

    def __init__(self, D, dims, levels, schur="reusken", inner="direct", inner_maxiter=100000):
        self.inner = inner
        self.inner_maxiter = int(inner_maxiter)
        self.inner_log = []
        self.levels = []
        A = sp.csr_matrix(D)
        d = tuple(dims)
        for (ptype, mu, inv) in levels:
            perm, nb = permute.permutation(d, ptype, mu, inv)
            blocks = partition(A, perm, nb)
            lu = sla.splu(blocks[3].tocsc()) if inner == "direct" else None
            self.levels.append(dict(index=len(self.levels), perm=np.asarray(perm), nb=nb,
                                    blocks=blocks, lu=lu))
            A = _approx_schur(A, perm, nb, schur)
            d = coarse_dims(d, ptype, mu)
        self.coarsest = sla.splu(A.tocsc())
        self.coarse_op = A

    def _solve_rr(self, lev, v):
        if lev["lu"] is not None:
            return lev["lu"].solve(v)
        Arr = lev["blocks"][3]
        z, info = krylov.bicgstab(lambda u: Arr @ u, v, tol=float(self.inner),
                                  maxiter=self.inner_maxiter)
        self.inner_log.append((lev["index"], info["iters"], info["converged"]))
        return z

    def apply(self, f, level=0):
        """x ~ A_level^-1 f by one V-cycle."""
        f = np.asarray(f, dtype=np.complex128)
        if level == len(self.levels):
            return self.coarsest.solve(f)
        lev = self.levels[level]
        _, Abr, Arb, _ = lev["blocks"]
        bi = expand_sites(lev["perm"][:lev["nb"]])
        ri = expand_sites(lev["perm"][lev["nb"]:])
        fb, fr = f[bi], f[ri]
        wb = fb - Abr @ self._solve_rr(lev, fr)
        xb = self.apply(wb, level + 1)
        xr = self._solve_rr(lev, fr - Arb @ xb)
        x = np.empty_like(f)
        x[bi] = xb
        x[ri] = xr
        return x


def preconditioned_bicgstab(D, f, vc, tol=1e-8, maxiter=10000):
    """Right-preconditioned BiCGStab for D x = f with V (one V-cycle) as the
    preconditioner.  x is accumulated from the preconditioned directions that
    were actually applied (V p and V s of each step), so that an inexact V
    (inner solves to a tolerance, hence not one fixed linear map) still gives
    the x whose residual the recurrence tracks.  Returns (x, info) with
    info["R"] the average convergence rate of the residual history."""
    f = np.asarray(f, dtype=np.complex128)
    bnorm = np.linalg.norm(f)
    x = np.zeros_like(f)
    r = f.copy()
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(f)
    p = np.zeros_like(f)
    hist = [np.linalg.norm(r)]
    converged = bnorm == 0.0
    it = 0
    while not converged and it < maxiter:
        it += 1
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = vc.apply(p)
        v = D @ ph
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * bnorm:
            x = x + alpha * ph
            r = s
            hist.append(np.linalg.norm(r))
            converged = True
            break
        sh = vc.apply(s)
        t = D @ sh
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho_old = rho
        hist.append(np.linalg.norm(r))
        converged = hist[-1] <= tol * bnorm
    info = {"iters": it, "history": hist, "converged": bool(converged),
            "R": krylov.convergence_rate(hist)}
    return x, info
