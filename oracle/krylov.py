"""Textbook Krylov solvers (oracle).

Test infrastructure, like the rest of ``oracle/``.

The paper's solver is "vanilla BiCGstab" (Section 4); the 8^4 workload asks
for restarted GMRES(30) on S_bb.  Both are written out below exactly as in
their original papers, in complex arithmetic, with the convergence test on
the recursively updated residual measured relative to ||b||:

* ``bicgstab`` -- H. A. van der Vorst, SIAM J. Sci. Stat. Comput. 13 (1992)
  631, Algorithm "Bi-CGSTAB" (unpreconditioned), shadow residual r0^ = r0.
* ``gmres``    -- Y. Saad and M. H. Schultz, SIAM J. Sci. Stat. Comput. 7
  (1986) 856, restarted GMRES(m) with modified Gram-Schmidt and Givens
  rotations for the small least-squares problem.

Both take a callable ``A(x) -> y`` so they serve D, D_rr and S_bb alike.  The
residual history is returned so the average convergence rate of Section 4
(R = average ratio of next to current residual) can be formed from it.

Pins (tests/test_oracle_krylov.py): each solver reaches the solution of a
direct sparse solve (scipy ``spsolve``) within its tolerance on a small
non-Hermitian system, and the final true residual meets the tolerance.
"""
from __future__ import annotations

import numpy as np

__all__ = ["bicgstab", "gmres", "convergence_rate", "mean_ratio"]


def _norm(v):
    return float(np.sqrt(np.vdot(v, v).real))


def bicgstab(A, b, tol=1e-12, maxiter=10000, x0=None):
    """Solve A x = b.  Returns (x, info) with info = dict(iters, history, converged)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - A(x) if x0 is not None else b.copy()
    bnorm = _norm(b)
    hist = [_norm(r)]
    if bnorm == 0.0:
        return np.zeros_like(b), dict(iters=0, history=hist, converged=True)
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    converged = hist[-1] <= tol * bnorm
    while not converged and it < maxiter:
        it += 1
        rho = np.vdot(rhat, r)
        if rho == 0:
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        if _norm(s) <= tol * bnorm:
            x = x + alpha * p
            r = s
            hist.append(_norm(r))
            converged = True
            break
        t = A(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        hist.append(_norm(r))
        converged = hist[-1] <= tol * bnorm
    return x, dict(iters=it, history=hist, converged=bool(converged))


def gmres(A, b, m=30, tol=1e-10, maxiter=100000, x0=None):
    """Restarted GMRES(m).  Returns (x, info); ``maxiter`` counts Arnoldi steps.

    Each cycle builds an orthonormal Krylov basis V with modified
    Gram-Schmidt, reduces the Hessenberg matrix H to upper-triangular form by
    complex Givens rotations G = [[conj(c), conj(s)], [-s, c]] (c = a/h,
    s = b/h, h = sqrt(|a|^2 + |b|^2)), and solves the triangular system for the
    update when the residual estimate |g_{j+1}| meets the tolerance, the basis
    is full, or the Krylov space is invariant.  The true residual b - A x is
    recomputed at every restart.
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), dict(iters=0, history=[0.0], converged=True)
    hist = []
    total = 0
    converged = False
    while True:
        r = b - A(x)
        beta = _norm(r)
        hist.append(beta)
        if beta <= tol * bnorm:
            converged = True
            break
        if total >= maxiter:
            break
        Vb = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        c = np.zeros(m, dtype=np.complex128)
        s = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Vb[0] = r / beta
        k = 0
        for j in range(m):
            w = A(Vb[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(Vb[i], w)
                w = w - H[i, j] * Vb[i]
            hnext = _norm(w)
            H[j + 1, j] = hnext
            if hnext != 0.0:
                Vb[j + 1] = w / hnext
            for i in range(j):                           # rotations so far
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = np.conj(c[i]) * hi + np.conj(s[i]) * hi1
                H[i + 1, j] = -s[i] * hi + c[i] * hi1
            a, bb = H[j, j], H[j + 1, j]                 # new rotation
            h = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            c[j], s[j] = (a / h, bb / h) if h != 0.0 else (1.0, 0.0)
            H[j, j] = h
            H[j + 1, j] = 0.0
            g[j + 1] = -s[j] * g[j]
            g[j] = np.conj(c[j]) * g[j]
            total += 1
            k = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * bnorm or hnext == 0.0 or total >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + Vb[:k].T @ y
    return x, dict(iters=total, history=hist, converged=converged)


def convergence_rate(history):
    """Average ratio of next to current residual (Section 4's R), as the
    geometric mean (||r_n|| / ||r_0||)^(1/n) over the recorded history."""
    h = np.asarray(history, dtype=float)
    h = h[h > 0]
    if h.size < 2:
        return 0.0
    return float((h[-1] / h[0]) ** (1.0 / (h.size - 1)))


def mean_ratio(history):
    """The other reading of Section 4's R: the arithmetic mean of the ratios
    ||r_{k+1}|| / ||r_k|| over the recorded history (never below the
    geometric mean, equal to it for a geometric sequence)."""
    h = np.asarray(history, dtype=float)
    h = h[h > 0]
    if h.size < 2:
        return 0.0
    return float(np.mean(h[1:] / h[:-1]))
