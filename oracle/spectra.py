"""Spectra of the Schur complement, its approximation and S~^-1 S (oracle).

Test infrastructure, like the rest of ``oracle/``.

Figures 2-4 of the paper (whose pictures are lost) show, on small lattices,
the spectrum of S_bb for the four permutations, of S_bb against its
Section 3 approximation S~_bb, and of S~_bb^-1 S_bb, which the text reports
clustered around one, best for the Type II and Type II inverse
permutations.  Dense eigenvalues, tiny lattices only.

    python -m oracle.spectra OUT.csv   writes the three spectra of the four
    permutations on a 4^4 plaquette-action field (beta = 5.4, 100 sweeps,
    seed 3), m0 = -0.4, as rows (permutation, quantity, re, im).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import permute, reusken, schur

__all__ = ["spectra", "PERMUTATIONS", "condition_number", "leftmost_eigenvalues"]

PERMUTATIONS = (("P_I", permute.TYPE_I, 0, False), ("P_II", permute.TYPE_II, 0, False),
                ("P_I^T", permute.TYPE_I, 0, True), ("P_II^T", permute.TYPE_II, 0, True))


def spectra(D, perm, n_b):
    """Eigenvalues of S_bb, S~_bb and S~_bb^-1 S_bb (dense)."""
    S = schur.schur_dense(D, perm, n_b)
    St = reusken.reusken_dense(D, perm, n_b)
    return (np.linalg.eigvals(S), np.linalg.eigvals(St), np.linalg.eigvals(np.linalg.solve(St, S)))


def condition_number(D, tol=1e-8, ncv=160):
    """2-norm condition number sigma_max / sigma_min of a sparse square D, the
    quantity of Table 1's second row (read as the 2-norm condition number).
    sigma_max^2 and sigma_min^2 are the largest and smallest eigenvalues of
    the Hermitian D^H D, each found by restarted Lanczos (ARPACK) on D^H D
    alone: no factorisation (a sparse LU of the 8^4 Wilson D holds 3.4e8
    entries).  Returns (kappa, sigma_min, sigma_max)."""
    import scipy.sparse.linalg as sla
    Dr = sp.csr_matrix(D)
    DH = Dr.conj().T.tocsr()
    n = Dr.shape[0]
    normal = sla.LinearOperator((n, n), matvec=lambda v: DH @ (Dr @ v), dtype=np.complex128)
    if n <= ncv + 1:                     # ARPACK needs ncv < n
        ev = np.linalg.eigvalsh(DH.toarray() @ Dr.toarray())
        lmin, lmax = ev[0], ev[-1]
    else:
        lmax = sla.eigsh(normal, k=1, which="LA", tol=tol, return_eigenvectors=False)[0]
        lmin = sla.eigsh(normal, k=1, which="SA", ncv=ncv, tol=tol, maxiter=100000,
                         return_eigenvectors=False)[0]
    smax, smin = float(np.sqrt(lmax)), float(np.sqrt(lmin))
    return smax / smin, smin, smax


def leftmost_eigenvalues(D, k=6, tol=1e-8, ncv=200):
    """The k eigenvalues of a sparse D with the smallest real part (implicitly
    restarted Arnoldi, ARPACK), sorted by real part.  A negative real part
    means the spectrum surrounds the origin, where unpreconditioned BiCGStab
    can stall."""
    import scipy.sparse.linalg as sla
    Dr = sp.csr_matrix(D)
    n = Dr.shape[0]
    if n <= ncv + 1:
        ev = np.linalg.eigvals(Dr.toarray())
    else:
        ev = sla.eigs(Dr, k=k, which="SR", ncv=ncv, tol=tol, maxiter=100000,
                      return_eigenvectors=False)
    ev = ev[np.lexsort((ev.imag, ev.real))]
    return ev[:k]


def _main(path):
    import csv
    import lattice_inputs as li
    from . import dirac
    dims = (4, 4, 4, 4)
    U = li.heatbath_gauge(dims, 5.4, 100, 3)
    D = dirac.wilson_matrix(U, dims, -0.4).tocsr()
    with open(path, "w", newline="") as fh:
        w = csv.writer(fh)
        w.writerow(["permutation", "quantity", "re", "im"])
        for name, t, mu, inv in PERMUTATIONS:
            perm, nb = permute.permutation(dims, t, mu, inv)
            for q, ev in zip(("S", "S~", "S~^-1 S"), spectra(D, perm, nb)):
                for z in ev:
                    w.writerow([name, q, "%.17g" % z.real, "%.17g" % z.imag])


if __name__ == "__main__":
    import sys
    _main(sys.argv[1] if len(sys.argv) > 1 else "spectra_4x4.csv")
