"""Site permutations of the paper (oracle).

Test infrastructure, like the rest of ``oracle/``.

Section 2: ``Permutation_block`` returns a permutation operator P(p) that
exchanges the rows of D, with p chosen so that the coarse-lattice sites are
labelled first (Fig. 1, a 4x4 example whose picture is lost).  Two types are
named -- Type I blocks the lattice in all directions, Type II blocks it "in
all directions, one direction at a time" -- plus the inverse of each, giving
p_I, p_II, p_I^-1, p_II^-1 with operators P_I, P_II, P_I^T, P_II^T.

Readings (the paper is silent or ambiguous on each):

* (P x)_i = x_{p(i)}; the permuted operator is P D P^T, whose (i, j) site
  block is D_{p(i), p(j)}.
* Type I: the coarse set b is every site with all coordinates even
  (N_b = V/16); p lists b in ascending site index, then the rest r in
  ascending site index (a stable partition).
* Type II with direction mu: one renormalisation step halves direction mu
  only; b is every site with x_mu even (N_b = V/2), stable partition.
  Blocking "all directions" is then four such steps, mu = 0, 1, 2, 3, each on
  the coarse lattice of the step before.
* Inverse types: the same Schur construction with p replaced by its inverse
  q = p^-1 (q[p[i]] = i) and the same N_b; the operator is P^T D P and the
  first N_b labels are the sites q(0), ..., q(N_b - 1).

Pins (tests/test_oracle_permute.py): q o p = id, P^T P = I, hand-derived
labels on the 4x4 lattice of Fig. 1's size, N_b counts, the b sets as
coordinate sets, and the quotient (nesting) property tying Type II to Type I
(tests/test_oracle_schur.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["TYPE_I", "TYPE_II", "permutation", "inverse", "perm_matrix",
           "coarse_sites", "expand_sites"]

TYPE_I = 1
TYPE_II = 2


def _coords(dims):
    dims = tuple(int(L) for L in dims)
    s = np.arange(int(np.prod(dims)))
    out = []
    stride = 1
    for L in dims:
        out.append((s // stride) % L)
        stride *= L
    return np.stack(out, axis=1)


def inverse(p):
    """q = p^-1, i.e. q[p[i]] = i."""
    p = np.asarray(p, dtype=np.int64)
    q = np.empty_like(p)
    q[p] = np.arange(p.size, dtype=np.int64)
    return q


def permutation(dims, ptype, mu=0, inv=False):
    """Return (perm, N_b): the label order of the sites and the coarse count.

    perm[i] is the original site placed at position i, so the coarse set is
    perm[:N_b] and the rest perm[N_b:].  ``dims`` may have any number of
    axes (the paper's Fig. 1 is two-dimensional; the operator is 4-D).
    """
    dims = tuple(int(L) for L in dims)
    x = _coords(dims)
    if ptype == TYPE_I:
        if any(L % 2 for L in dims):
            raise ValueError("Type I blocking needs even extents")
        is_b = np.all(x % 2 == 0, axis=1)
    elif ptype == TYPE_II:
        if not 0 <= mu < len(dims) or dims[mu] % 2:
            raise ValueError("Type II blocking needs an even extent along mu")
        is_b = x[:, mu] % 2 == 0
    else:
        raise ValueError("unknown permutation type")
    sites = np.arange(x.shape[0], dtype=np.int64)
    p = np.concatenate([sites[is_b], sites[~is_b]])
    n_b = int(is_b.sum())
    return (inverse(p) if inv else p), n_b


def perm_matrix(perm, ncomp=1):
    """Sparse P with (P x)_i = x_{perm[i]}, acting on ncomp components per site."""
    perm = np.asarray(perm, dtype=np.int64)
    n = perm.size * ncomp
    rows = np.arange(n)
    cols = (ncomp * perm[:, None] + np.arange(ncomp)[None, :]).ravel()
    return sp.csr_matrix((np.ones(n), (rows, cols)), shape=(n, n))


def coarse_sites(perm, n_b):
    """The coarse set b (in label order) and the rest r (in label order)."""
    perm = np.asarray(perm, dtype=np.int64)
    return perm[:n_b], perm[n_b:]


def expand_sites(sites, ncomp=12):
    """Vector indices of a list of sites (ncomp components per site)."""
    sites = np.asarray(sites, dtype=np.int64)
    return (ncomp * sites[:, None] + np.arange(ncomp)[None, :]).ravel()
