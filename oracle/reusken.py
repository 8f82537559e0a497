"""The second-order Schur-complement approximation of Section 3 (oracle).

Test infrastructure, like the rest of ``oracle/``.

Section 3 of the paper keeps one power of D_rr and replaces its inverse by
Reusken's second-order expression:

    S~_bb = D_bb - D_br M D_rb,   M = d^-1 + d~^-1 - d^-1 D_rr d~^-1,

with d the diagonal of D_rr and d~ the diagonal matrix of the sums of the
rows of D_rr.  Reading (the paper is silent on the block structure): both
are site-block diagonal, 12 x 12 per rest site (spin x colour),

    d_x  = (D_rr)_{x,x},           d~_x = sum_{y in r} (D_rr)_{x,y},

so that for the Wilson operator d = (m0 + 4) 1 and d~_x is m0 + 4 minus the
hopping blocks of the rest-set neighbours of x.  The point-wise reading (a
scalar row sum over complex entries) mixes spin and colour components and
is not used.

Section 3 also names the earlier, cruder approximation that ignores D_rr
(cited there as the choice that keeps the coarse operator's sparsity).
Reading: D_rr is replaced by its diagonal d, i.e. M = d^-1, the first-order
truncation of the same expansion (``order=1``); dropping the whole
D_br D_rr^-1 D_rb term instead would leave S = D_bb = (m0 + 4) 1 for Type I,
no coarse operator at all.

Pins (tests/test_oracle_reusken.py), from the algebra of M:
  * for every block-constant vector 1_c (the same 12-vector c on every rest
    site) D_rr 1_c = d~ 1_c, hence M D_rr 1_c = 1_c exactly;
  * if D_rr is site-block diagonal, d = d~ = D_rr and M = D_rr^-1, S~ = S;
  * with the hopping scaled by t, D_rr^-1 - M = O(t^2), so the error of the
    correction term, ||S - S~|| / ||S - D_bb||, falls like t^2;
  * for order=1, D_rr^-1 - d^-1 = O(t), so the same ratio falls like t.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .schur import partition

__all__ = ["site_blocks", "block_row_sums", "ReuskenOperator", "reusken_dense"]

ORDERS = (1, 2)


def site_blocks(Drr):
    """The 12 x 12 diagonal blocks of D_rr: array (n_r, 12, 12)."""
    n = Drr.shape[0] // 12
    A = Drr.tocsr()
    out = np.empty((n, 12, 12), dtype=np.complex128)
    for x in range(n):
        out[x] = A[12 * x:12 * x + 12, 12 * x:12 * x + 12].toarray()
    return out


def block_row_sums(Drr):
    """d~_x = sum_y (D_rr)_{x,y}: D_rr applied to the block-constant identity
    columns, array (n_r, 12, 12)."""
    n = Drr.shape[0] // 12
    E = sp.kron(np.ones((n, 1)), sp.identity(12), format="csr")
    S = Drr @ E
    S = S.toarray() if sp.issparse(S) else np.asarray(S)
    return S.reshape(n, 12, 12)


class ReuskenOperator:
    """y_b = S~_bb x_b with M = d^-1 + d~^-1 - d^-1 D_rr d~^-1 (order 2, the
    Section 3 formula) or M = d^-1 (order 1, D_rr's couplings ignored);
    blocks inverted site by site."""

    def __init__(self, D, perm, n_b, order=2):
        self._setup(*partition(D, perm, n_b), order=order)

    @classmethod
    def from_blocks(cls, Dbb, Dbr, Drb, Drr, order=2):
        op = cls.__new__(cls)
        op._setup(Dbb, Dbr, Drb, sp.csr_matrix(Drr), order=order)
        return op

    def _setup(self, Dbb, Dbr, Drb, Drr, order=2):
        if order not in ORDERS:
            raise ValueError("order must be 1 or 2")
        self.order = order
        self.Dbb, self.Dbr, self.Drb, self.Drr = Dbb, Dbr, Drb, Drr
        self.n_r = self.Drr.shape[0] // 12
        self.dinv = np.linalg.inv(site_blocks(self.Drr))
        self.dtinv = np.linalg.inv(block_row_sums(self.Drr)) if order == 2 else None

    def _blocks(self, Binv, v):
        return np.einsum("xab,xb->xa", Binv, np.asarray(v).reshape(self.n_r, 12)).ravel()

    def M(self, v):
        """The approximate inverse of D_rr applied to a rest vector."""
        if self.order == 1:
            return self._blocks(self.dinv, v)
        w = self._blocks(self.dtinv, v)
        return self._blocks(self.dinv, v) + w - self._blocks(self.dinv, self.Drr @ w)

    def __call__(self, xb):
        xb = np.asarray(xb, dtype=np.complex128)
        return self.Dbb @ xb - self.Dbr @ self.M(self.Drb @ xb)


def reusken_dense(D, perm, n_b, order=2):
    """Dense S~_bb (tiny lattices only), column by column."""
    op = ReuskenOperator(D, perm, n_b, order)
    nb12 = op.Dbb.shape[0]
    out = np.empty((nb12, nb12), dtype=np.complex128)
    e = np.zeros(nb12, dtype=np.complex128)
    for j in range(nb12):
        e[j] = 1.0
        out[:, j] = op(e)
        e[j] = 0.0
    return out
