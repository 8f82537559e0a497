"""Wilson-Dirac operator, assembled as a sparse matrix (oracle).

Test infrastructure, like the rest of ``oracle/``.

The paper blocks "the Wilson-Dirac operator" (Section 2, around Fig. 2), calls
its off-diagonal part the "hopping matrix" and quotes the hopping parameter
kappa (Section 3 and Section 4), but never writes the operator out.  The
reading used here is the textbook Wilson operator with Wilson parameter r = 1:

    (D psi)(x) = (m0 + 4 r) psi(x)
                 - 1/2 sum_mu [ (r - gamma_mu) U_mu(x)          psi(x + mu)
                              + (r + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]

with kappa = 1 / (2 m0 + 8 r), periodic boundaries in all four directions.

Gamma matrices: the DeGrand-Rossi chiral basis, gamma_5 = g1 g2 g3 g4 =
diag(1, 1, -1, -1); direction mu = 0..3 (lattice axis x0..x3) carries
gamma_{mu+1}.

Vector layout: index 12*s + 3*spin + colour, site s = x0 + L0*(x1 + L1*(x2 +
L2*x3)).  Every 12x12 site block is kron(spin matrix, colour matrix).

Pins (tests/test_oracle_dirac.py): Clifford algebra and hermiticity of the
gammas; plane-wave closed form D(p) = m0 + r sum(1 - cos p) + i sum gamma sin p
at U = 1; free-field spectrum; gamma_5-hermiticity; gauge covariance under
random SU(3) gauge transformations; the 2^4 lattice (both hops to one
neighbour add).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["GAMMA", "GAMMA5", "neighbour", "wilson_matrix", "kappa_to_m0"]

_i = 1j
# DeGrand-Rossi basis.  GAMMA[mu] acts along lattice axis x_mu.
GAMMA = np.array([
    [[0, 0, 0, _i], [0, 0, _i, 0], [0, -_i, 0, 0], [-_i, 0, 0, 0]],   # gamma_1
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],       # gamma_2
    [[0, 0, _i, 0], [0, 0, 0, -_i], [-_i, 0, 0, 0], [0, _i, 0, 0]],   # gamma_3
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],         # gamma_4
], dtype=np.complex128)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def kappa_to_m0(kappa: float, r: float = 1.0) -> float:
    """m0 from the hopping parameter: kappa = 1 / (2 m0 + 8 r)."""
    return 1.0 / (2.0 * kappa) - 4.0 * r


def coords(dims):
    """(V, 4) int array of site coordinates in site order (x0 fastest)."""
    L0, L1, L2, L3 = dims
    s = np.arange(L0 * L1 * L2 * L3)
    x0 = s % L0
    x1 = (s // L0) % L1
    x2 = (s // (L0 * L1)) % L2
    x3 = s // (L0 * L1 * L2)
    return np.stack([x0, x1, x2, x3], axis=1)


def site_index(x, dims):
    L0, L1, L2, L3 = dims
    return x[..., 0] + L0 * (x[..., 1] + L1 * (x[..., 2] + L2 * x[..., 3]))


def neighbour(dims, mu, step):
    """Site index of x + step*mu-hat for every site x (periodic)."""
    x = coords(dims).copy()
    x[:, mu] = (x[:, mu] + step) % dims[mu]
    return site_index(x, dims)


def wilson_matrix(U, dims, m0, r=1.0, rows_of=None):
    """Assembled (12V x 12V) CSR matrix of the Wilson-Dirac operator above.

    U: complex128 (V, 4, 3, 3), U[s, mu] the link from s to s + mu-hat.
    Duplicate (row-block, column-block) entries -- the forward and backward
    hop reach the same site when L_mu = 2 -- are summed.
    rows_of: optional list of sites; then only their block rows are built
    and the result is (12 len(rows_of) x 12V), row block i = site rows_of[i]
    (to check large lattices on sampled sites).
    """
    dims = tuple(int(L) for L in dims)
    V = int(np.prod(dims))
    U = np.asarray(U, dtype=np.complex128).reshape(V, 4, 3, 3)
    I4 = np.eye(4)
    rows, cols, vals = [], [], []
    all_sites = np.arange(V)
    site = all_sites if rows_of is None else np.asarray(rows_of, dtype=np.int64)
    nrow = site.size
    out_row = np.arange(nrow)

    def add_blocks(row_sites, col_sites, blocks):
        # blocks: (nrow, 12, 12); row_sites index the output block rows
        rr = 12 * row_sites[:, None, None] + np.arange(12)[None, :, None]
        cc = 12 * col_sites[:, None, None] + np.arange(12)[None, None, :]
        rr, cc = np.broadcast_arrays(rr, cc)
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(blocks.ravel())

    diag = np.broadcast_to((m0 + 4.0 * r) * np.eye(12), (nrow, 12, 12))
    add_blocks(out_row, site, diag)
    for mu in range(4):
        fwd = neighbour(dims, mu, +1)[site]
        bwd = neighbour(dims, mu, -1)[site]
        Pm = -0.5 * (r * I4 - GAMMA[mu])    # multiplies U_mu(x) psi(x+mu)
        Pp = -0.5 * (r * I4 + GAMMA[mu])    # multiplies U_mu(x-mu)^dag psi(x-mu)
        Uf = U[site, mu]                                # U_mu(x)
        Ub = np.conj(np.swapaxes(U[bwd, mu], -1, -2))   # U_mu(x-mu)^dagger
        Bf = np.einsum("ab,sij->saibj", Pm, Uf).reshape(nrow, 12, 12)
        Bb = np.einsum("ab,sij->saibj", Pp, Ub).reshape(nrow, 12, 12)
        add_blocks(out_row, fwd, Bf)
        add_blocks(out_row, bwd, Bb)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    D = sp.coo_matrix((vals, (rows, cols)), shape=(12 * nrow, 12 * V)).tocsr()
    D.sum_duplicates()
    return D
