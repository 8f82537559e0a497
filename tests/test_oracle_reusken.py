"""Pins of the second-order Schur-complement approximation (Section 3)
from the algebra of M = d^-1 + d~^-1 - d^-1 D_rr d~^-1."""
import numpy as np
import pytest
import scipy.sparse as sp

import lattice_inputs as li
from oracle import dirac, permute, reusken, schur

TYPES = [(permute.TYPE_I, 0, False), (permute.TYPE_II, 0, False), (permute.TYPE_I, 0, True),
         (permute.TYPE_II, 1, True)]


@pytest.mark.parametrize("t,mu,inv", TYPES)
def test_exact_on_images_of_block_constant_vectors(t, mu, inv):
    """D_rr 1_c = d~ 1_c by the definition of the row sums, so
    M D_rr 1_c = d^-1 d~ 1_c + 1_c - d^-1 D_rr 1_c = 1_c exactly."""
    dims = (4, 4, 4, 4)
    U = li.random_gauge(dims, 0.5, 3)
    D = dirac.wilson_matrix(U, dims, 0.1)
    perm, nb = permute.permutation(dims, t, mu, inv)
    op = reusken.ReuskenOperator(D, perm, nb)
    rng = np.random.default_rng(1)
    c = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    one_c = np.tile(c, op.n_r)
    back = op.M(op.Drr @ one_c)
    assert np.abs(back - one_c).max() <= 1e-12 * np.abs(one_c).max()
    # and not for a generic vector (the approximation is not the inverse)
    v = rng.standard_normal(one_c.size) + 1j * rng.standard_normal(one_c.size)
    assert np.linalg.norm(op.M(op.Drr @ v) - v) > 1e-3 * np.linalg.norm(v)


def test_block_diagonal_D_rr_gives_the_exact_Schur_complement():
    """With the rest-rest hopping removed, d = d~ = D_rr and M = D_rr^-1."""
    dims = (4, 4, 4, 4)
    U = li.random_gauge(dims, 0.5, 4)
    D = dirac.wilson_matrix(U, dims, -0.2)
    perm, nb = permute.permutation(dims, permute.TYPE_II, 2, False)
    Dbb, Dbr, Drb, Drr = schur.partition(D, perm, nb)
    blocks = reusken.site_blocks(Drr)
    n = blocks.shape[0]
    Drr_bd = sp.bsr_matrix((blocks, np.arange(n), np.arange(n + 1)), shape=Drr.shape).tocsr()
    op = reusken.ReuskenOperator.from_blocks(Dbb, Dbr, Drb, Drr_bd)
    rng = np.random.default_rng(2)
    xb = rng.standard_normal(Dbb.shape[0]) + 1j * rng.standard_normal(Dbb.shape[0])
    exact = Dbb @ xb - Dbr @ np.linalg.solve(Drr_bd.toarray(), Drb @ xb)
    assert np.abs(op(xb) - exact).max() <= 1e-12 * np.abs(exact).max()


def test_error_of_the_correction_is_second_order_in_the_hopping():
    """D_t = (m0 + 4) + t H: D_rr^-1 - M = d^-1 E d^-1 (E - e) d^-1 + O(t^3), so
    ||S - S~|| / ||S - D_bb|| falls like t^2 (halving t divides it by ~4)."""
    dims = (4, 4, 4, 4)
    U = li.random_gauge(dims, 0.4, 5)
    m0 = 0.3
    D1 = dirac.wilson_matrix(U, dims, m0).tocsr()
    diag = (m0 + 4.0) * sp.identity(D1.shape[0], format="csr")
    H = D1 - diag
    perm, nb = permute.permutation(dims, permute.TYPE_I)
    errs = []
    for tt in (0.4, 0.2, 0.1):
        D = (diag + tt * H).tocsr()
        S = schur.schur_dense(D, perm, nb)
        St = reusken.reusken_dense(D, perm, nb)
        Dbb = schur.partition(D, perm, nb)[0].toarray()
        errs.append(np.linalg.norm(S - St) / np.linalg.norm(S - Dbb))
    r1, r2 = errs[1] / errs[0], errs[2] / errs[1]
    assert 0.18 < r1 < 0.32 and 0.2 < r2 < 0.3, errs


def test_free_field_type_I_row_sums_closed_form():
    """U = 1, Type I: every rest neighbour of a rest site is in r except the
    coarse ones; d~_x = (m0 + 4) - 1/2 sum over rest neighbours of (1 -+ gamma)
    x 1_colour, so d~_x - d_x is - 1/2 sum of those projectors; checked on a
    site whose eight neighbours are all rest sites (x = (1, 1, 1, 1))."""
    dims = (4, 4, 4, 4)
    U = np.broadcast_to(np.eye(3), (256, 4, 3, 3)).astype(np.complex128).copy()
    m0 = 0.2
    D = dirac.wilson_matrix(U, dims, m0)
    perm, nb = permute.permutation(dims, permute.TYPE_I)
    _, _, _, Drr = schur.partition(D, perm, nb)
    dt = reusken.block_row_sums(Drr)
    site = 1 + 4 + 16 + 64
    k = int(np.where(perm[nb:] == site)[0][0])
    expect = (m0 + 4.0) * np.eye(12)
    for mu in range(4):
        g = dirac.GAMMA[mu]
        expect = expect - 0.5 * np.kron((np.eye(4) - g) + (np.eye(4) + g), np.eye(3))
    assert np.abs(dt[k] - expect).max() <= 1e-13


def test_first_order_truncation_error_is_first_order_in_the_hopping():
    """order=1 (M = d^-1, D_rr's couplings ignored): D_rr^-1 - d^-1 = O(t), so
    ||S - S_1|| / ||S - D_bb|| halves with t, while the Section 3 formula's
    ratio falls by four and stays below it (P_II^T, direction 1, whose D_bb
    and D_rr both have hops)."""
    dims = (4, 4, 4, 4)
    U = li.random_gauge(dims, 0.4, 5)
    m0 = 0.3
    D1 = dirac.wilson_matrix(U, dims, m0).tocsr()
    diag = (m0 + 4.0) * sp.identity(D1.shape[0], format="csr")
    H = D1 - diag
    perm, nb = permute.permutation(dims, permute.TYPE_II, 1, True)
    e1, e2 = [], []
    for tt in (0.4, 0.2, 0.1):
        D = (diag + tt * H).tocsr()
        S = schur.schur_dense(D, perm, nb)
        Dbb = schur.partition(D, perm, nb)[0].toarray()
        den = np.linalg.norm(S - Dbb)
        e1.append(np.linalg.norm(S - reusken.reusken_dense(D, perm, nb, order=1)) / den)
        e2.append(np.linalg.norm(S - reusken.reusken_dense(D, perm, nb, order=2)) / den)
    for a, b in zip(e1, e1[1:]):
        assert 0.4 < b / a < 0.6, e1
    for a, b in zip(e2, e2[1:]):
        assert 0.15 < b / a < 0.35, e2
    assert all(x2 < x1 for x1, x2 in zip(e1, e2))


def test_first_order_is_d_inverse_for_wilson():
    """For the Wilson D the site-block diagonal of D_rr is (m0 + 4) 1, so the
    first-order operator is D_bb - D_br D_rb / (m0 + 4) exactly."""
    dims = (4, 4, 2, 4)
    U = li.random_gauge(dims, 0.3, 6)
    m0 = -0.3
    D = dirac.wilson_matrix(U, dims, m0).tocsr()
    perm, nb = permute.permutation(dims, permute.TYPE_I, 0, True)
    Dbb, Dbr, Drb, _ = schur.partition(D, perm, nb)
    want = Dbb.toarray() - (Dbr @ Drb).toarray() / (m0 + 4.0)
    got = reusken.reusken_dense(D, perm, nb, order=1)
    assert np.abs(got - want).max() <= 1e-13
    with pytest.raises(ValueError):
        reusken.ReuskenOperator(D, perm, nb, order=3)
