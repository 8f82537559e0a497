"""The paper's statements about the spectrum of S~^-1 S (Section 4, Fig. 4):
clustered around one, best for the Type II and Type II inverse permutations.
Checked on a 4^4 plaquette-action field at beta = 5.4 (the paper's smallest
coupling), m0 = -0.4."""
import numpy as np

import lattice_inputs as li
from oracle import dirac, permute, spectra


def test_approximate_schur_spectrum_clusters_around_one_best_for_type_II():
    dims = (4, 4, 4, 4)
    U = li.heatbath_gauge(dims, 5.4, 100, 3)
    D = dirac.wilson_matrix(U, dims, -0.4).tocsr()
    spread = {}
    for name, t, mu, inv in spectra.PERMUTATIONS:
        perm, nb = permute.permutation(dims, t, mu, inv)
        ev_S, ev_St, ev = spectra.spectra(D, perm, nb)
        assert ev_S.size == ev_St.size == ev.size == nb * 12
        assert np.abs(ev - 1).max() < 0.1            # clustered around one
        # det(S~^-1 S) = det S / det S~: the three spectra belong together
        lhs = np.log(np.abs(ev)).sum()
        rhs = np.log(np.abs(ev_S)).sum() - np.log(np.abs(ev_St)).sum()
        assert abs(lhs - rhs) <= 1e-8 * max(1.0, abs(rhs))
        assert abs(rhs) > 1e-3                       # S and S~ differ in determinant
        spread[name] = np.abs(ev - 1).mean()
    assert max(spread["P_II"], spread["P_II^T"]) < spread["P_I"]
    assert min(spread["P_II"], spread["P_II^T"]) <= spread["P_I^T"]


def test_condition_number_matches_dense_svd():
    """The Lanczos estimate (extreme eigenvalues of D^H D, small Krylov space
    so that ARPACK restarts) equals the 2-norm condition number of a dense
    SVD on a 2^4 and a 4x2x2x2 field."""
    for dims, m0 in (((2, 2, 2, 2), -0.5), ((4, 2, 2, 2), -0.9)):
        U = li.random_gauge(dims, 0.5, 7)
        D = dirac.wilson_matrix(U, dims, m0).tocsr()
        sv = np.linalg.svd(D.toarray(), compute_uv=False)
        kappa, smin, smax = spectra.condition_number(D, tol=1e-12, ncv=24)
        assert abs(smax - sv[0]) <= 1e-8 * sv[0]
        assert abs(smin - sv[-1]) <= 1e-8 * sv[0]
        assert abs(kappa - sv[0] / sv[-1]) <= 1e-7 * kappa


def test_leftmost_eigenvalues_match_dense():
    """Arnoldi's leftmost eigenvalues (restarted, small Krylov space) are the
    dense spectrum's eigenvalues of smallest real part, on a 4x2x2x2 field."""
    dims = (4, 2, 2, 2)
    U = li.random_gauge(dims, 0.5, 8)
    D = dirac.wilson_matrix(U, dims, -0.9).tocsr()
    dense = np.linalg.eigvals(D.toarray())
    want = np.sort(dense.real)[:4]
    for ncv in (120, 400):                         # Arnoldi, then the dense branch
        got = spectra.leftmost_eigenvalues(D, k=4, tol=1e-12, ncv=ncv)
        assert np.all(np.diff(got.real) >= -1e-12)  # returned by real part
        assert np.allclose(got.real, want, atol=1e-8)
        for z in got:                              # each is an eigenvalue of D
            assert np.abs(dense - z).min() < 1e-8
