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
        spread[name] = np.abs(ev - 1).mean()
    assert max(spread["P_II"], spread["P_II^T"]) < spread["P_I"]
    assert min(spread["P_II"], spread["P_II^T"]) <= spread["P_I^T"]
