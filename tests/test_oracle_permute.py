"""Pins of the oracle's site permutations (Section 2 and Fig. 1's 4x4 size)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import permute
from oracle.permute import TYPE_I, TYPE_II


def _read_golden(path):
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, labels = line.split(":")
        name, nb = head.split()
        out[name] = (int(nb), np.array([int(v) for v in labels.split()]))
    return out


def test_4x4_hand_derived(golden_dir):
    g = _read_golden(os.path.join(golden_dir, "perm_4x4.txt"))
    cases = {"p_I": (TYPE_I, 0, False), "q_I": (TYPE_I, 0, True),
             "p_II0": (TYPE_II, 0, False), "q_II0": (TYPE_II, 0, True),
             "p_II1": (TYPE_II, 1, False), "q_II1": (TYPE_II, 1, True)}
    for name, (t, mu, inv) in cases.items():
        perm, nb = permute.permutation((4, 4), t, mu, inv)
        assert nb == g[name][0], name
        assert np.array_equal(perm, g[name][1]), name


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 2, 8)])
@pytest.mark.parametrize("t,mu", [(TYPE_I, 0), (TYPE_II, 0), (TYPE_II, 2), (TYPE_II, 3)])
def test_inverse_round_trip(dims, t, mu):
    p, nb = permute.permutation(dims, t, mu, False)
    q, nb2 = permute.permutation(dims, t, mu, True)
    assert nb == nb2
    V = int(np.prod(dims))
    assert np.array_equal(np.sort(p), np.arange(V))
    assert np.array_equal(p[q], np.arange(V))
    assert np.array_equal(q[p], np.arange(V))
    P = permute.perm_matrix(p, 12)
    assert (P.T @ P != sp.eye(V * 12, format='csr')).nnz == 0
    x = np.arange(V * 12)
    assert np.array_equal(P.T @ (P @ x), x)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
def test_coarse_sets_as_coordinates(dims):
    V = int(np.prod(dims))
    s = np.arange(V)
    x0 = s % dims[0]
    x1 = (s // dims[0]) % dims[1]
    x2 = (s // (dims[0] * dims[1])) % dims[2]
    x3 = s // (dims[0] * dims[1] * dims[2])
    X = np.stack([x0, x1, x2, x3], 1)
    p, nb = permute.permutation(dims, TYPE_I)
    assert nb == V // 16
    assert np.array_equal(p[:nb], s[np.all(X % 2 == 0, axis=1)])
    assert np.all(np.diff(p[:nb]) > 0) and np.all(np.diff(p[nb:]) > 0)
    for mu in range(4):
        p, nb = permute.permutation(dims, TYPE_II, mu)
        assert nb == V // 2
        assert np.array_equal(p[:nb], s[X[:, mu] % 2 == 0])
        assert np.all(np.diff(p[nb:]) > 0)


def test_inverse_type_II_closed_form():
    """For Type II along x0 with L0 even, the label of site j is j/2 for even
    j and V/2 + (j-1)/2 for odd j, so q[j] has that closed form and the
    coarse set of P_II^T is the two slabs s < V/4 and V/2 <= s < 3V/4
    (on 8^4: x3 in {0, 1, 4, 5})."""
    dims = (8, 8, 8, 8)
    V = 4096
    q, nb = permute.permutation(dims, TYPE_II, 0, True)
    j = np.arange(V)
    assert np.array_equal(q, np.where(j % 2 == 0, j // 2, V // 2 + (j - 1) // 2))
    b = np.sort(q[:nb])
    x3 = b // 512
    assert set(np.unique(x3)) == {0, 1, 4, 5}


def test_inverse_type_I_brute_force():
    """q[j] = rank of site j in the label order, counted by brute force."""
    dims = (4, 2, 2, 4)
    p, nb = permute.permutation(dims, TYPE_I)
    q, _ = permute.permutation(dims, TYPE_I, 0, True)
    V = 64
    for j in range(V):
        rank = [i for i in range(V) if p[i] == j]
        assert q[j] == rank[0]


def test_rejects_odd_extent():
    with pytest.raises(ValueError):
        permute.permutation((3, 4, 4, 4), TYPE_I)
    with pytest.raises(ValueError):
        permute.permutation((3, 4, 4, 4), TYPE_II, 0)
    permute.permutation((3, 4, 4, 4), TYPE_II, 1)


def test_inverse_type_I_coarse_set_4x4x4x4_hand_derived():
    """P_I^T on 4^4 (s = x0 + 4 x1 + 16 x2 + 64 x3): the coarse set is
    {q(0), ..., q(15)}, the labels of sites 0..15 (x2 = x3 = 0).  Of these the
    all-even sites 0, 2, 8, 10 are the first four coarse sites of P_I (labels
    0..3); the other twelve are the first twelve rest sites (labels 16..27).
    As sites: x0 = 0..3 with x1 = x2 = 0, and x0 = 0..3, x1 = 0..2, x2 = 1."""
    q, nb = permute.permutation((4, 4, 4, 4), TYPE_I, 0, True)
    assert nb == 16
    assert list(q[:16]) == [0, 16, 1, 17, 18, 19, 20, 21, 2, 22, 3, 23, 24, 25, 26, 27]
    assert sorted(q[:16]) == list(range(4)) + list(range(16, 28))
