"""Seeded synthetic inputs: SU(3) gauge fields and fermion sources.

This module is shared by the CPU oracle, the tests and the benchmark.  It
holds none of the Schur-complement method's arithmetic (no Dirac operator,
no site permutation, no Krylov solver); it only manufactures the background
gauge fields and right-hand sides the method is applied to.

The paper computes its Schur complements "in a SU(3) background field using
the plaquette action" at beta = 5.4, 5.7, 5.9 (Section 1, around Fig. 2, and
Section 4, Table 1).  Those ensembles are not available, so three seeded
stand-ins are produced here:

* ``random_gauge``: U = exp(i eps H), H traceless Hermitian with Gaussian
  entries (a rough field whose roughness is set by eps);
* ``ape_smear``: APE smearing of a field, projected back to SU(3);
* ``heatbath_gauge``: the plaquette (Wilson) action sampled by a
  Cabibbo-Marinari pseudo-heatbath over the three SU(2) subgroups, each SU(2)
  drawn with the Kennedy-Pendleton algorithm (Phys. Lett. B156 (1985) 393).

Layout conventions (shared with the CUDA library by agreement, not code):

* lattice extents ``dims = (L0, L1, L2, L3)``; site index
  ``s = x0 + L0*(x1 + L1*(x2 + L2*x3))`` (x0 fastest);
* gauge field ``U`` is complex128 of shape ``(V, 4, 3, 3)``: ``U[s, mu]`` is the
  3x3 matrix on the link from site s to s + mu-hat, row-major (row = first
  colour index);
* spinor fields are complex128 of shape ``(V, 4, 3)``: ``[site][spin][colour]``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "random_gauge",
    "ape_smear",
    "heatbath_gauge",
    "average_plaquette",
    "gaussian_source",
    "point_sources",
    "training_gauge",
    "prepare_training_gauges",
    "coupling_gauge",
    "workload_gauge",
    "random_su3",
]


def volume(dims) -> int:
    v = 1
    for L in dims:
        v *= int(L)
    return v


# ---------------------------------------------------------------------------
# lattice helpers (pure data movement on the (L3, L2, L1, L0, ...) grid)
# ---------------------------------------------------------------------------

def _to_grid(U, dims):
    L0, L1, L2, L3 = dims
    return U.reshape(L3, L2, L1, L0, *U.shape[1:])


def _shift(F, mu, step):
    """F(x + step*mu-hat) on a grid array with axes (x3, x2, x1, x0, ...)."""
    axis = 3 - mu
    return np.roll(F, -step, axis=axis)


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _parity_mask(dims):
    L0, L1, L2, L3 = dims
    x3, x2, x1, x0 = np.meshgrid(np.arange(L3), np.arange(L2), np.arange(L1),
                                 np.arange(L0), indexing="ij")
    return ((x0 + x1 + x2 + x3) % 2).astype(np.int8)


# ---------------------------------------------------------------------------
# exp(i eps H)
# ---------------------------------------------------------------------------

def _traceless_hermitian(A):
    H = 0.5 * (A + _dag(A))
    tr = np.trace(H, axis1=-2, axis2=-1)
    return H - (tr / 3.0)[..., None, None] * np.eye(3)


def _expi_hermitian(H, eps):
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", v, ph, np.conj(v))


def random_gauge(dims, eps, seed) -> np.ndarray:
    """U_mu(x) = exp(i eps H_mu(x)), H traceless Hermitian from Gaussian A.

    A has i.i.d. N(0,1) real and imaginary parts, drawn from
    ``numpy.random.default_rng(seed)`` as one array of shape
    (2, L3, L2, L1, L0, 4, 3, 3): index 0 is the real part, 1 the imaginary.
    H = (A + A^dagger)/2 - tr(.)/3.  The exponential is taken through ``eigh``.
    """
    L0, L1, L2, L3 = dims
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((2, L3, L2, L1, L0, 4, 3, 3))
    A = g[0] + 1j * g[1]
    U = _expi_hermitian(_traceless_hermitian(A), eps)
    return np.ascontiguousarray(U.reshape(volume(dims), 4, 3, 3))


def random_su3(shape, seed) -> np.ndarray:
    """Haar-ish random SU(3) matrices (QR of a complex Gaussian, phase-fixed)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((2, *shape, 3, 3))
    Z = g[0] + 1j * g[1]
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[..., None, None]


# ---------------------------------------------------------------------------
# APE smearing
# ---------------------------------------------------------------------------

def _project_su3(M):
    """Nearest unitary by polar decomposition, then remove the phase of det."""
    u, _, vh = np.linalg.svd(M)
    W = u @ vh
    det = np.linalg.det(W)
    return W * np.exp(-1j * np.angle(det) / 3.0)[..., None, None]


def ape_smear(U, dims, alpha, steps) -> np.ndarray:
    """APE smearing, ``steps`` times:

    U'_mu(x) = Proj_SU(3)[ (1 - alpha) U_mu(x) + alpha/6 * sum_{nu != mu} C_mu,nu(x) ]

    with the two staples C = U_nu(x) U_mu(x+nu) U_nu(x+mu)^dagger
    + U_nu(x-nu)^dagger U_mu(x-nu) U_nu(x-nu+mu).  All directions are updated
    from the same old field in each step.
    """
    G = _to_grid(np.asarray(U, dtype=np.complex128), dims).copy()
    for _ in range(int(steps)):
        new = np.empty_like(G)
        for mu in range(4):
            C = np.zeros(G.shape[:4] + (3, 3), dtype=np.complex128)
            for nu in range(4):
                if nu == mu:
                    continue
                Un = G[..., nu, :, :]
                Um = G[..., mu, :, :]
                up = Un @ _shift(Um, nu, 1) @ _dag(_shift(Un, mu, 1))
                Un_m = _shift(Un, nu, -1)
                dn = _dag(Un_m) @ _shift(Um, nu, -1) @ _shift(Un_m, mu, 1)
                C += up + dn
            new[..., mu, :, :] = _project_su3((1.0 - alpha) * G[..., mu, :, :]
                                              + (alpha / 6.0) * C)
        G = new
    return np.ascontiguousarray(G.reshape(volume(dims), 4, 3, 3))


# ---------------------------------------------------------------------------
# plaquette-action pseudo-heatbath
#
# A heatbath chain amplifies the last bit of any rounding difference into a
# different configuration after a few hundred sweeps, so every step below
# uses only IEEE-754 operations that are correctly rounded on every machine
# (+, -, x, /, sqrt on float64 arrays, one operation per numpy call, and
# frexp): no BLAS products, no library log / cos, no SVD.  The same seed gives
# the same field bit for bit on x86 and on Arm.
# ---------------------------------------------------------------------------

def _cmm(A, B):
    """Complex matrix product A @ B for stacks (..., n, k) x (..., k, m) in
    real arithmetic with a fixed summation order."""
    Ar, Ai, Br, Bi = A.real, A.imag, B.real, B.imag
    Cr = Ar[..., :, 0:1] * Br[..., 0:1, :]
    Cr = Cr - Ai[..., :, 0:1] * Bi[..., 0:1, :]
    Ci = Ar[..., :, 0:1] * Bi[..., 0:1, :]
    Ci = Ci + Ai[..., :, 0:1] * Br[..., 0:1, :]
    for j in range(1, A.shape[-1]):
        Cr = Cr + Ar[..., :, j:j + 1] * Br[..., j:j + 1, :]
        Cr = Cr - Ai[..., :, j:j + 1] * Bi[..., j:j + 1, :]
        Ci = Ci + Ar[..., :, j:j + 1] * Bi[..., j:j + 1, :]
        Ci = Ci + Ai[..., :, j:j + 1] * Br[..., j:j + 1, :]
    C = np.empty(Cr.shape, dtype=np.complex128)
    C.real = Cr
    C.imag = Ci
    return C


def _reunitarize(M):
    """SU(3) from the first two rows of each 3 x 3 matrix: Gram-Schmidt, then
    row 3 = conj(row 1 x row 2) (determinant 1 by construction)."""
    ur, ui = M[..., 0, :].real.copy(), M[..., 0, :].imag.copy()
    vr, vi = M[..., 1, :].real.copy(), M[..., 1, :].imag.copy()
    n = np.sqrt(ur[..., 0] * ur[..., 0] + ui[..., 0] * ui[..., 0] + ur[..., 1] * ur[..., 1]
                + ui[..., 1] * ui[..., 1] + ur[..., 2] * ur[..., 2] + ui[..., 2] * ui[..., 2])
    ur = ur / n[..., None]
    ui = ui / n[..., None]
    # <u, v> = sum conj(u_i) v_i
    pr = ur[..., 0] * vr[..., 0] + ui[..., 0] * vi[..., 0]
    pi = ur[..., 0] * vi[..., 0] - ui[..., 0] * vr[..., 0]
    for i in (1, 2):
        pr = pr + ur[..., i] * vr[..., i]
        pr = pr + ui[..., i] * vi[..., i]
        pi = pi + ur[..., i] * vi[..., i]
        pi = pi - ui[..., i] * vr[..., i]
    vr = vr - (pr[..., None] * ur - pi[..., None] * ui)
    vi = vi - (pr[..., None] * ui + pi[..., None] * ur)
    n = np.sqrt(vr[..., 0] * vr[..., 0] + vi[..., 0] * vi[..., 0] + vr[..., 1] * vr[..., 1]
                + vi[..., 1] * vi[..., 1] + vr[..., 2] * vr[..., 2] + vi[..., 2] * vi[..., 2])
    vr = vr / n[..., None]
    vi = vi / n[..., None]
    out = np.empty(M.shape, dtype=np.complex128)
    out[..., 0, :].real, out[..., 0, :].imag = ur, ui
    out[..., 1, :].real, out[..., 1, :].imag = vr, vi
    for c, (a, b) in enumerate(((1, 2), (2, 0), (0, 1))):
        # (u x v)_c = u_a v_b - u_b v_a; row 3 is its complex conjugate
        xr = (ur[..., a] * vr[..., b] - ui[..., a] * vi[..., b]) - (ur[..., b] * vr[..., a] - ui[..., b] * vi[..., a])
        xi = (ur[..., a] * vi[..., b] + ui[..., a] * vr[..., b]) - (ur[..., b] * vi[..., a] + ui[..., b] * vr[..., a])
        out[..., 2, c].real = xr
        out[..., 2, c].imag = -xi
    return out


_LN2 = 0.6931471805599453


def _log(x):
    """Natural logarithm of positive float64 values: x = m 2^e exactly
    (frexp), m moved into [1/sqrt 2, sqrt 2), log m = 2 atanh(s) with
    s = (m - 1) / (m + 1), |s| < 0.172, summed as the odd series to s^25
    (error below 1e-17 relative to log m)."""
    m, e = np.frexp(x)
    low = m < 0.7071067811865476
    m = np.where(low, m * 2.0, m)
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    acc = np.full_like(s, 1.0 / 25.0)
    for k in range(23, 0, -2):
        acc = acc * s2 + 1.0 / k
    return e * _LN2 + 2.0 * s * acc


def _unit_circle(n, rng):
    """n points (c, s) uniform on the unit circle, by rejection from the square."""
    c = np.empty(n)
    s = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x = 2.0 * rng.random(todo.size) - 1.0
        y = 2.0 * rng.random(todo.size) - 1.0
        r2 = x * x + y * y
        ok = (r2 <= 1.0) & (r2 > 1e-12)
        r = np.sqrt(r2[ok])
        c[todo[ok]] = x[ok] / r
        s[todo[ok]] = y[ok] / r
        todo = todo[~ok]
    return c, s


def _staple_sum(G, mu):
    """A_mu(x) with Re tr(U_mu(x) A_mu(x)) = sum of the 6 plaquettes through the link."""
    A = np.zeros(G.shape[:4] + (3, 3), dtype=np.complex128)
    Um = G[..., mu, :, :]
    for nu in range(4):
        if nu == mu:
            continue
        Un = G[..., nu, :, :]
        # forward: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        A = A + _cmm(_cmm(_shift(Un, mu, 1), _dag(_shift(Um, nu, 1))), _dag(Un))
        # backward: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        Un_m = _shift(Un, nu, -1)
        A = A + _cmm(_cmm(_dag(_shift(Un_m, mu, 1)), _dag(_shift(Um, nu, -1))), Un_m)
    return A


def _nbr_tables(dims):
    """Flat site indices of x + mu and x - mu for every site, per direction
    (site order: x0 fastest), periodic."""
    L0, L1, L2, L3 = dims
    idx = np.arange(volume(dims)).reshape(L3, L2, L1, L0)
    fwd = [np.roll(idx, -1, axis=3 - mu).ravel() for mu in range(4)]
    bwd = [np.roll(idx, 1, axis=3 - mu).ravel() for mu in range(4)]
    return fwd, bwd


def _staple_sites(Gf, mu, S, fwd, bwd):
    """_staple_sum restricted to the sites S (flat indices; Gf: (V, 4, 3, 3)),
    term for term in the same order, so its values equal those of the whole-
    lattice sum at those sites bit for bit."""
    A = np.zeros((S.size, 3, 3), dtype=np.complex128)
    xm = fwd[mu][S]
    for nu in range(4):
        if nu == mu:
            continue
        xn, xb = fwd[nu][S], bwd[nu][S]
        A = A + _cmm(_cmm(Gf[xm, nu], _dag(Gf[xn, mu])), _dag(Gf[S, nu]))
        xmb = bwd[nu][xm]
        A = A + _cmm(_cmm(_dag(Gf[xmb, nu]), _dag(Gf[xb, mu])), Gf[xb, nu])
    return A


def _kp_sample_x0(alpha, rng):
    """Kennedy-Pendleton: x0 in [-1, 1] with density ~ sqrt(1 - x0^2) exp(alpha x0).
    cos^2 of a uniform angle is the squared first coordinate of a uniform
    point on the unit circle."""
    n = alpha.shape[0]
    out = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        a = alpha[todo]
        r1 = 1.0 - rng.random(todo.size)
        c, _ = _unit_circle(todo.size, rng)
        r3 = 1.0 - rng.random(todo.size)
        r4 = rng.random(todo.size)
        delta = -(_log(r1) + (c * c) * _log(r3)) / a
        ok = r4 * r4 <= 1.0 - 0.5 * delta
        out[todo[ok]] = 1.0 - delta[ok]
        todo = todo[~ok]
    return out


def _su2_heatbath_update(Ulinks, A, beta, rng, sub):
    """One Cabibbo-Marinari SU(2) subgroup update of a batch of SU(3) links.

    Ulinks, A: (n, 3, 3).  Returns the updated links.
    """
    i, j = sub
    W = _cmm(Ulinks, A)
    w00, w01, w10, w11 = W[:, i, i], W[:, i, j], W[:, j, i], W[:, j, j]
    a0 = 0.5 * (w00 + w11).real
    a3 = 0.5 * (w00 - w11).imag
    a2 = 0.5 * (w01 - w10).real
    a1 = 0.5 * (w01 + w10).imag
    k = np.sqrt(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3)
    k = np.maximum(k, 1e-300)
    x0 = _kp_sample_x0(2.0 * beta * k / 3.0, rng)
    # uniform direction for the remaining three components
    rad = np.sqrt(np.maximum(0.0, 1.0 - x0 * x0))
    cth = 2.0 * rng.random(x0.shape[0]) - 1.0
    cph, sph = _unit_circle(x0.shape[0], rng)
    sth = np.sqrt(1.0 - cth * cth)
    x1 = rad * sth * cph
    x2 = rad * sth * sph
    x3 = rad * cth
    # quaternion product x * what^dagger, what = (a0, a1, a2, a3)/k
    b0, b1, b2, b3 = a0 / k, -a1 / k, -a2 / k, -a3 / k
    r0 = x0 * b0 - x1 * b1 - x2 * b2 - x3 * b3
    r1 = x0 * b1 + x1 * b0 - x2 * b3 + x3 * b2
    r2 = x0 * b2 + x2 * b0 - x3 * b1 + x1 * b3
    r3 = x0 * b3 + x3 * b0 - x1 * b2 + x2 * b1
    # embedded 2x2: r0 + i (r1 s1 + r2 s2 + r3 s3)
    R = np.empty((x0.shape[0], 2, 2), dtype=np.complex128)
    R[:, 0, 0].real, R[:, 0, 0].imag = r0, r3
    R[:, 0, 1].real, R[:, 0, 1].imag = r2, r1
    R[:, 1, 0].real, R[:, 1, 0].imag = -r2, r1
    R[:, 1, 1].real, R[:, 1, 1].imag = r0, -r3
    rows = Ulinks[:, [i, j], :]
    out = Ulinks.copy()
    out[:, [i, j], :] = _cmm(R, rows)
    return out


def heatbath_gauge(dims, beta, sweeps, seed, start=None) -> np.ndarray:
    """Quenched SU(3) field from the Wilson plaquette action at coupling beta.

    Cold start (all links = 1) unless ``start`` is given; each sweep visits
    mu = 0..3 and, for each mu, the even then the odd sites (checkerboard:
    links of one direction on one parity share no staple), and performs the
    three Cabibbo-Marinari subgroup updates (0,1), (1,2), (0,2).  All L_mu
    must be even.  Random numbers come from ``numpy.random.default_rng(seed)``;
    only correctly rounded float64 operations act on them, so the field is the
    same bit for bit on every machine.
    """
    if any(int(L) % 2 for L in dims):
        raise ValueError("heatbath checkerboard needs even extents")
    rng = np.random.default_rng(seed)
    V = volume(dims)
    if start is None:
        G = np.broadcast_to(np.eye(3, dtype=np.complex128),
                            (V, 4, 3, 3)).copy()
    else:
        G = np.array(start, dtype=np.complex128, copy=True)
    G = np.ascontiguousarray(G.reshape(V, 4, 3, 3))
    par = _parity_mask(dims).ravel()
    sites = [np.flatnonzero(par == p) for p in (0, 1)]
    fwd, bwd = _nbr_tables(dims)
    for _ in range(int(sweeps)):
        for mu in range(4):
            for p in (0, 1):
                S = sites[p]
                As = _staple_sites(G, mu, S, fwd, bwd)
                links = G[S, mu]
                for sub in ((0, 1), (1, 2), (0, 2)):
                    links = _su2_heatbath_update(links, As, beta, rng, sub)
                G[S, mu] = links
        # keep the links unitary against rounding drift
        G = _reunitarize(G)
    return G


def average_plaquette(U, dims) -> float:
    """<(1/3) Re tr U_mu,nu(x)> over sites and the 6 planes (a checksum)."""
    G = _to_grid(np.asarray(U), dims)
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Um, Un = G[..., mu, :, :], G[..., nu, :, :]
            P = Um @ _shift(Un, mu, 1) @ _dag(_shift(Um, nu, 1)) @ _dag(Un)
            tot += np.trace(P, axis1=-2, axis2=-1).real.mean() / 3.0
    return tot / 6.0


# ---------------------------------------------------------------------------
# sources
# ---------------------------------------------------------------------------

def gaussian_source(dims, seed, n_src=1) -> np.ndarray:
    """Complex Gaussian source(s): re and im parts i.i.d. N(0,1).

    Drawn as one array of shape (2, n_src, V, 4, 3).  Returns (V, 4, 3) for
    n_src == 1, else (n_src, V, 4, 3).
    """
    V = volume(dims)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((2, n_src, V, 4, 3))
    src = g[0] + 1j * g[1]
    return src[0] if n_src == 1 else src


def point_sources(dims, site=0) -> np.ndarray:
    """The 12 spin-colour point sources delta_{x,site} delta_{a,spin} delta_{i,col}."""
    V = volume(dims)
    out = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for k in range(12):
        out[k, site, k // 3, k % 3] = 1.0
    return out


# ---------------------------------------------------------------------------
# on-disk cache for the slow generators (a convenience; never required)
# ---------------------------------------------------------------------------

# bumped whenever a generator's output changes, so that no stale field is read
# (2: the heatbath in correctly rounded arithmetic only)
_CACHE_VERSION = 2


def _cache_path(name):
    import os
    root = os.environ.get("GSCHUR_FIELD_CACHE")
    if root is None:
        root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            ".cache", "fields")
    return os.path.join(root, "%s.v%d.npy" % (name, _CACHE_VERSION))


def cached(name, make):
    """Load ``name`` from the field cache, else build it with ``make()`` and store it."""
    import os
    path = _cache_path(name)
    if os.path.exists(path):
        try:
            return np.load(path)
        except (OSError, ValueError):
            pass
    arr = make()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d.npy" % os.getpid()
        np.save(tmp, arr)
        os.replace(tmp, path)
    except OSError:
        pass
    return arr


def training_gauge(kind, index):
    """The seeded gauge fields the learned preconditioner is trained on (8^4).

    * ``"heatbath"``: plaquette action beta = 5.4, 200 Cabibbo-Marinari
      sweeps from a cold start, seed 11 + index (the ensemble of the
      ``"8^4 heatbath b5.4"`` workload, other seeds);
    * ``"ape"``: exp(i 0.2 H) seed 100 + index, then 10 APE steps alpha 0.5
      (the recipe of the ``"32^3x64 eps0.2 ape10"`` workload on 8^4).
    """
    dims = (8, 8, 8, 8)
    if kind == "heatbath":
        seed = 11 + int(index)
        return dims, cached("train_8p4_heatbath_b5.4_s%d" % seed, lambda: heatbath_gauge(dims, 5.4, 200, seed))
    if kind == "ape":
        seed = 100 + int(index)
        return dims, cached("train_8p4_eps0.2_ape10_s%d" % seed,
                            lambda: ape_smear(random_gauge(dims, 0.2, seed), dims, 0.5, 10))
    raise KeyError(kind)


def coupling_gauge(beta, index=0):
    """8^4 plaquette-action field at coupling beta (200 Cabibbo-Marinari
    sweeps from a cold start, seed 21 + index + 100 (beta - 5.4) rounded),
    the stand-ins for the paper's beta = 5.4, 5.7, 5.9 ensembles (cached)."""
    dims = (8, 8, 8, 8)
    seed = 21 + int(index) + int(round(100 * (beta - 5.4)))
    key = "coupling_8p4_b%.2f_s%d" % (beta, seed)
    return dims, cached(key, lambda: heatbath_gauge(dims, beta, 200, seed))


def _make_training_gauge(args):
    training_gauge(*args)
    return True


def prepare_training_gauges(kind, n=8, processes=8):
    """Fill the field cache with training_gauge(kind, 0 .. n-1), generating
    the missing ones in parallel worker processes (started with ``spawn``,
    so this is safe in a process that already uses CUDA)."""
    import multiprocessing as mp
    import os
    todo = [(kind, i) for i in range(n)
            if not os.path.exists(_cache_path(("train_8p4_heatbath_b5.4_s%d" % (11 + i)) if kind == "heatbath"
                                              else ("train_8p4_eps0.2_ape10_s%d" % (100 + i))))]
    if not todo:
        return
    with mp.get_context("spawn").Pool(min(processes, len(todo))) as pool:
        pool.map(_make_training_gauge, todo)


def _make_gauge(spec):
    kind, a, b = spec
    if kind == "training":
        training_gauge(a, b)
    elif kind == "coupling":
        coupling_gauge(a, b)
    else:
        workload_gauge(a)
    return True


def _gauge_cached(spec):
    import os
    kind, a, b = spec
    if kind == "training":
        key = ("train_8p4_heatbath_b5.4_s%d" % (11 + b)) if a == "heatbath" else \
            ("train_8p4_eps0.2_ape10_s%d" % (100 + b))
    elif kind == "coupling":
        key = "coupling_8p4_b%.2f_s%d" % (a, 21 + int(b) + int(round(100 * (a - 5.4))))
    else:
        key = a.replace("^", "p").replace(" ", "_")
    return os.path.exists(_cache_path(key))


def prepare_gauges(specs, processes=16):
    """Fill the field cache for several fields at once, generating the missing
    ones in parallel worker processes (started with ``spawn``, so this is safe
    in a process that already uses CUDA).  specs: ("training", kind, i),
    ("coupling", beta, index) or ("workload", name, None)."""
    import multiprocessing as mp
    import os
    todo = [tuple(sp) for sp in specs if not _gauge_cached(sp)]
    if not todo:
        return 0
    n = max(1, min(processes, len(todo), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(_make_gauge, todo)
    return len(todo)


def workload_gauge(name):
    """The seeded gauge field of one of the named workloads.

    * ``"4^4 eps0.3"``            : 4^4, exp(i 0.3 H), seed 0
    * ``"8^4 heatbath b5.4"``     : 8^4, plaquette action beta = 5.4,
                                    200 Cabibbo-Marinari sweeps, cold start, seed 1
    * ``"16^3x32 eps0.25 ape5"``  : 16^3 x 32, exp(i 0.25 H) seed 2, 5 APE steps alpha 0.5
    * ``"24^3x48 eps0.2"``        : 24^3 x 48, exp(i 0.2 H), seed 3
    * ``"16^4 eps0.2"``           : 16^4, exp(i 0.2 H), seed 4
    * ``"8^4 eps0.2"``            : 8^4, exp(i 0.2 H), seed 6
    * ``"32^3x64 eps0.2 ape10"``  : 32^3 x 64, exp(i 0.2 H) seed 5, 10 APE steps alpha 0.5
    """
    table = {
        "4^4 eps0.3": ((4, 4, 4, 4), lambda d: random_gauge(d, 0.3, 0)),
        "8^4 heatbath b5.4": ((8, 8, 8, 8), lambda d: heatbath_gauge(d, 5.4, 200, 1)),
        "16^3x32 eps0.25 ape5": ((16, 16, 16, 32),
                                 lambda d: ape_smear(random_gauge(d, 0.25, 2), d, 0.5, 5)),
        "24^3x48 eps0.2": ((24, 24, 24, 48), lambda d: random_gauge(d, 0.2, 3)),
        "16^4 eps0.2": ((16, 16, 16, 16), lambda d: random_gauge(d, 0.2, 4)),
        "8^4 eps0.2": ((8, 8, 8, 8), lambda d: random_gauge(d, 0.2, 6)),
        "32^3x64 eps0.2 ape10": ((32, 32, 32, 64),
                                 lambda d: ape_smear(random_gauge(d, 0.2, 5), d, 0.5, 10)),
    }
    dims, make = table[name]
    key = name.replace("^", "p").replace(" ", "_")
    return dims, cached(key, lambda: make(dims))
