"""Training orchestration of the learned preconditioner (row A12).

Every arithmetic step runs in the library's kernels: the training pairs come
from the library's own inner solve (gs_solve_rr) or from its stencil
(t = D_rr z for a given z), the forward, backward and
Adam steps from gs_net_train_step.  This module only chooses the order of
the samples (a seeded generator), moves vectors between the complex128
solver layout and the complex64 training layout, and loops.
"""
from __future__ import annotations

import numpy as np

from ._binding import GS_F32, GS_INNER_FGMRES_NET, Net, gs_default_opts


def identity_like_weights(channels, m0, seed, noise=0.02):
    """Initial weights: M ~ 1/(m0 + 4) (the inverse of D_rr's diagonal) carried
    through channel 0 of every layer, plus seeded Gaussian noise."""
    rng = np.random.default_rng(seed)
    C = channels
    shapes = [(9, 4 * C, 4), (9, 4 * C, 4 * C), (9, 4, 4 * C)]
    Ws = []
    for shape in shapes:
        g = rng.standard_normal((2,) + shape)
        Ws.append((noise * (g[0] + 1j * g[1]) / np.sqrt(9 * shape[2])).astype(np.complex64))
    for s in range(4):
        Ws[0][0, s, s] += 1.0
        Ws[1][0, s, s] += 1.0
        Ws[2][0, s, s] += 1.0 / (m0 + 4.0)
    return Ws


def make_pairs(torch, ctx, ptype, dir, inverse, sources, inner_tol=1e-8):
    """z = D_rr^-1 t for every rest-set source (complex128 [n][n_r][12] numpy).
    Returns device complex64 tensors T, Z of shape [n, n_r, 12]."""
    n = sources.shape[0]
    opts = gs_default_opts(inner_prec=GS_F32, inner_tol=inner_tol)
    T = torch.from_numpy(np.ascontiguousarray(sources)).to("cuda")
    Z = torch.empty_like(T)
    for i in range(n):
        ctx.solve_rr(ptype, dir, inverse, T[i], Z[i], opts)
    return T.to(torch.complex64).contiguous(), Z.to(torch.complex64).contiguous()


def make_pairs_apply(torch, ctx, ptype, dir, inverse, Z):
    """Pairs (t, D_rr^-1 t) made the cheap way round: z is given (complex128
    [n][n_r][12], numpy or device), t = D_rr z.  D_rr z is the rest part of
    P D P^T [0; z] (the library's permute_sites and wilson_apply), so each
    pair costs one stencil application instead of an inner solve.  With z
    Gaussian the loss ||M t - z||^2 / ||z||^2 weighs every eigenmode of D_rr
    alike, the small ones included.  Returns device complex64 T, Z."""
    Zd = torch.as_tensor(np.ascontiguousarray(Z) if isinstance(Z, np.ndarray) else Z,
                         device="cuda").to(torch.complex128)
    n, nr = Zd.shape[0], Zd.shape[1]
    V = ctx.volume
    nb = V - nr
    lab = torch.zeros((V, 12), dtype=torch.complex128, device="cuda")
    site = torch.empty_like(lab)
    dsite = torch.empty_like(lab)
    dlab = torch.empty_like(lab)
    T = torch.empty((n, nr, 12), dtype=torch.complex64, device="cuda")
    for i in range(n):
        lab[nb:] = Zd[i]
        ctx.permute_sites(ptype, dir, inverse, 1, lab, site)
        ctx.wilson_apply(site, dsite)
        ctx.permute_sites(ptype, dir, inverse, 0, dsite, dlab)
        T[i] = dlab[nb:]
    return T, Zd.to(torch.complex64).contiguous()


def train(torch, net, datasets, steps, batch, lr, seed):
    """datasets: list of (ctx, ptype, dir, inverse, T, Z).  Each step picks a
    data set and `batch` pairs with a seeded generator and runs one training
    step.  Returns the loss history."""
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(steps):
        ctx, ptype, dir, inverse, T, Z = datasets[int(rng.integers(len(datasets)))]
        idx = torch.from_numpy(rng.choice(T.shape[0], size=batch, replace=False)).to(T.device)
        tb = T.index_select(0, idx).contiguous()
        zb = Z.index_select(0, idx).contiguous()
        hist.append(net.train_step(ctx.handle, ptype, dir, inverse, batch, tb, zb, lr))
    return hist


def fgmres_net_opts(**kw):
    """Solver options that run the inner solve as FGMRES with the attached network."""
    o = dict(inner_prec=GS_F32, inner_solver=GS_INNER_FGMRES_NET)
    o.update(kw)
    return gs_default_opts(**o)


__all__ = ["Net", "identity_like_weights", "make_pairs", "make_pairs_apply", "train", "fgmres_net_opts"]
