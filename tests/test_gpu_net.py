"""The learned preconditioner: forward and backward kernels against the
oracle, training on pairs made by the method itself, FGMRES with the
network, and what the trained network gains over the method without it."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import lattice_inputs as li
from oracle import dirac, net as onet, permute
from tests.gpu_util import close, lib, maxrel, rel, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


def _ctx(gs, torch, dims, m0, U):
    ctx = gs.Context(dims, m0, torch.cuda.current_stream().cuda_stream)
    ctx.set_gauge(to_dev(U, torch))
    return ctx


@pytest.mark.parametrize("C", [4, 24])
def test_forward_backward_match_oracle(env, C):
    torch, gs = env
    dims, m0 = (4, 4, 2, 4), 0.1
    V = li.volume(dims)
    U = li.random_gauge(dims, 0.4, 2)
    ctx = _ctx(gs, torch, dims, m0, U)
    perm, nb = permute.permutation(dims, 1)
    nr = V - nb
    Ws = [w.astype(np.complex64) for w in onet.init_weights(C, 5, scale=0.25)]
    nt = gs.Net(C)
    for l, w in enumerate(Ws):
        nt.set_weights(l, w)
    rng = np.random.default_rng(1)
    t = (rng.standard_normal((nr, 12)) + 1j * rng.standard_normal((nr, 12))).astype(np.complex64)
    z = (rng.standard_normal((nr, 12)) + 1j * rng.standard_normal((nr, 12))).astype(np.complex64)
    # oracle on the same (rounded) numbers
    tr = onet.transports(U, dims)
    W64 = [w.astype(np.complex128) for w in Ws]
    tfull = np.zeros((V, 12), complex)
    tfull[perm[nb:]] = t
    acts = onet.forward(W64, tfull.reshape(V, 4, 3), tr)
    y = acts[-1].reshape(V, 12)
    L = onet.loss(y[perm[nb:]], z.astype(np.complex128))
    gy = np.zeros((V, 12), complex)
    gy[perm[nb:]] = 2.0 * (y[perm[nb:]] - z) / np.vdot(z, z).real
    G = onet.backward(W64, acts, gy.reshape(V, 1, 4, 3), tr)
    # GPU: one training step without update (FP32 weights)
    td = torch.from_numpy(t).to("cuda:0")[None].contiguous()
    zd = torch.from_numpy(z).to("cuda:0")[None].contiguous()
    loss = nt.train_step(ctx.handle, 1, 0, 0, 1, td, zd, 0.0, update=False)
    assert abs(loss - L) <= 1e-4 * L
    for l in range(3):
        g = nt.get(1, l).astype(np.complex128)
        assert close(g, G[l], 1e-4), l
    # inference (BF16 weights) against the oracle output
    t64 = to_dev(t.astype(np.complex128), torch)
    y64 = torch.empty_like(t64)
    nt.apply(ctx.handle, 1, 0, 0, t64, y64)
    torch.cuda.synchronize()
    got = y64.cpu().numpy()
    assert rel(got, y[perm[nb:]]) <= 3e-2 and maxrel(got, y[perm[nb:]]) <= 2 * 3e-2
    nt.close()
    ctx.close()


def _pairs(gs, torch, ctx, dims, nb, n, seed):
    from paper_0704_2341_gb300 import learned
    nr = li.volume(dims) - nb
    src = li.gaussian_source(dims, seed, n_src=n).reshape(n, -1, 12)[:, :nr]
    return learned.make_pairs(torch, ctx, 1, 0, 0, np.ascontiguousarray(src))


def test_training_reduces_loss_and_fgmres_net_solves(env):
    torch, gs = env
    from paper_0704_2341_gb300 import learned
    dims, m0 = (4, 4, 4, 4), 0.2
    U = li.random_gauge(dims, 0.3, 0)
    ctx = _ctx(gs, torch, dims, m0, U)
    perm, nb = permute.permutation(dims, 1)
    T, Z = _pairs(gs, torch, ctx, dims, nb, 24, 77)
    nt = gs.Net(8)
    for l, w in enumerate(learned.identity_like_weights(8, m0, 3)):
        nt.set_weights(l, w)
    hist = learned.train(torch, nt, [(ctx, 1, 0, 0, T, Z)], steps=80, batch=4, lr=2e-3, seed=5)
    assert np.mean(hist[-10:]) < 0.6 * np.mean(hist[:5])
    # the network inside FGMRES: the same 1e-10 solution as a direct solve
    ctx.set_net(nt)
    f = li.gaussian_source(dims, 100)
    fd = to_dev(f, torch)
    xd = torch.empty_like(fd)
    st = ctx.schur_solve(1, 0, 0, fd, xd, learned.fgmres_net_opts())
    xs = sla.spsolve(dirac.wilson_matrix(U, dims, m0).tocsc(), f.ravel())
    assert close(xd.cpu().numpy(), xs, 1e-9)
    assert st.true_residual <= 1e-10
    ctx.set_net(None)
    nt.close()
    ctx.close()


def test_learned_gain_over_the_method_without_it(env):
    """8^4 fields of the learned-preconditioner recipe (exp(i 0.2 H) + 10 APE
    steps, alpha 0.5), m0 = -0.38, Type I.  Train on pairs (t, D_rr^-1 t) from
    three seeded fields, then solve D_rr z = t on a held-out field to 1e-8:
    FGMRES with the trained network needs fewer Krylov steps than with the
    untrained (diagonal-inverse) network, and fewer D_rr applications than the
    plain BiCGStab; the answer is the same to the tolerance."""
    torch, gs = env
    from paper_0704_2341_gb300 import learned
    dims, m0 = (8, 8, 8, 8), -0.38
    perm, nb = permute.permutation(dims, 1)
    nr = li.volume(dims) - nb
    data, ctxs = [], []
    for s in (10, 11, 12):
        U = li.ape_smear(li.random_gauge(dims, 0.2, s), dims, 0.5, 10)
        ctx = _ctx(gs, torch, dims, m0, U)
        T, Z = _pairs(gs, torch, ctx, dims, nb, 64, 200 + s)
        data.append((ctx, 1, 0, 0, T, Z))
        ctxs.append(ctx)
    C = 24
    w0 = learned.identity_like_weights(C, m0, 4)
    nt = gs.Net(C)
    for l, w in enumerate(w0):
        nt.set_weights(l, w)
    hist = learned.train(torch, nt, data, steps=150, batch=4, lr=1e-3, seed=6)
    assert np.mean(hist[-10:]) < np.mean(hist[:5])
    U = li.ape_smear(li.random_gauge(dims, 0.2, 17), dims, 0.5, 10)
    ctx = _ctx(gs, torch, dims, m0, U)
    t = to_dev(li.gaussian_source(dims, 900).reshape(-1, 12)[:nr], torch)
    z_plain = torch.empty_like(t)
    st_plain = ctx.solve_rr(1, 0, 0, t, z_plain, gs.gs_default_opts(inner_prec=gs.GS_F32, inner_tol=1e-8))
    ctx.set_net(nt)
    z_net = torch.empty_like(t)
    st_net = ctx.solve_rr(1, 0, 0, t, z_net, learned.fgmres_net_opts(inner_tol=1e-8, lowp_tol=1e-8,
                                                                     inner_restart=64))
    untrained = gs.Net(C)
    for l, w in enumerate(w0):
        untrained.set_weights(l, w)
    ctx.set_net(untrained)
    z_id = torch.empty_like(t)
    st_id = ctx.solve_rr(1, 0, 0, t, z_id, learned.fgmres_net_opts(inner_tol=1e-8, lowp_tol=1e-8,
                                                                    inner_restart=64))
    ctx.set_net(None)
    assert close(z_net.cpu().numpy(), z_plain.cpu().numpy(), 1e-6)
    assert st_net.inner_iters < st_id.inner_iters
    assert st_net.inner_iters < 2 * st_plain.inner_iters   # D_rr applications: 1 vs 2 per step
    print("\nlearned gain on 8^4: FGMRES+trained net %d steps, FGMRES+untrained %d, "
          "BiCGStab %d iterations (%d D_rr applications)"
          % (st_net.inner_iters, st_id.inner_iters, st_plain.inner_iters, 2 * st_plain.inner_iters))
    for c in ctxs + [ctx]:
        c.close()
    nt.close()
    untrained.close()


@pytest.mark.parametrize("dims", [(4, 4, 2, 4), (16, 16, 16, 4)])
def test_tensor_core_layer_matches_cuda_cores_and_oracle(env, dims):
    """The 24 -> 24 layer on the tensor cores (BF16 transported activations,
    FP32 accumulation in tensor memory) against the CUDA-core path (FP32
    activations, same BF16 weights) and the FP64 oracle.  (4,4,2,4): 384
    GEMM rows, a ragged second tile; 16^3 x 4: 192 tiles, so CTAs run several
    tiles and the pipeline's barrier phases carry across tiles."""
    torch, gs = env
    m0 = -0.2
    V = li.volume(dims)
    U = li.random_gauge(dims, 0.5, 8)
    ctx = _ctx(gs, torch, dims, m0, U)
    perm, nb = permute.permutation(dims, 1)
    nr = V - nb
    Ws = [w.astype(np.complex64) for w in onet.init_weights(24, 11)]
    nt = gs.Net(24)
    for l, w in enumerate(Ws):
        nt.set_weights(l, w)
    t = li.gaussian_source(dims, 12).reshape(V, 12)[:nr]
    td = to_dev(t, torch)
    y_tc = torch.empty_like(td)
    y_cc = torch.empty_like(td)
    assert ctx.get_option(gs.GS_OPT_NET_KERNEL) == 0
    nt.apply(ctx.handle, 1, 0, 0, td, y_tc)
    ctx.set_option(gs.GS_OPT_NET_KERNEL, 1)
    nt.apply(ctx.handle, 1, 0, 0, td, y_cc)
    ctx.set_option(gs.GS_OPT_NET_KERNEL, 0)
    torch.cuda.synchronize()
    y_tc, y_cc = y_tc.cpu().numpy(), y_cc.cpu().numpy()
    assert np.isfinite(y_tc).all()
    # BF16 rounding of the transported activations only: ~1e-3 relative
    assert rel(y_tc, y_cc) <= 5e-3 and maxrel(y_tc, y_cc) <= 2 * 5e-3
    tfull = np.zeros((V, 12), complex)
    tfull[perm[nb:]] = t
    y = onet.forward([w.astype(np.complex128) for w in Ws], tfull.reshape(V, 4, 3),
                     onet.transports(U, dims))[-1].reshape(V, 12)[perm[nb:]]
    assert rel(y_tc, y) <= 1e-2 and maxrel(y_tc, y) <= 2 * 1e-2
    assert rel(y_cc, y) <= 1e-2 and maxrel(y_cc, y) <= 2 * 1e-2
    # repeated application is deterministic
    y2 = torch.empty_like(td)
    nt.apply(ctx.handle, 1, 0, 0, td, y2)
    assert np.array_equal(y2.cpu().numpy(), y_tc)
    nt.close()
    ctx.close()
