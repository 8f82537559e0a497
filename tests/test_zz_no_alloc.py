"""wilson_apply_noalloc against wilson_apply (GPU, through the C ABI).

The no-allocation entry point serves callers that cannot allocate device
memory themselves -- for instance a service whose device memory is all handed
out by its own pool, or one that cannot afford the device-wide
synchronisation that freeing memory implies.  It must give the same D x as the
context-based entry point while keeping its scratch (neighbour table, packed
links) in one static device array that every call reuses.  This file is named
to be collected last.
"""
import numpy as np
import pytest

import lattice_inputs as li
from oracle import dirac
from tests.gpu_util import lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_noalloc_matches_wilson_apply_on_two_calls_in_a_row():
    torch = torch_cuda()
    gs = lib()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row on different lattices: the second must not see the
    # first call's tables left in the shared array
    for dims, eps, m0, seed in [((8, 8, 8, 8), 0.3, -0.4, 1), ((4, 6, 2, 6), 0.5, 0.2, 2)]:
        U = to_dev(li.random_gauge(dims, eps, seed), torch)
        x = to_dev(li.gaussian_source(dims, seed + 10), torch)
        y_ref = torch.empty_like(x)
        ctx = gs.Context(dims, m0, stream)
        ctx.set_gauge(U)
        ctx.wilson_apply(x, y_ref)
        y = torch.full_like(x, float("nan"))
        status = gs.wilson_apply_noalloc(dims, m0, U, x, y, stream)
        assert status == gs.GS_OK
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
        # and directly against the oracle's assembled D, element by element
        ref = dirac.wilson_matrix(U.cpu().numpy(), dims, m0) @ x.cpu().numpy().ravel()
        assert np.abs(a.ravel() - ref).max() <= 1e-13 * np.abs(ref).max()
        ctx.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    torch = torch_cuda()
    gs = lib()
    dims = (16, 16, 8, 8)   # 16384 sites > 8192
    z = torch.zeros(1, dtype=torch.complex128, device="cuda:0")
    assert gs.wilson_apply_noalloc(dims, 0.1, z, z, z, None) == gs.GS_ETOOLARGE
    assert gs.wilson_apply_noalloc((1, 8, 8, 8), 0.1, z, z, z, None) == gs.GS_EINVAL


def test_noalloc_refuses_undersized_or_mistyped_buffers():
    """The binding checks the buffer sizes and types the lattice needs before
    any pointer reaches the library (the library itself cannot see them)."""
    torch = torch_cuda()
    gs = lib()
    dims = (8, 8, 8, 8)
    V = li.volume(dims)
    U = torch.zeros(V * 36, dtype=torch.complex128, device="cuda:0")
    x = torch.zeros(V * 12, dtype=torch.complex128, device="cuda:0")
    for args in ((U[:-1], x, x.clone()), (U, x[:V], x.clone()), (U, x, x[:-12]),
                 (U, x.to(torch.complex64), x.clone())):
        with pytest.raises(gs.GschurError) as e:
            gs.wilson_apply_noalloc(dims, 0.1, *args)
        assert e.value.status == gs.GS_EINVAL
