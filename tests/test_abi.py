"""CPU checks of the C ABI: the library loads and exports every declared symbol;
the product package does not reach the oracle and the oracle does not reach
the product package."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gschur.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(\w+)\s*\([^;{]*\)\s*;", src)
    return sorted(set(n for n in names if n not in ("if", "while", "for", "sizeof")))


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    import paper_0704_2341_gb300 as gs
    lib = ctypes.CDLL(gs.LIB_PATH)
    decl = _declared()
    assert len(decl) >= 11
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) == set(gs.EXPORTS)
    assert gs.gs_version().startswith("gschur")


def test_calls_without_gpu_fail_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_0704_2341_gb300 as gs
    with pytest.raises(gs.GschurError):
        gs.gs_create((4, 4, 4, 4), 0.1)
    o = gs.gs_default_opts()
    assert o.tol == 1e-10 and o.restart == 30 and o.inner_tol == 1e-12
    assert o.inner_relax == 1 and o.relax_cap == 1e-4


def test_oracle_and_product_are_independent():
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_0704_2341_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b\s*(import|\.)|from\s+oracle|import\s+oracle", txt), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"(from|import)\s+paper_0704_2341_gb300|libgschur", txt), f


def test_context_refuses_short_buffers_before_any_device_access():
    """The binding checks every full-lattice buffer against the context's
    volume (GS_EINVAL) before it forms a pointer, so a short tensor can never
    reach a kernel; CPU tensors of the right size then fail at the pointer
    check.  A context object without a device handle is enough for both."""
    import torch
    import paper_0704_2341_gb300 as gs
    ctx = object.__new__(gs.Context)
    ctx.dims, ctx.m0, ctx.handle = (4, 4, 2, 2), 0.1, None
    ctx.volume = 64
    short = torch.zeros(64 * 12 - 1, dtype=torch.complex128)
    full = torch.zeros(64, 4, 3, dtype=torch.complex128)
    for call in (lambda: ctx.wilson_apply(short, full), lambda: ctx.wilson_apply(full, short),
                 lambda: ctx.permute_sites(1, 0, 0, 0, full, short),
                 lambda: ctx.schur_solve(1, 0, 0, short, full),
                 lambda: ctx.schur_solve_multi(1, 0, 0, 2, full, full),
                 lambda: ctx.set_gauge(torch.zeros(64, 4, 3, 2, dtype=torch.complex128))):
        with pytest.raises(gs.GschurError) as e:
            call()
        assert e.value.status == gs.GS_EINVAL
    with pytest.raises(ValueError):                     # right size, but not on a GPU
        ctx.wilson_apply(full, full.view(torch.float64))
    with pytest.raises(ValueError):
        ctx.set_gauge(torch.zeros(64, 4, 3, 3, dtype=torch.complex128))


def test_argument_checks_come_before_any_cuda_call():
    """gs_create and wilson_apply_noalloc validate their arguments on the host
    first: bad extents, a non-finite mass or a lattice past the index range
    give GS_EINVAL, a lattice past the no-allocation scratch GS_ETOOLARGE,
    all without a device; well-formed arguments then reach CUDA and, with no
    GPU, give GS_ECUDA."""
    import ctypes as ct
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_0704_2341_gb300 as gs
    lib = gs._binding.lib

    def create(dims, m0):
        h = ct.c_void_p()
        return lib.gs_create(ct.byref(h), (ct.c_int * 4)(*dims), ct.c_double(m0), None)

    assert create((1, 4, 4, 4), 0.1) == gs.GS_EINVAL
    assert create((4, 4, 0, 4), 0.1) == gs.GS_EINVAL
    assert create((4, 4, 4, 4), float("nan")) == gs.GS_EINVAL
    assert create((1024, 1024, 64, 64), 0.1) == gs.GS_EINVAL      # V * 12 >= 2^31
    assert create((4, 4, 4, 4), 0.1) == gs._binding.GS_ECUDA
    fake = 256                                   # never dereferenced: rejected first
    assert gs.wilson_apply_noalloc((4, 4, 1, 4), 0.1, fake, fake, fake) == gs.GS_EINVAL
    assert gs.wilson_apply_noalloc((4, 4, 4, 4), float("inf"), fake, fake, fake) == gs.GS_EINVAL
    assert gs.wilson_apply_noalloc((16, 16, 16, 16), 0.1, fake, fake, fake) == \
        gs._binding.GS_ETOOLARGE
    # extents whose product overflows 64 bits: each factor is bounded before
    # it multiplies, so the library (called directly, past the binding's own
    # check) still refuses them
    big = (ct.c_int * 4)(*([2 ** 31 - 1] * 4))
    assert lib.wilson_apply_noalloc(big, ct.c_double(0.1), fake, fake, fake, None) == \
        gs._binding.GS_ETOOLARGE
    assert create((2 ** 31 - 1,) * 4, 0.1) == gs.GS_EINVAL
    assert create((2 ** 16, 2 ** 16, 2 ** 16, 2 ** 16), 0.1) == gs.GS_EINVAL
    assert gs.gs_last_error(None) == "null context"
