"""ctypes binding of the gschur C ABI (include/gschur.h).

Argument marshalling only: every function here forwards to the entry point of
the same name in ``libgschur.so``; tensors are turned into device pointers,
options into the C structs.  There is no fallback: if the library is missing
the import fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgschur.so")

GS_OK, GS_EINVAL, GS_ENOMEM, GS_MAXITER, GS_BREAKDOWN, GS_NONFINITE, GS_TIMEOUT, \
    GS_ECUDA, GS_ENOGAUGE, GS_ETOOLARGE = range(10)
STATUS_NAMES = {0: "GS_OK", 1: "GS_EINVAL", 2: "GS_ENOMEM", 3: "GS_MAXITER",
                4: "GS_BREAKDOWN", 5: "GS_NONFINITE", 6: "GS_TIMEOUT", 7: "GS_ECUDA",
                8: "GS_ENOGAUGE", 9: "GS_ETOOLARGE"}
GS_TYPE_I, GS_TYPE_II = 1, 2
GS_F64, GS_F32, GS_BF16 = 0, 1, 2
GS_GMRES, GS_BICGSTAB = 0, 1
GS_INNER_BICGSTAB, GS_INNER_FGMRES_NET = 0, 1
GS_OPT_STENCIL_VARIANT, GS_OPT_INNER_KERNEL, GS_OPT_NET_KERNEL, GS_OPT_MULTI_BATCH, \
    GS_OPT_WAIT_LIMIT_US, GS_OPT_COOP_BLOCKS, GS_OPT_BATCH_LANES = 1, 2, 3, 4, 5, 6, 7
GS_PROF_STENCIL_F64, GS_PROF_STENCIL_F32, GS_PROF_STENCIL_BF16, GS_PROF_SOLVER_F64, \
    GS_PROF_SOLVER_LP = range(5)

# every symbol the header declares
EXPORTS = ("gs_create", "gs_destroy", "gs_set_gauge", "gs_default_opts", "wilson_apply",
           "permute_sites", "gs_get_permutation", "schur_apply", "schur_solve",
           "gs_last_error", "gs_version", "gs_profile", "gs_profile_read",
           "wilson_apply_noalloc", "gs_lowp_pack", "gs_lowp_unpack", "wilson_apply_lowp", "gs_set_option",
           "gs_get_option", "schur_solve_multi", "schur_solve_batched", "gs_lowp_pack_multi",
           "gs_lowp_unpack_multi", "wilson_apply_lowp_multi", "gs_solve_rr", "gs_net_create",
           "gs_net_destroy", "gs_net_set_weights", "gs_net_get", "gs_net_apply",
           "gs_net_train_step", "gs_set_net", "gs_profile_phases", "schur_apply_reusken",
           "gs_selftest_wait", "schur_apply_approx", "gs_vcycle_create", "gs_vcycle_destroy",
           "gs_vcycle_apply", "gs_vcycle_level", "gs_vcycle_operator_apply", "gs_solve_bicgstab",
           "gs_fp64_peak", "gs_profile_timeline", "gs_condition_number", "gs_leftmost_eigenvalues")


class gs_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("restart", ctypes.c_int), ("outer_solver", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("inner_max_iter", ctypes.c_int),
                ("inner_prec", ctypes.c_int), ("check_every", ctypes.c_int),
                ("lowp_tol", ctypes.c_double), ("inner_relax", ctypes.c_int),
                ("relax_cap", ctypes.c_double), ("inner_solver", ctypes.c_int),
                ("inner_restart", ctypes.c_int)]


class gs_solve_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("inner_solves", ctypes.c_int), ("inner_iters", ctypes.c_longlong),
                ("inner_max_seen", ctypes.c_int), ("outer_residual", ctypes.c_double),
                ("true_residual", ctypes.c_double), ("inner_residual", ctypes.c_double),
                ("stencil_sites", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("lowp_cycles", ctypes.c_longlong), ("lowp_fallbacks", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gs_kernel_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("sites", ctypes.c_longlong), ("hops", ctypes.c_longlong),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libgschur.so is not built (expected at %s); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
    sig = {
        "gs_create": (i32, [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ctypes.c_double, vp]),
        "gs_destroy": (i32, [vp]),
        "gs_set_gauge": (i32, [vp, vp]),
        "gs_default_opts": (None, [ctypes.POINTER(gs_solve_opts)]),
        "wilson_apply": (i32, [vp, vp, vp]),
        "permute_sites": (i32, [vp, i32, i32, i32, i32, vp, vp, i64p]),
        "gs_get_permutation": (i32, [vp, i32, i32, i32, vp, i64p]),
        "schur_apply": (i32, [vp, i32, i32, i32, vp, vp, ctypes.POINTER(gs_solve_opts),
                              ctypes.POINTER(gs_solve_stats)]),
        "schur_solve": (i32, [vp, i32, i32, i32, vp, vp, ctypes.POINTER(gs_solve_opts),
                              ctypes.POINTER(gs_solve_stats)]),
        "gs_last_error": (ctypes.c_char_p, [vp]),
        "gs_version": (ctypes.c_char_p, []),
        "gs_profile": (i32, [vp, i32]),
        "wilson_apply_noalloc": (i32, [ctypes.POINTER(ctypes.c_int), ctypes.c_double, vp, vp,
                                       vp, vp]),
        "gs_profile_read": (i32, [vp, i32, ctypes.POINTER(gs_kernel_profile)]),
        "gs_lowp_pack": (i32, [vp, i32, i32, i32, i32, vp, vp]),
        "gs_set_option": (i32, [vp, i32, i32]),
        "gs_solve_rr": (i32, [vp, i32, i32, i32, vp, vp, ctypes.POINTER(gs_solve_opts),
                              ctypes.POINTER(gs_solve_stats)]),
        "gs_net_create": (i32, [ctypes.POINTER(vp), i32]),
        "gs_net_destroy": (i32, [vp]),
        "gs_net_set_weights": (i32, [vp, i32, vp]),
        "gs_net_get": (i32, [vp, i32, i32, vp]),
        "gs_net_apply": (i32, [vp, vp, i32, i32, i32, vp, vp]),
        "gs_net_train_step": (i32, [vp, vp, i32, i32, i32, i32, vp, vp, ctypes.c_float, i32,
                                    ctypes.POINTER(ctypes.c_float)]),
        "gs_set_net": (i32, [vp, vp]),
        "gs_profile_phases": (i32, [vp, ctypes.POINTER(ctypes.c_double), i32]),
        "schur_apply_reusken": (i32, [vp, i32, i32, i32, vp, vp]),
        "gs_selftest_wait": (i32, [vp, i32]),
        "schur_apply_approx": (i32, [vp, i32, i32, i32, i32, vp, vp]),
        "gs_vcycle_create": (i32, [vp, i32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int), i32, ctypes.c_double, i32,
                                   ctypes.POINTER(vp)]),
        "gs_vcycle_destroy": (i32, [vp]),
        "gs_fp64_peak": (i32, [vp, ctypes.POINTER(ctypes.c_double)]),
        "gs_condition_number": (i32, [vp, vp, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int)]),
        "gs_leftmost_eigenvalues": (i32, [vp, vp, i32, i32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
        "gs_profile_timeline": (i32, [vp, i32, ctypes.POINTER(ctypes.c_double), i32,
                                      ctypes.POINTER(ctypes.c_int)]),
        "gs_vcycle_apply": (i32, [vp, vp, vp, ctypes.POINTER(gs_solve_stats)]),
        "gs_vcycle_level": (i32, [vp, i32, ctypes.POINTER(ctypes.c_int), i64p, i64p,
                                  ctypes.POINTER(ctypes.c_int)]),
        "gs_vcycle_operator_apply": (i32, [vp, i32, vp, vp]),
        "gs_solve_bicgstab": (i32, [vp, vp, vp, vp, ctypes.c_double, i32, ctypes.POINTER(gs_solve_stats),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    i32]),
        "schur_solve_multi": (i32, [vp, i32, i32, i32, i32, vp, vp, ctypes.POINTER(gs_solve_opts),
                                    ctypes.POINTER(gs_solve_stats)]),
        "schur_solve_batched": (i32, [i32, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp),
                                      ctypes.POINTER(vp), ctypes.POINTER(gs_solve_opts),
                                      ctypes.POINTER(gs_solve_stats)]),
        "gs_lowp_pack_multi": (i32, [vp, i32, i32, i32, i32, i32, vp, vp]),
        "gs_lowp_unpack_multi": (i32, [vp, i32, i32, i32, i32, i32, vp, vp]),
        "wilson_apply_lowp_multi": (i32, [vp, i32, i32, i32, i32, i32, vp, vp]),
        "gs_get_option": (i32, [vp, i32, ctypes.POINTER(ctypes.c_int)]),
        "gs_lowp_unpack": (i32, [vp, i32, i32, i32, i32, vp, vp]),
        "wilson_apply_lowp": (i32, [vp, i32, i32, i32, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


class GschurError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(t):
    """Device pointer of a tensor (checked: CUDA, contiguous) or an int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _need(t, nbytes, what):
    """Refuse a tensor smaller than the nbytes the call reads or writes
    (GS_EINVAL), before any device access; raw integer pointers are the
    caller's responsibility."""
    if t is None or isinstance(t, int):
        return
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise GschurError(GS_EINVAL, "%s holds %d bytes, the call needs %d" % (what, have, nbytes))


SPINOR_BYTES = 192          # complex128 [4][3] per site
LINK_BYTES = 4 * 9 * 16     # complex128 [4][3][3] per site


def _check(ctx, status, allow=(GS_OK,)):
    if status not in allow:
        raise GschurError(status, gs_last_error(ctx))
    return status


def gs_version():
    return lib.gs_version().decode()


def gs_last_error(ctx):
    return lib.gs_last_error(ctx).decode()


def gs_default_opts(**overrides):
    o = gs_solve_opts()
    lib.gs_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def gs_create(dims, m0, stream=None):
    """Returns the opaque context handle (an int).  stream: a cudaStream_t as int or None."""
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(L) for L in dims])
    st = lib.gs_create(ctypes.byref(h), d, float(m0), stream)
    if st != GS_OK:
        raise GschurError(st, "gs_create failed")
    return h.value


def gs_destroy(ctx):
    return lib.gs_destroy(ctx)


def gs_set_gauge(ctx, U):
    return _check(ctx, lib.gs_set_gauge(ctx, _ptr(U)))


def wilson_apply(ctx, x, y):
    return _check(ctx, lib.wilson_apply(ctx, _ptr(x), _ptr(y)))


def permute_sites(ctx, ptype, dir, inverse, transpose, x, y):
    nb = ctypes.c_int64()
    _check(ctx, lib.permute_sites(ctx, ptype, dir, int(bool(inverse)), int(bool(transpose)),
                                  _ptr(x), _ptr(y), ctypes.byref(nb)))
    return nb.value


def gs_get_permutation(ctx, ptype, dir, inverse, perm):
    nb = ctypes.c_int64()
    _check(ctx, lib.gs_get_permutation(ctx, ptype, dir, int(bool(inverse)), _ptr(perm),
                                       ctypes.byref(nb)))
    return nb.value


def schur_apply(ctx, ptype, dir, inverse, xb, yb, opts=None, allow=(GS_OK,)):
    o = opts if opts is not None else gs_default_opts()
    st = gs_solve_stats()
    _check(ctx, lib.schur_apply(ctx, ptype, dir, int(bool(inverse)), _ptr(xb), _ptr(yb),
                                ctypes.byref(o), ctypes.byref(st)), allow)
    return st


def schur_solve(ctx, ptype, dir, inverse, f, x, opts=None, allow=(GS_OK,)):
    o = opts if opts is not None else gs_default_opts()
    st = gs_solve_stats()
    _check(ctx, lib.schur_solve(ctx, ptype, dir, int(bool(inverse)), _ptr(f), _ptr(x),
                                ctypes.byref(o), ctypes.byref(st)), allow)
    return st


NOALLOC_MAX_SITES = 8192    # the static scratch of wilson_apply_noalloc


def _need_c128(t, what):
    """Refuse a tensor that is not complex128 (GS_EINVAL)."""
    if t is None or isinstance(t, int):
        return
    import torch
    if t.dtype != torch.complex128:
        raise GschurError(GS_EINVAL, "%s must be complex128, not %s" % (what, t.dtype))


def wilson_apply_noalloc(dims, m0, U, x, y, stream=None):
    """y = D x without a context and without allocating.  Returns the status;
    extents the library rejects come back as GS_EINVAL / GS_ETOOLARGE, and
    tensors that are smaller than the lattice needs or not complex128 raise
    GschurError(GS_EINVAL) before any pointer reaches the library."""
    d = [int(L) for L in dims]
    if len(d) != 4 or min(d) < 2:
        return GS_EINVAL
    V = 1
    for L in d:
        if L > NOALLOC_MAX_SITES // V:
            return GS_ETOOLARGE
        V *= L
    for t, nbytes, what in ((U, V * LINK_BYTES, "U"), (x, V * SPINOR_BYTES, "x"),
                            (y, V * SPINOR_BYTES, "y")):
        _need_c128(t, what)
        _need(t, nbytes, what)
    return lib.wilson_apply_noalloc((ctypes.c_int * 4)(*d), float(m0), _ptr(U), _ptr(x),
                                    _ptr(y), stream)


def gs_profile(ctx, enable):
    return _check(ctx, lib.gs_profile(ctx, int(bool(enable))))


def schur_apply_reusken(ctx, ptype, dir, inverse, xb, yb):
    return _check(ctx, lib.schur_apply_reusken(ctx, ptype, dir, int(bool(inverse)), _ptr(xb), _ptr(yb)))


def schur_apply_approx(ctx, ptype, dir, inverse, order, xb, yb):
    return _check(ctx, lib.schur_apply_approx(ctx, ptype, dir, int(bool(inverse)), int(order),
                                              _ptr(xb), _ptr(yb)))


def gs_selftest_wait(ctx, which):
    """Run a bounded device wait that is meant to run out; returns the status
    (GS_TIMEOUT is the intended outcome)."""
    return lib.gs_selftest_wait(ctx, int(which))


def gs_profile_phases(ctx):
    """Cycles per phase of the persistent FP64 solver (block 0) while profiling was on."""
    out = (ctypes.c_double * 15)()
    _check(ctx, lib.gs_profile_phases(ctx, out, 15))
    return list(out)


def gs_profile_read(ctx, prec=GS_F64):
    out = gs_kernel_profile()
    _check(ctx, lib.gs_profile_read(ctx, prec, ctypes.byref(out)))
    return out


def schur_solve_multi(ctx, ptype, dir, inverse, nrhs, f, x, opts=None, allow=(GS_OK,)):
    o = opts if opts is not None else gs_default_opts(inner_prec=GS_F32)
    st = gs_solve_stats()
    _check(ctx, lib.schur_solve_multi(ctx, ptype, dir, int(bool(inverse)), nrhs, _ptr(f), _ptr(x),
                                      ctypes.byref(o), ctypes.byref(st)), allow)
    return st


def schur_solve_batched(problems, opts=None):
    """problems: list of dicts with keys ctx (handle), type, dir, inverse, nrhs, f, x.
    Returns (status, [gs_solve_stats])."""
    n = len(problems)
    o = opts if opts is not None else gs_default_opts(inner_prec=GS_F32)
    VP = ctypes.c_void_p
    IA = ctypes.c_int * n
    ctxs = (VP * n)(*[p["ctx"] for p in problems])
    ty = IA(*[p["type"] for p in problems])
    di = IA(*[p.get("dir", 0) for p in problems])
    iv = IA(*[int(bool(p.get("inverse", 0))) for p in problems])
    nr = IA(*[p["nrhs"] for p in problems])
    fs = (VP * n)(*[_ptr(p["f"]) for p in problems])
    xs = (VP * n)(*[_ptr(p["x"]) for p in problems])
    sts = (gs_solve_stats * n)()
    status = lib.schur_solve_batched(n, ctxs, ty, di, iv, nr, fs, xs, ctypes.byref(o), sts)
    return status, list(sts)


def gs_lowp_pack_multi(ctx, ptype, dir, inverse, prec, nrhs, x, x_lp):
    return _check(ctx, lib.gs_lowp_pack_multi(ctx, ptype, dir, int(bool(inverse)), prec, nrhs,
                                              _ptr(x), _ptr(x_lp)))


def gs_lowp_unpack_multi(ctx, ptype, dir, inverse, prec, nrhs, x_lp, x):
    return _check(ctx, lib.gs_lowp_unpack_multi(ctx, ptype, dir, int(bool(inverse)), prec, nrhs,
                                                _ptr(x_lp), _ptr(x)))


def wilson_apply_lowp_multi(ctx, ptype, dir, inverse, prec, nrhs, x_lp, y_lp):
    return _check(ctx, lib.wilson_apply_lowp_multi(ctx, ptype, dir, int(bool(inverse)), prec, nrhs,
                                                   _ptr(x_lp), _ptr(y_lp)))


def gs_solve_rr(ctx, ptype, dir, inverse, t, z, opts=None, allow=(GS_OK,)):
    o = opts if opts is not None else gs_default_opts()
    st = gs_solve_stats()
    _check(ctx, lib.gs_solve_rr(ctx, ptype, dir, int(bool(inverse)), _ptr(t), _ptr(z),
                                ctypes.byref(o), ctypes.byref(st)), allow)
    return st


class Net:
    """Owns one gs_net (weights as numpy complex64 [9][4 C_out][4 C_in] per layer)."""

    def __init__(self, channels):
        h = ctypes.c_void_p()
        st = lib.gs_net_create(ctypes.byref(h), int(channels))
        if st != GS_OK:
            raise GschurError(st, "gs_net_create failed")
        self.handle = h.value
        self.channels = int(channels)

    def shapes(self):
        C = self.channels
        return [(9, 4 * C, 4), (9, 4 * C, 4 * C), (9, 4, 4 * C)]

    def set_weights(self, layer, w):
        import numpy as np
        a = np.ascontiguousarray(w, dtype=np.complex64)
        if a.shape != self.shapes()[layer]:
            raise ValueError("weights of layer %d must have shape %s" % (layer, self.shapes()[layer]))
        st = lib.gs_net_set_weights(self.handle, layer, a.ctypes.data)
        if st != GS_OK:
            raise GschurError(st, "gs_net_set_weights failed")

    def get(self, what, layer):
        import numpy as np
        a = np.empty(self.shapes()[layer], dtype=np.complex64)
        st = lib.gs_net_get(self.handle, what, layer, a.ctypes.data)
        if st != GS_OK:
            raise GschurError(st, "gs_net_get failed")
        return a

    def apply(self, ctx, ptype, dir, inverse, t, y):
        return _check(ctx, lib.gs_net_apply(ctx, self.handle, ptype, dir, int(bool(inverse)),
                                            _ptr(t), _ptr(y)))

    def train_step(self, ctx, ptype, dir, inverse, batch, t, z, lr, update=True):
        loss = ctypes.c_float()
        _check(ctx, lib.gs_net_train_step(ctx, self.handle, ptype, dir, int(bool(inverse)), batch,
                                          _ptr(t), _ptr(z), float(lr), int(bool(update)),
                                          ctypes.byref(loss)))
        return loss.value

    def close(self):
        if self.handle:
            lib.gs_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_set_net(ctx, net):
    return _check(ctx, lib.gs_set_net(ctx, net.handle if net is not None else None))


def gs_set_option(ctx, option, value):
    return _check(ctx, lib.gs_set_option(ctx, option, value))


def gs_get_option(ctx, option):
    v = ctypes.c_int()
    _check(ctx, lib.gs_get_option(ctx, option, ctypes.byref(v)))
    return v.value


def lowp_bytes(n_sites, prec):
    """Size of a low-precision vector of n sites."""
    return n_sites * (48 if prec == GS_BF16 else 96)


def gs_lowp_pack(ctx, ptype, dir, inverse, prec, x, x_lp):
    return _check(ctx, lib.gs_lowp_pack(ctx, ptype, dir, int(bool(inverse)), prec, _ptr(x),
                                        _ptr(x_lp)))


def gs_lowp_unpack(ctx, ptype, dir, inverse, prec, x_lp, x):
    return _check(ctx, lib.gs_lowp_unpack(ctx, ptype, dir, int(bool(inverse)), prec, _ptr(x_lp),
                                          _ptr(x)))


def wilson_apply_lowp(ctx, ptype, dir, inverse, prec, x_lp, y_lp):
    return _check(ctx, lib.wilson_apply_lowp(ctx, ptype, dir, int(bool(inverse)), prec,
                                             _ptr(x_lp), _ptr(y_lp)))


class VCycle:
    """Owns one gs_vcycle of a context (Section 4's V-cycle preconditioner).
    levels: one (type, dir, inverse) per coarsening step."""

    def __init__(self, ctx, levels, order=2, rest_tol=1e-2, rest_max_iter=100000):
        n = len(levels)
        IA = ctypes.c_int * max(n, 1)
        ty = IA(*[int(l[0]) for l in levels])
        di = IA(*[int(l[1]) for l in levels])
        iv = IA(*[int(bool(l[2])) for l in levels])
        h = ctypes.c_void_p()
        self.ctx = ctx
        self.handle = None
        _check(ctx.handle, lib.gs_vcycle_create(ctx.handle, n, ty, di, iv, int(order),
                                                float(rest_tol), int(rest_max_iter),
                                                ctypes.byref(h)))
        self.handle = h.value
        self.nlevels = n + 1

    def apply(self, f, x):
        self.ctx._need_lattice(f=f, x=x)
        st = gs_solve_stats()
        _check(self.ctx.handle, lib.gs_vcycle_apply(self.handle, _ptr(f), _ptr(x), ctypes.byref(st)))
        return st

    def level(self, l):
        d = (ctypes.c_int * 4)()
        n, b, cc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        st = lib.gs_vcycle_level(self.handle, int(l), d, ctypes.byref(n), ctypes.byref(b),
                                 ctypes.byref(cc))
        if st != GS_OK:
            raise GschurError(st, "gs_vcycle_level failed")
        return {"dims": tuple(d), "sites": n.value, "blocks": b.value, "colours": cc.value}

    def operator_apply(self, l, x, y):
        sites = self.level(l)["sites"]
        _need(x, sites * SPINOR_BYTES, "x")
        _need(y, sites * SPINOR_BYTES, "y")
        return _check(self.ctx.handle, lib.gs_vcycle_operator_apply(self.handle, int(l), _ptr(x),
                                                                    _ptr(y)))

    def close(self):
        if self.handle:
            lib.gs_vcycle_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_solve_bicgstab(ctx, vc, f, x, tol=1e-8, max_iter=3000, history_cap=4096,
                      allow=(GS_OK,)):
    """BiCGStab on D x = f (right-preconditioned by the V-cycle vc, or plain if
    None).  Returns (stats, R, residual history)."""
    st = gs_solve_stats()
    R = ctypes.c_double()
    hist = (ctypes.c_double * history_cap)()
    _check(ctx, lib.gs_solve_bicgstab(ctx, vc.handle if vc is not None else None, _ptr(f), _ptr(x),
                                      float(tol), int(max_iter), ctypes.byref(st), ctypes.byref(R),
                                      hist, int(history_cap)), allow)
    return st, R.value, [h for h in hist if h >= 0.0]


class Context:
    """Owns one gs_ctx; methods forward to the functions above."""

    def __init__(self, dims, m0, stream=None):
        self.dims = tuple(int(L) for L in dims)
        self.m0 = float(m0)
        self.volume = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.handle = gs_create(self.dims, self.m0, stream)

    def close(self):
        if self.handle:
            gs_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _need_lattice(self, nrhs=1, **tensors):
        for name, t in tensors.items():
            _need(t, nrhs * self.volume * SPINOR_BYTES, name)

    def set_gauge(self, U):
        _need(U, self.volume * LINK_BYTES, "U")
        return gs_set_gauge(self.handle, U)

    def wilson_apply(self, x, y):
        self._need_lattice(x=x, y=y)
        return wilson_apply(self.handle, x, y)

    def permute_sites(self, ptype, dir, inverse, transpose, x, y):
        self._need_lattice(x=x, y=y)
        return permute_sites(self.handle, ptype, dir, inverse, transpose, x, y)

    def get_permutation(self, ptype, dir, inverse, perm):
        return gs_get_permutation(self.handle, ptype, dir, inverse, perm)

    def schur_apply(self, ptype, dir, inverse, xb, yb, opts=None, allow=(GS_OK,)):
        return schur_apply(self.handle, ptype, dir, inverse, xb, yb, opts, allow)

    def schur_solve(self, ptype, dir, inverse, f, x, opts=None, allow=(GS_OK,)):
        self._need_lattice(f=f, x=x)
        return schur_solve(self.handle, ptype, dir, inverse, f, x, opts, allow)

    def schur_solve_multi(self, ptype, dir, inverse, nrhs, f, x, opts=None, allow=(GS_OK,)):
        if 1 <= int(nrhs) <= 32:            # other counts: the library reports GS_EINVAL
            self._need_lattice(int(nrhs), f=f, x=x)
        return schur_solve_multi(self.handle, ptype, dir, inverse, nrhs, f, x, opts, allow)

    def lowp_pack_multi(self, ptype, dir, inverse, prec, nrhs, x, x_lp):
        return gs_lowp_pack_multi(self.handle, ptype, dir, inverse, prec, nrhs, x, x_lp)

    def lowp_unpack_multi(self, ptype, dir, inverse, prec, nrhs, x_lp, x):
        return gs_lowp_unpack_multi(self.handle, ptype, dir, inverse, prec, nrhs, x_lp, x)

    def wilson_apply_lowp_multi(self, ptype, dir, inverse, prec, nrhs, x_lp, y_lp):
        return wilson_apply_lowp_multi(self.handle, ptype, dir, inverse, prec, nrhs, x_lp, y_lp)

    def profile(self, enable):
        return gs_profile(self.handle, enable)

    def profile_read(self, prec=GS_F64):
        return gs_profile_read(self.handle, prec)

    def profile_phases(self):
        return gs_profile_phases(self.handle)

    def profile_timeline(self, family):
        """[(start_ms, end_ms)] of the family's timed launches, on the device's
        common time origin."""
        n = ctypes.c_int()
        _check(self.handle, lib.gs_profile_timeline(self.handle, int(family), None, 0, ctypes.byref(n)))
        buf = (ctypes.c_double * max(2 * n.value, 1))()
        _check(self.handle, lib.gs_profile_timeline(self.handle, int(family), buf, 2 * n.value,
                                                    ctypes.byref(n)))
        return [(buf[2 * i], buf[2 * i + 1]) for i in range(n.value)]

    def selftest_wait(self, which):
        return gs_selftest_wait(self.handle, which)

    def fp64_peak(self):
        """Measured FP64 TFLOP/s of this GPU (gs_fp64_peak)."""
        v = ctypes.c_double()
        _check(self.handle, lib.gs_fp64_peak(self.handle, ctypes.byref(v)))
        return v.value

    def condition_number(self, start, max_steps=20000, tol=1e-6, allow=(GS_OK,)):
        """(kappa, sigma_min, sigma_max, steps) of D by Lanczos on D^H D."""
        self._need_lattice(start=start)
        k, lo, hi, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(self.handle, lib.gs_condition_number(self.handle, _ptr(start), int(max_steps), float(tol),
                                                    ctypes.byref(k), ctypes.byref(lo), ctypes.byref(hi),
                                                    ctypes.byref(n)), allow)
        return k.value, lo.value, hi.value, n.value

    def leftmost_eigenvalues(self, start, m, k=6):
        """The k eigenvalues of D with the smallest real part from m Arnoldi steps."""
        self._need_lattice(start=start)
        re, im, n = (ctypes.c_double * k)(), (ctypes.c_double * k)(), ctypes.c_int()
        _check(self.handle, lib.gs_leftmost_eigenvalues(self.handle, _ptr(start), int(m), int(k), re, im,
                                                        ctypes.byref(n)))
        return [complex(re[i], im[i]) for i in range(n.value)]

    def solve_bicgstab(self, vc, f, x, tol=1e-8, max_iter=3000, allow=(GS_OK,)):
        self._need_lattice(f=f, x=x)
        return gs_solve_bicgstab(self.handle, vc, f, x, tol, max_iter, allow=allow)

    def schur_apply_reusken(self, ptype, dir, inverse, xb, yb):
        return schur_apply_reusken(self.handle, ptype, dir, inverse, xb, yb)

    def schur_apply_approx(self, ptype, dir, inverse, order, xb, yb):
        return schur_apply_approx(self.handle, ptype, dir, inverse, order, xb, yb)

    def solve_rr(self, ptype, dir, inverse, t, z, opts=None, allow=(GS_OK,)):
        return gs_solve_rr(self.handle, ptype, dir, inverse, t, z, opts, allow)

    def set_net(self, net):
        return gs_set_net(self.handle, net)

    def set_option(self, option, value):
        return gs_set_option(self.handle, option, value)

    def get_option(self, option):
        return gs_get_option(self.handle, option)

    def lowp_pack(self, ptype, dir, inverse, prec, x, x_lp):
        return gs_lowp_pack(self.handle, ptype, dir, inverse, prec, x, x_lp)

    def lowp_unpack(self, ptype, dir, inverse, prec, x_lp, x):
        return gs_lowp_unpack(self.handle, ptype, dir, inverse, prec, x_lp, x)

    def wilson_apply_lowp(self, ptype, dir, inverse, prec, x_lp, y_lp):
        return wilson_apply_lowp(self.handle, ptype, dir, inverse, prec, x_lp, y_lp)
