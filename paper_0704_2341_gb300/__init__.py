"""GB300 (sm_103a) library for the gauged renormalisation-group step of
lattice Wilson fermions: the Schur complement S_bb = D_bb - D_br D_rr^-1 D_rb
under the Type I / Type II site permutations and their inverses.

The compute path is the CUDA library ``libgschur.so`` (C ABI in
``include/gschur.h``); this package is its ctypes binding.  PyTorch is used by
callers only for device memory and streams.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import (Context, GschurError, EXPORTS, LIB_PATH, Net, VCycle, gs_default_opts,  # noqa: F401
                       gs_solve_opts, gs_solve_stats, lib)

__all__ = ["Context", "GschurError", "gs_create", "gs_destroy", "gs_set_gauge",
           "gs_default_opts", "wilson_apply", "permute_sites", "gs_get_permutation",
           "schur_apply", "schur_solve", "gs_last_error", "gs_version", "gs_profile",
           "gs_profile_read", "wilson_apply_noalloc", "GS_ETOOLARGE", "gs_lowp_pack",
           "gs_lowp_unpack", "wilson_apply_lowp", "lowp_bytes", "gs_set_option",
           "gs_get_option", "GS_OPT_STENCIL_VARIANT", "GS_OPT_INNER_KERNEL", "GS_OPT_NET_KERNEL", "GS_PROF_STENCIL_F64",
           "GS_PROF_STENCIL_F32", "GS_PROF_STENCIL_BF16", "GS_PROF_SOLVER_F64", "GS_PROF_SOLVER_LP",
           "schur_solve_multi", "schur_solve_batched", "gs_lowp_pack_multi", "gs_lowp_unpack_multi",
           "wilson_apply_lowp_multi", "gs_solve_rr", "Net", "gs_set_net", "GS_INNER_BICGSTAB",
           "GS_INNER_FGMRES_NET",
           "GS_TYPE_I", "GS_TYPE_II", "GS_F64", "GS_F32", "GS_BF16", "GS_GMRES",
           "GS_BICGSTAB", "GS_OK", "GS_MAXITER", "GS_BREAKDOWN", "STATUS_NAMES",
           "schur_apply_reusken", "GS_OPT_MULTI_BATCH", "GS_OPT_WAIT_LIMIT_US", "GS_OPT_COOP_BLOCKS", "GS_OPT_BATCH_LANES",
           "gs_selftest_wait", "schur_apply_approx", "VCycle", "gs_solve_bicgstab"]
