"""Table 1 of the paper on synthetic fields (oracle).

Test infrastructure, like the rest of ``oracle/``; slow (minutes), not part
of the test suite.

Section 4 solves D x = f to 1e-8 at kappa = 1/6 (m0 = -1 with
D = (m0 + 4) - 1/2 H) on lattices at beta = 5.4, 5.7, 5.9 with BiCGStab,
plain and right-preconditioned by a 3-level V-cycle built on the Section 3
approximation (coarsest level inverted exactly, the D_rr solves of every level
by BiCGStab to 1e-2), with P_I^T for the first two couplings and P_II^T for
the third, and reports the average convergence rate R of both.

Stand-ins: the paper's ensembles are not available, so the fields are seeded
8^4 plaquette-action heatbath fields (``lattice_inputs.coupling_gauge``); "8^8"
is read as 8^4.  The condition number of the table's second row is read as
the 2-norm condition number of D (``spectra.condition_number``: Lanczos on
D^H D and on its inverse through one sparse LU of D).

    python -m oracle.table1          prints one JSON line per coupling
    python -m oracle.table1 --cond   adds the condition number of D and its
                                     eigenvalue of smallest real part
    python -m oracle.table1 --type1  also runs beta = 5.9 with P_I^T at both
                                     levels (the case the paper reports as not
                                     converging; 30 outer steps at most, the
                                     rest-set solves capped at 2000 steps)
    --kappa K (default 1/6, m0 = 1/(2K) - 4) and --beta B ... choose the
    hopping parameter and the couplings; --schur first uses the first-order
    coarse operator (D_rr's couplings ignored) in the V-cycle; --no-plain
    skips the unpreconditioned solve; --index I ... runs further stand-in
    fields of each coupling (other heatbath seeds).
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import dirac, krylov, permute, spectra, vcycle

__all__ = ["run", "run_field", "LEVELS", "PAPER"]

LEVELS = {
    5.4: [(permute.TYPE_I, 0, True), (permute.TYPE_I, 0, True)],
    5.7: [(permute.TYPE_I, 0, True), (permute.TYPE_I, 0, True)],
    5.9: [(permute.TYPE_II, 0, True), (permute.TYPE_II, 1, True)],
}


# Table 1's printed values per coupling: condition number, R of BiCGStab, R
# of BiCGStab preconditioned by the 3-level V-cycle.
PAPER = {5.4: {"condition": 57, "R_plain": 0.76, "R_preconditioned": 0.05},
         5.7: {"condition": 480, "R_plain": 0.83, "R_preconditioned": 0.16},
         5.9: {"condition": 905, "R_plain": 0.89, "R_preconditioned": 0.48}}


def run(beta, m0=-1.0, index=0, levels=None, **kw):
    """One Table 1 column on the stand-in field of coupling beta (``index``
    picks another heatbath seed); keywords as for ``run_field``."""
    import lattice_inputs as li
    dims, U = li.coupling_gauge(beta, index)
    out = {"beta": beta, "field_index": index, "plaquette": li.average_plaquette(U, dims),
           "paper": PAPER.get(beta)}
    out.update(run_field(U, dims, m0, LEVELS[beta] if levels is None else levels, **kw))
    return out


def run_field(U, dims, m0, levels, tol=1e-8, inner_tol=1e-2, maxiter=3000, seed_source=100,
              cond=False, plain=True, maxiter_pc=200, inner_maxiter=100000, schur="reusken"):
    """Section 4's comparison on one field: plain BiCGStab and BiCGStab with
    the V-cycle (levels: (ptype, mu, inverse) per coarsening) for D x = f, f a
    Gaussian source, each to tol; reports steps, R (geometric and arithmetic
    mean of the residual ratios) and the true residual of the returned x."""
    import lattice_inputs as li
    D = dirac.wilson_matrix(U, dims, m0).tocsr()
    f = li.gaussian_source(dims, seed_source).ravel()
    out = {"m0": m0, "dims": list(dims)}
    if cond:
        kappa, smin, smax = spectra.condition_number(D, tol=1e-6)
        ev = spectra.leftmost_eigenvalues(D, k=2, tol=1e-6)
        out["condition"] = {"kappa": kappa, "sigma_min": smin, "sigma_max": smax,
                            "leftmost_eigenvalue": [float(ev[0].real), float(abs(ev[0].imag))]}
    if plain:
        t0 = time.time()
        x, info = krylov.bicgstab(lambda v: D @ v, f, tol=tol, maxiter=maxiter)
        out["plain"] = {"iters": info["iters"], "converged": info["converged"],
                        "R": krylov.convergence_rate(info["history"]),
                        "R_arith": krylov.mean_ratio(info["history"]),
                        "residual": float(np.linalg.norm(D @ x - f) / np.linalg.norm(f)),
                        "history": [float(h) for h in info["history"]],
                        "seconds": time.time() - t0}
    t0 = time.time()
    vc = vcycle.VCycle(D, dims, levels, schur=schur, inner=inner_tol,
                       inner_maxiter=inner_maxiter)
    x, info = vcycle.preconditioned_bicgstab(D, f, vc, tol=tol, maxiter=maxiter_pc)
    out["preconditioned"] = {"levels": [list(map(int, lv)) for lv in levels], "schur": schur,
                             "iters": info["iters"], "converged": info["converged"], "R": info["R"],
                             "R_arith": krylov.mean_ratio(info["history"]),
                             "residual": float(np.linalg.norm(D @ x - f) / np.linalg.norm(f)),
                             "history": [float(h) for h in info["history"]],
                             "inner_solves": len(vc.inner_log),
                             "inner_steps_max": max((s for _, s, _ in vc.inner_log), default=0),
                             "inner_not_converged": sum(1 for *_, c in vc.inner_log if not c),
                             "seconds": time.time() - t0}
    return out


def _main(argv):
    import argparse
    ap = argparse.ArgumentParser(prog="python -m oracle.table1")
    ap.add_argument("--cond", action="store_true")
    ap.add_argument("--type1", action="store_true")
    ap.add_argument("--kappa", type=float, default=1.0 / 6.0)
    ap.add_argument("--beta", type=float, nargs="*", default=[5.4, 5.7, 5.9])
    ap.add_argument("--schur", default="reusken", choices=["reusken", "first"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--index", type=int, nargs="*", default=[0],
                    help="stand-in field indices per coupling (seeds differ)")
    a = ap.parse_args(argv)
    m0 = 1.0 / (2.0 * a.kappa) - 4.0
    for b in a.beta:
        for i in a.index:
            print(json.dumps(run(b, m0=m0, cond=a.cond, schur=a.schur, plain=not a.no_plain,
                                 index=i)), flush=True)
    if a.type1:
        print(json.dumps(run(5.9, m0=m0, levels=LEVELS[5.4], plain=False, maxiter_pc=30,
                             inner_maxiter=2000)), flush=True)


if __name__ == "__main__":
    import sys
    _main(sys.argv[1:])
