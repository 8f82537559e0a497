"""Plain FP64 CPU oracle for the gauged renormalisation-group step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library (``paper_0704_2341_gb300``); the two
agree only on conventions (site order, gamma basis, vector layout), which
each side writes out on its own.

Everything here is complex128 and written for clarity, not speed:

* ``dirac``   -- gamma matrices and the assembled sparse Wilson-Dirac matrix
                 (the operator the paper blocks; Section 1, Section 3);
* ``permute`` -- the Type I / Type II site permutations and their inverses
                 (Section 2, Fig. 1 and the list of four permutation types);
* ``schur``   -- the 2x2 partition, the Schur complement S_bb, its apply,
                 and the solve of D x = f through the block UL factorisation
                 (Section 1, the partition, Eq. for S_bb and the UL product);
* ``krylov``  -- textbook BiCGStab (van der Vorst 1992) and restarted
                 GMRES(m) (Saad & Schultz 1986), the solvers the paper uses
                 or the configuration asks for (Section 4);
* ``reusken`` -- the second-order Schur-complement approximation of
                 Section 3 (site-block diagonal d and row sums d~);
* ``vcycle``  -- the cyclic-reduction V-cycle preconditioner of Section 4
                 built from it, and BiCGStab preconditioned by it (R);
* ``spectra`` -- dense spectra of S, S~ and S~^-1 S (Figs. 2-4), and the
                 condition number and leftmost eigenvalues of a sparse D;
* ``table1``  -- the Section 4 experiment of Table 1 on seeded stand-in
                 fields (a script: ``python -m oracle.table1``).

Parity status of each function is listed in the module headers; every
function listed is pinned by a ``-m "not gpu"`` test except where a module
header says "parity unpinned".
"""
from . import dirac, permute, schur, krylov, net, reusken, vcycle  # noqa: F401
