"""The Table 1 driver (Section 4's experiment) on a small field: both solves
reach the tolerance in the true residual, the V-cycle needs fewer steps and
a smaller average convergence rate, and the reported R values follow their
definitions (geometric mean never above the arithmetic one)."""
import numpy as np

import lattice_inputs as li
from oracle import permute, table1


def test_run_field_on_a_small_heatbath_field():
    dims = (4, 4, 4, 4)
    U = li.heatbath_gauge(dims, 5.4, 20, 3)
    out = table1.run_field(U, dims, -0.6, [(permute.TYPE_I, 0, True)] * 2, inner_tol=1e-2,
                           maxiter=2000, maxiter_pc=100)
    p, q = out["plain"], out["preconditioned"]
    assert p["converged"] and q["converged"]
    assert p["residual"] <= 2e-8 and q["residual"] <= 1e-7
    assert q["iters"] < p["iters"] and q["R"] < p["R"] < 1.0
    for r in (p, q):
        assert 0.0 < r["R"] <= r["R_arith"] + 1e-15
    assert q["inner_solves"] > 0 and q["inner_not_converged"] == 0
    assert out["dims"] == list(dims) and np.isfinite(q["seconds"])
    assert set(table1.LEVELS) == {5.4, 5.7, 5.9}
