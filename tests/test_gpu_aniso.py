"""The anisotropic workload's precision x polynomial sweep at a reduced size: every
combination converges, and its solution agrees with the FP64 solution."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_precision_polynomial_sweep_small():
    from paper_2109_01232_b300 import aniso_sweep
    p, rows = aniso_sweep.run(side=200)
    assert len(rows) == 1 + 3 * 4
    for r in rows:
        assert r["status"] == "OK", r
        assert r["relres"] <= 1.0001e-10 or r["solver"].startswith("FP64 GMRES (reference")
        # the error against the reference is bounded by the residual times a modest condition
        # number estimate of this small problem
        assert r["err"] <= 1e-5, r
