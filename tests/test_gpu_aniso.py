"""The anisotropic workload's precision x polynomial sweep at a reduced size: every
configuration of Section 5.4 (FP64 GMRES with an FP64 or an FP32 polynomial, GMRES-IR with
FP32/FP16/BF16 storage) converges, and its solution agrees with the oracle's exact solve."""
import pytest

import gen
from oracle.direct import direct_solve

pytestmark = pytest.mark.gpu


def test_precision_polynomial_sweep_small():
    from paper_2109_01232_b300 import aniso_sweep
    p, b = gen.config_aniso_2d(side=200)
    p, rows = aniso_sweep.run(side=200, x_ref=direct_solve(p, b))
    assert len(rows) == 3 * 5
    for r in rows:
        assert r["status"] == "OK", r
        assert r["relres"] <= 1.0001e-10
        # the error against the exact solution is bounded by the residual times a modest
        # condition number estimate of this small problem
        assert r["err"] <= 1e-5, r
