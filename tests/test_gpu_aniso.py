"""The anisotropic workload's precision x polynomial sweep at a reduced size: every
configuration of Section 5.4 (FP64 GMRES with an FP64 or an FP32 polynomial, GMRES-IR with
FP32/FP16/BF16 storage) converges, and its solution agrees with the oracle's exact solve."""
import os

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


REF = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "aniso2000_reference.npy")


@pytest.mark.skipif(not os.path.exists(REF),
                    reason="the oracle's exact 2000^2 solve is not recorded here "
                           "(python -m oracle.record_aniso_reference)")
def test_full_size_degree_40_against_the_exact_solve():
    """Section 5.4's configuration at full size (2000^2, 4M rows, polynomial degree 40): FP64
    GMRES with the FP64 polynomial and GMRES-IR with the FP32 inner cycle both reach 1e-10,
    and both solutions agree with the oracle's sparse direct solve (hash-checked) to 1e-8."""
    import numpy as np
    import torch

    import paper_2109_01232_b300 as g
    from paper_2109_01232_b300 import aniso_sweep
    p, b = gen.config_aniso_2d(side=2000)
    xr = aniso_sweep.reference_solution(2000)
    A = g.DeviceCSR.from_problem(p)
    bt = torch.tensor(b, device="cuda")
    for fn, kw in ((g.gmres_solve, {}), (g.gmres_ir_solve, dict(inner_prec="fp32"))):
        x = torch.zeros_like(bt)
        r = fn(A, bt, x, restart_m=50, rtol=1e-10, poly_degree=40, seed=7, max_iters=20000, **kw)
        assert r.status == g.OK and r.relres <= 1.0001e-10, (fn.__name__, r)
        err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= 1e-8, (fn.__name__, err)
