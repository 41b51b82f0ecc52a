"""The bounded waits of the TMA-fed CGS kernels: a wait that runs out ends the solve with
GMRES_ERR_DEVICE_TIMEOUT, with no fault and no hang, and the GPU stays usable.

The test hook `tma_test_withhold` makes each launch's producer warp issue the copies of its
first row block only; the consumer warps' wait for the second block then cannot complete and
ends by the bound `tma_wait_cycles` (about half a millisecond here).  The producer still
waits for the copies it did issue before its CTA exits.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2109_01232_b300 as lib
    lib.lib()
    return lib


@pytest.mark.parametrize("kind,prec", [("ir", "fp32"), ("gmres", "fp32"), ("ir", "fp16")])
def test_tma_wait_expires_with_timeout_status(g, kind, prec):
    import torch
    # 60^3 = 216,000 rows: 848 row blocks of 256 over ~300 CTAs, so every CTA has a second
    # block to wait for
    p = gen.conv_diff_3d(60, 10.0, (1.0, 0.5, -0.2))
    A = g.DeviceCSR.from_problem(p)
    b = torch.ones(p.n, dtype=torch.float64, device="cuda")
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    plan = g.Plan(A, kind, restart_m=8, inner_prec=prec, cgs_kernel="tma",
                  tma_wait_cycles=1 << 20, tma_test_withhold=1)
    assert plan.info()["grid_vec"] * 2 <= (p.n + 255) // 256
    with pytest.raises(g.GmresError) as e:
        plan.solve(b, x)
    assert e.value.code == g.ERR_DEVICE_TIMEOUT
    plan.close()
    torch.cuda.synchronize()  # the context is still usable
    # the same plan shape without the hook solves the system
    plan = g.Plan(A, kind, restart_m=8, inner_prec=prec, cgs_kernel="tma",
                  tma_wait_cycles=1 << 20, rtol=1e-8, max_iters=4000)
    x.zero_()
    res = plan.solve(b, x)
    assert res.status == g.OK
    relres = np.linalg.norm(1.0 - oracle.spmv(p, x.cpu().numpy())) / np.sqrt(p.n)
    assert relres <= 1.0001e-8
    plan.close()


def test_negative_wait_bound_is_invalid(g):
    p = gen.conv_diff_2d(16, 1.0, (1.0, 0.0))
    A = g.DeviceCSR.from_problem(p)
    with pytest.raises(g.GmresError) as e:
        g.Plan(A, "ir", restart_m=4, tma_wait_cycles=-1)
    assert e.value.code == g.ERR_INVALID
