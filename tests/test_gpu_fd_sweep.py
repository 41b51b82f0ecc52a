"""The GMRES-FD switch-point sweep driver (Section 5.1) at a reduced size: every GMRES-FD
run converges to the tolerance, the switch points are restart multiples, and the FP32 stage
ends where it was told to."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,side", [("laplace3d", 30), ("uniflow2d", 120)])
def test_fd_sweep_small(kind, side):
    from paper_2109_01232_b300 import fd_sweep
    res = fd_sweep.run(kind, side, m=30, coarse=4, log=lambda *a: None)
    assert res["fp64"]["status"] == "OK" and res["ir"]["status"] == "OK"
    assert res["fd"], res
    for r in res["fd"]:
        assert r["switch"] % 30 == 0
        assert r["status"] == "OK" and r["relres"] <= 1.0001e-10, r
        assert r["fp32_iters"] <= r["switch"]
    assert res["best_fd"]["ms"] == min(r["ms"] for r in res["fd"])
    assert "best GMRES-FD" in fd_sweep.table(res)
