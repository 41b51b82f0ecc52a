"""GMRES-FD (Section 3.3): single-precision GMRES followed by FP64 GMRES at a restart,
against the oracle's GMRES-FD on the same seeded systems."""
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


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _problem():
    p, b, _ = gen.config_small_2d(32)
    return p, b


@pytest.mark.parametrize("switch", [30, 60, 150])
def test_fd_matches_oracle(g, torch, switch):
    p, b = _problem()
    A = g.DeviceCSR.from_problem(p)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    r32, r64 = g.gmres_fd_solve(A, torch.tensor(b, device="cuda"), x, switch, restart_m=30, rtol=1e-10)
    xo, i32, i64 = oracle.gmres_fd(p, b, switch, m=30, rtol=1e-10)
    assert r64.status == g.OK
    assert r32.iters == switch or (r32.iters < switch and r32.status == g.OK)
    # the same split of the work between the stages, up to one cycle each
    assert abs(r32.iters - i32.iters) <= 30
    assert abs(r64.iters - i64.iters) <= 30
    xg = x.cpu().numpy()
    M = p.scipy()
    assert np.linalg.norm(b - M @ xg) / np.linalg.norm(b) <= 1e-10
    assert np.abs(xg - xo).max() / np.abs(xo).max() <= 1e-7


def test_fp32_gmres_stagnates_at_single_precision(g, torch):
    """GMRES run entirely in FP32 cannot go below ~u32 * cond: its true residual stalls."""
    p, b = _problem()
    A = g.DeviceCSR.from_problem(p)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    plan = g.Plan(A, "fp32", restart_m=30, rtol=1e-10, max_iters=600)
    r = plan.solve(torch.tensor(b, device="cuda"), x)
    plan.close()
    assert r.status == g.NOT_CONVERGED and r.iters == 600
    xg = x.cpu().numpy()
    rel = np.linalg.norm(b - p.scipy() @ xg) / np.linalg.norm(b)
    assert 1e-9 < rel < 1e-4
    assert np.array_equal(xg, xg.astype(np.float32).astype(np.float64))  # x stays in FP32


def test_fd_switch_zero_is_fp64_gmres(g, torch):
    p, b = _problem()
    A = g.DeviceCSR.from_problem(p)
    bt = torch.tensor(b, device="cuda")
    xa = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    xb = torch.zeros_like(xa)
    r32, r64 = g.gmres_fd_solve(A, bt, xa, 0, restart_m=30, rtol=1e-10)
    r = g.gmres_solve(A, bt, xb, restart_m=30, rtol=1e-10)
    assert r32.iters == 0 and r64.iters == r.iters
    assert torch.equal(xa, xb)
