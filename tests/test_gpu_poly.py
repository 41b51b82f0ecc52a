"""GPU parity of the GMRES-polynomial right preconditioner (Section 3.4)."""
import numpy as np
import pytest

import gen
import oracle
from oracle.gmres import _fp64

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


def _dev(torch, *arrs):
    return [torch.tensor(a, dtype=torch.float64, device="cuda") for a in arrs]


@pytest.mark.parametrize("degree", [4, 10, 25])
def test_device_polynomial_satisfies_gmres_identity(g, torch, degree):
    """A p(A) v0 is the (d+1)-step GMRES approximation of v0, so ||v0 - A p(A) v0|| equals
    the oracle's GMRES residual from v0 (independent of how the roots are computed)."""
    p = gen.conv_diff_2d(45, 80.0, (0.9, 0.4))
    seed = 21
    A = g.DeviceCSR.from_problem(p)
    plan = g.Plan(A, "gmres", restart_m=10, poly_degree=degree, seed=seed)
    v0 = oracle.splitmix64_uniform(seed, p.n)
    z = plan.poly_apply(torch.tensor(v0, device="cuda")).cpu().numpy()
    op = lambda v: oracle.spmv(p, v)
    res_dev = np.linalg.norm(v0 - op(z)) / np.linalg.norm(v0)
    cyc = oracle.gmres_cycle(op, v0, degree + 1, -1.0, _fp64(p.n))
    assert res_dev == pytest.approx(cyc.hist[-1], rel=1e-6)
    # same operator as the oracle's product form with the oracle's own roots
    th = oracle.poly_roots(op, p.n, degree, seed=seed)
    zo = oracle.poly_apply(op, th, v0)
    assert np.linalg.norm(z - zo) <= 1e-7 * np.linalg.norm(zo)
    assert len(plan.roots()) == degree + 1
    plan.close()


def test_fp32_polynomial_apply_matches_emulated_oracle(g, torch):
    p = gen.conv_diff_2d(45, 30.0, (0.2, 1.0))
    A = g.DeviceCSR.from_problem(p)
    plan = g.Plan(A, "ir", restart_m=10, poly_degree=10, seed=3, inner_prec="fp32")
    v = np.random.default_rng(4).uniform(-1, 1, p.n)
    z = plan.poly_apply(torch.tensor(v, device="cuda")).double().cpu().numpy()
    pm = oracle.Precision.for_inner("fp32", p)
    a_low = pm.matrix_values(p.vals)
    op_low = lambda x: pm.rw(pm.s_A * oracle.spmv(p, x, a_low))
    th = oracle.poly_roots(lambda x: oracle.spmv(p, x), p.n, 10, seed=3)
    zo = oracle.poly_apply(op_low, th, pm.rw(v), pm.rw)
    assert np.linalg.norm(z - zo) <= 1e-5 * np.linalg.norm(zo)
    plan.close()


@pytest.mark.parametrize("kind,prec", [("gmres", "fp64"), ("ir", "fp32"), ("ir", "fp16"),
                                       ("ir", "bf16")])
def test_preconditioned_solves(g, torch, kind, prec):
    p, b = gen.config_aniso_2d(side=64)
    A = g.DeviceCSR.from_problem(p)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    fn = g.gmres_solve if kind == "gmres" else g.gmres_ir_solve
    r = fn(A, bt, xt, restart_m=30, rtol=1e-10, poly_degree=10, seed=7,
           inner_prec=prec if kind == "ir" else "fp32", max_iters=20000)
    x = xt.cpu().numpy()
    relres = np.linalg.norm(b - oracle.spmv(p, x)) / np.linalg.norm(b)
    assert r.status == g.OK and relres <= 1.0001e-10, (r, relres)
    op = lambda v: oracle.spmv(p, v)
    th = oracle.poly_roots(op, p.n, 10, seed=7)
    r0 = fn(A, bt, xt.zero_(), restart_m=30, rtol=1e-10, max_iters=20000,
            inner_prec=prec if kind == "ir" else "fp32")
    assert r.iters < r0.iters  # the preconditioner reduces the iteration count
    if kind == "gmres":
        _, io = oracle.gmres(p, b, m=30, rtol=1e-10, poly_roots=th)
        assert abs(r.iters - io.iters) <= 30
    else:
        assert r.iters % 30 == 0
        if prec == "fp32":
            _, io = oracle.gmres_ir(p, b, m=30, rtol=1e-10, poly_roots=th, inner="fp32")
            assert abs(r.iters - io.iters) <= 60


def test_fp64_gmres_with_fp32_polynomial(g, torch):
    """FP64 GMRES with the polynomial applied in FP32 (Section 5.4's middle configuration):
    the apply matches the emulated FP32 oracle, and the solve reaches 1e-10 in about the
    iterations of the all-FP64 preconditioned solve."""
    p, b = gen.config_aniso_2d(side=64)
    A = g.DeviceCSR.from_problem(p)
    plan = g.Plan(A, "gmres", restart_m=30, poly_degree=10, seed=7, poly_in_fp32=1)
    v = np.random.default_rng(5).uniform(-1, 1, p.n)
    z = plan.poly_apply(torch.tensor(v, device="cuda"))
    assert z.dtype == torch.float32
    pm = oracle.Precision.for_inner("fp32", p)
    a_low = pm.matrix_values(p.vals)
    op_low = lambda x: pm.rw(pm.s_A * oracle.spmv(p, x, a_low))
    th = oracle.poly_roots(lambda x: oracle.spmv(p, x), p.n, 10, seed=7)
    zo = oracle.poly_apply(op_low, th, pm.rw(v), pm.rw)
    assert np.linalg.norm(z.double().cpu().numpy() - zo) <= 1e-5 * np.linalg.norm(zo)
    plan.close()
    bt, xt = _dev(torch, b, np.zeros(p.n))
    r = g.gmres_solve(A, bt, xt, restart_m=30, rtol=1e-10, poly_degree=10, seed=7, poly_in_fp32=1,
                      max_iters=20000)
    x = xt.cpu().numpy()
    relres = np.linalg.norm(b - oracle.spmv(p, x)) / np.linalg.norm(b)
    assert r.status == g.OK and relres <= 1.0001e-10
    r64 = g.gmres_solve(A, bt, xt.zero_(), restart_m=30, rtol=1e-10, poly_degree=10, seed=7,
                        max_iters=20000)
    assert abs(r.iters - r64.iters) <= 30


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_polynomial_path_with_a_matrix_larger_than_l2(g, torch, prec):
    """On a 1500^2 anisotropic problem the inner copy of A (90 MB in FP32) and the
    polynomial's vectors exceed three quarters of the L2, so the plan streams the matrix
    through the polynomial's SpMVs evict-first: the apply still matches the emulated oracle
    (FP32) and GMRES-IR with the degree-10 polynomial reaches 1e-10 by the oracle's explicit
    residual."""
    p, b = gen.config_aniso_2d(side=1500)
    A = g.DeviceCSR.from_problem(p)
    plan = g.Plan(A, "ir", restart_m=50, inner_prec=prec, poly_degree=10, seed=7, max_iters=20000)
    if prec == "fp32":
        pm = oracle.Precision("fp32", "fp32", p.n)
        a32 = pm.matrix_values(p.vals)
        op = lambda v: pm.rw(oracle.spmv(p, v, a32))
        v = oracle.splitmix64_uniform(3, p.n)
        z = plan.poly_apply(torch.tensor(v, device="cuda")).double().cpu().numpy()
        zo = oracle.poly_apply(op, plan.roots(), pm.rw(v), pm.rw)
        assert np.linalg.norm(z - zo) <= 1e-5 * np.linalg.norm(zo)
    bt, xt = _dev(torch, b, np.zeros(p.n))
    res = plan.solve(bt, xt)
    assert res.status == g.OK
    x = xt.cpu().numpy()
    assert np.linalg.norm(b - oracle.spmv(p, x)) / np.linalg.norm(b) <= 1.0001e-10
    plan.close()
