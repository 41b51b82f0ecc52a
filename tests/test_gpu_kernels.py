"""Kernel parity on the GPU: the fused SpMV and the Arnoldi/CGS2 cycle kernels against the
CPU oracle on the same seeded inputs (several tiles and a ragged tail in every case)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "fp32", "fp16", "bf16"]


def _irregular(n=3000, seed=9):
    """CSR with empty rows and two rows longer than one shared-memory chunk."""
    g = np.random.default_rng(seed)
    lens = g.poisson(6, n)
    lens[[10, 11, 2999]] = 0
    lens[100] = 9000
    lens[2000] = 17000
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    cols = np.concatenate([np.sort(g.integers(0, n, L)) for L in lens]).astype(np.int32)
    vals = g.standard_normal(int(rp[-1]))
    return gen.Problem("irregular", n, rp.astype(np.int32), cols, vals)


PROBLEMS = {
    "2d": lambda: gen.conv_diff_2d(71, 25.0, (0.6, 0.8)),
    "3d": lambda: gen.conv_diff_3d(17, 10.0, (1.0, -2.0, 0.5)),
    "irregular": _irregular,
}


@pytest.fixture(scope="module")
def g():
    import paper_2109_01232_b300 as lib
    lib.lib()
    return lib


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _plan(g, p, prec, m=4):
    A = g.DeviceCSR.from_problem(p)
    kind = "gmres" if prec == "fp64" else "ir"
    return A, g.Plan(A, kind, restart_m=m, inner_prec=prec if prec != "fp64" else "fp32")


@pytest.mark.parametrize("which", list(PROBLEMS))
@pytest.mark.parametrize("prec", PRECS)
def test_spmv_parity(g, torch, which, prec):
    p = PROBLEMS[which]()
    A, plan = _plan(g, p, prec)
    v = np.random.default_rng(1).uniform(-1.0, 1.0, p.n)
    y = plan.spmv(torch.tensor(v, device="cuda")).double().cpu().numpy()
    pm = oracle.Precision.for_inner(prec, p)
    a_low = pm.matrix_values(p.vals)
    v_low = pm.store_vector(v)
    y_ref = pm.s_A * oracle.spmv(p, v_low, a_low)
    absA = pm.s_A * oracle.spmv(p, np.abs(v_low), np.abs(a_low))  # (|A| |v|) per row
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert np.all(np.abs(y - y_ref) <= tol * absA + 1e-300)
    assert np.linalg.norm(y - y_ref) <= tol * np.linalg.norm(absA)
    plan.close()


def test_splitmix64_device_matches_oracle(g, torch):
    dev = g.splitmix64(100003, 77).cpu().numpy()
    np.testing.assert_array_equal(dev, oracle.splitmix64_uniform(77, 100003))


def _basis(V, pm):
    return V.double().cpu().numpy().T / pm.s_v


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_arnoldi_fp64_matches_oracle(g, torch, which):
    p = PROBLEMS[which]()
    steps = 30
    A, plan = _plan(g, p, "fp64", m=steps)
    v0 = oracle.splitmix64_uniform(5, p.n)
    V, H, k = plan.arnoldi(torch.tensor(v0, device="cuda"), steps)
    op = lambda v: oracle.spmv(p, v)
    Vo, Ho, ko = oracle.arnoldi(op, v0, steps)
    assert k == ko == steps
    M = oracle.dense(p)
    nA = np.linalg.norm(M, 2)
    Vg = V.cpu().numpy().T
    # elementwise parity with the oracle's Arnoldi (FP64, different summation order)
    assert np.abs(H - Ho).max() <= 1e-12 * nA
    assert np.abs(Vg - Vo).max() <= 1e-11
    # Arnoldi relation and orthogonality of the GPU basis
    assert np.linalg.norm(M @ Vg[:, :k] - Vg @ H, 2) / nA <= 1e-12
    assert np.linalg.norm(np.eye(k + 1) - Vg.T @ Vg, 2) <= 1e-12
    plan.close()


@pytest.mark.parametrize("prec,orth_tol,rel_tol,h_tol", [
    ("fp32", 1e-5, 1e-5, 1e-5), ("fp16", 3e-2, 3e-3, 3e-3), ("bf16", 2e-1, 3e-2, 3e-2)])
def test_arnoldi_low_precision(g, torch, prec, orth_tol, rel_tol, h_tol):
    p = PROBLEMS["2d"]()
    steps = 20
    A, plan = _plan(g, p, prec, m=steps)
    v0 = oracle.splitmix64_uniform(6, p.n)
    V, H, k = plan.arnoldi(torch.tensor(v0, device="cuda"), steps)
    assert k == steps
    pm = oracle.Precision.for_inner(prec, p)
    Vg = _basis(V, pm)
    M = oracle.dense(p)
    nA = np.linalg.norm(M, 2)
    assert np.linalg.norm(np.eye(k + 1) - Vg.T @ Vg, 2) <= orth_tol
    assert np.linalg.norm(M @ Vg[:, :k] - Vg @ H, 2) / nA <= rel_tol
    # the oracle's emulated low-precision Arnoldi on the same input agrees on H
    a_low = pm.matrix_values(p.vals)
    op = lambda v: pm.rw(pm.s_A * oracle.spmv(p, v, a_low))
    _, Ho, ko = oracle.arnoldi(op, v0, steps, pm)
    assert ko == k
    assert np.abs(H[:6, :5] - Ho[:6, :5]).max() <= h_tol * nA
    plan.close()


# steps chosen so that the TMA-fed CGS kernels run for the first steps and the register
# kernels for the last ones (the basis block of a step stops fitting two shared-memory
# stages at 26 columns in FP64 and 53 in FP32; u1 keeps 64 column accumulators)
@pytest.mark.parametrize("prec,steps,tol", [
    ("fp64", 30, 1e-12), ("fp32", 56, 2e-5), ("fp16", 68, 2e-3), ("bf16", 68, 2e-2)])
def test_arnoldi_cgs_kernel_forms_agree(g, torch, prec, steps, tol):
    """The TMA-fed and register-fed CGS2 kernels compute the same step (only the order of
    the row sums inside a CTA differs), so the Hessenberg matrices agree to rounding."""
    p = PROBLEMS["3d"]()  # n = 4913: 20 row blocks of 256 and a ragged tail
    v0 = torch.tensor(oracle.splitmix64_uniform(8, p.n), device="cuda")
    A = g.DeviceCSR.from_problem(p)
    kind = "gmres" if prec == "fp64" else "ir"
    ip = prec if prec != "fp64" else "fp32"
    Hs = []
    for form in ("tma", "register"):
        plan = g.Plan(A, kind, restart_m=steps, inner_prec=ip, cgs_kernel=form)
        V, H, k = plan.arnoldi(v0, steps)
        assert k == steps
        Hs.append(H)
        plan.close()
    nA = np.abs(oracle.dense(p)).sum(axis=1).max()
    # the first steps agree to the working precision; later ones drift apart at most as
    # fast as the Arnoldi process amplifies rounding in the low-precision basis
    assert np.abs(Hs[0][:9, :8] - Hs[1][:9, :8]).max() <= tol * nA
    for H in Hs:
        assert np.isfinite(H).all()


def test_poly_roots_match_oracle(g, torch):
    p = gen.conv_diff_2d(40, 60.0, (1.0, 0.3))
    A = g.DeviceCSR.from_problem(p)
    for d in (5, 12):
        r_dev = g.poly_roots(A, d, seed=11)
        op = lambda v: oracle.spmv(p, v)
        r_ora = oracle.poly_roots(op, p.n, d, seed=11)
        assert len(r_dev) == len(r_ora) == d + 1
        np.testing.assert_allclose(np.sort_complex(r_dev), np.sort_complex(r_ora), rtol=1e-7)
        # the GMRES-polynomial identity with the device roots, evaluated by the oracle
        v0 = oracle.splitmix64_uniform(11, p.n)
        res = np.linalg.norm(v0 - op(oracle.poly_apply(op, r_dev, v0))) / np.linalg.norm(v0)
        res_o = np.linalg.norm(v0 - op(oracle.poly_apply(op, r_ora, v0))) / np.linalg.norm(v0)
        assert res == pytest.approx(res_o, rel=1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_plain_spmv_parity(g, torch, prec):
    """The SpMV-only timing kernel computes the same product as the oracle."""
    p = PROBLEMS["3d"]()
    A, plan = _plan(g, p, prec)
    v = np.random.default_rng(2).uniform(-1.0, 1.0, p.n)
    x = torch.tensor(v, device="cuda", dtype=torch.float64 if prec == "fp64" else torch.float32)
    y, ms = plan.spmv_timed(x, 3)
    pm = oracle.Precision.for_inner(prec, p)
    a_low = pm.matrix_values(p.vals)
    xv = x.double().cpu().numpy()
    y_ref = pm.s_A * oracle.spmv(p, xv, a_low)
    absA = pm.s_A * oracle.spmv(p, np.abs(xv), np.abs(a_low))
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert np.all(np.abs(y.double().cpu().numpy() - y_ref) <= tol * absA + 1e-300)
    assert ms > 0
    plan.close()
