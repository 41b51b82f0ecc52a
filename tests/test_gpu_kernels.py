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


def _wide(n=40000, seed=10):
    """Five random columns per row anywhere in [0, n) plus the diagonal: |column - row| reaches
    past 32767, so the plan keeps 32-bit column entries in its SELL copy."""
    g = np.random.default_rng(seed)
    cols = np.sort(np.concatenate([g.integers(0, n, (n, 5)), np.arange(n)[:, None]], axis=1), axis=1)
    vals = g.standard_normal((n, 6))
    vals[cols == np.arange(n)[:, None]] = 8.0
    rp = np.arange(0, 6 * n + 1, 6, dtype=np.int32)
    return gen.Problem("wide", n, rp, cols.ravel().astype(np.int32), vals.ravel())


PROBLEMS = {
    "2d": lambda: gen.conv_diff_2d(71, 25.0, (0.6, 0.8)),
    "3d": lambda: gen.conv_diff_3d(17, 10.0, (1.0, -2.0, 0.5)),
    "irregular": _irregular,
    "wide": _wide,
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


def _norm_inf(p):
    """||A||_inf (largest absolute row sum) from the CSR arrays."""
    rows = np.repeat(np.arange(p.n), np.diff(p.row_ptr))
    return float(np.bincount(rows, weights=np.abs(p.vals), minlength=p.n).max())


# n >= 10^4 with a ragged tail: the SELL kernels run many slices per warp tile, many CTAs
# per launch and a partial last tile (16,900 and 19,683 are no multiple of 32 VEC rows).
LARGE = {
    "2d130": lambda: gen.conv_diff_2d(130, 25.0, (0.6, 0.8)),
    "3d27": lambda: gen.conv_diff_3d(27, 10.0, (1.0, -2.0, 0.5)),
}


def _column_errors(Vg, H, Vo, Ho, nA):
    """Per column c: ||V_gpu[:, c] - V_oracle[:, c]||_2 and ||H_gpu[:, c] - H_oracle[:, c]||_2
    / ||A||_inf (the Hessenberg column c has c + 2 entries)."""
    k = H.shape[1]
    dV = np.linalg.norm(Vg[:, :k + 1] - Vo[:, :k + 1], axis=0)
    dH = np.array([np.linalg.norm(H[:c + 2, c] - Ho[:c + 2, c]) for c in range(k)]) / nA
    return dV, dH


# FP64 plans with at least 1024 rows per SM run the step kernels with four rows per thread,
# smaller ones with two: 3d56 (175,616 rows) takes the four-row kernels on a 148-SM B300.
FP64_WIDE = {"3d56": lambda: gen.conv_diff_3d(56, 10.0, (1.0, -2.0, 0.5))}


@pytest.mark.parametrize("which", ["2d", "3d", "2d130", "3d27", "3d56"])
def test_arnoldi_fp64_matches_oracle(g, torch, which):
    """FP64 Arnoldi/CGS2 (Algorithm 1, Section 3.1) against the oracle, every column of V
    and H to 1e-13 (normwise, H relative to ||A||).  The two differ only in the order of
    their sums; measured on a B300 the gap grows from ~1e-16 to ~4e-15 (V) and stays below
    2e-16 ||A|| (H) over 50 steps, the same size as the oracle's own spread when its start
    vector is perturbed by one unit roundoff.  Both FP64 kernel sets are covered (two rows
    per thread below 1024 rows per SM, four above)."""
    p = (PROBLEMS.get(which) or LARGE.get(which) or FP64_WIDE[which])()
    if which in FP64_WIDE:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert p.n >= 1024 * sms  # the four-row kernels run
    steps = 30 if which in PROBLEMS or which in FP64_WIDE else 50
    A, plan = _plan(g, p, "fp64", m=steps)
    v0 = oracle.splitmix64_uniform(5, p.n)
    V, H, k = plan.arnoldi(torch.tensor(v0, device="cuda"), steps)
    op = lambda v: oracle.spmv(p, v)
    Vo, Ho, ko = oracle.arnoldi(op, v0, steps)
    assert k == ko == steps
    nA = _norm_inf(p)
    Vg = V.cpu().numpy().T
    dV, dH = _column_errors(Vg, H, Vo, Ho, nA)
    assert dV.max() <= 1e-13, dV
    assert dH.max() <= 1e-13, dH
    if p.n <= 6000:  # Arnoldi relation and orthogonality of the GPU basis (dense check)
        M = oracle.dense(p)
        n2 = np.linalg.norm(M, 2)
        assert np.linalg.norm(M @ Vg[:, :k] - Vg @ H, 2) / n2 <= 1e-12
        assert np.linalg.norm(np.eye(k + 1) - Vg.T @ Vg, 2) <= 1e-12
    plan.close()


# Bounds per column against the emulated oracle (same stored roundings, FP32 or FP64 sums in
# a different order).  Measured on a B300 over 50 steps at n = 16,900 / 19,683: FP32 V 1.9e-6,
# H 1.2e-8 ||A||; FP16 V 1.5e-3 (~3 u_fp16), H 7.6e-6 ||A||; BF16 V 1.1e-2 (~3 u_bf16),
# H 3.7e-5 ||A||.  A stored value that rounds to the other neighbour on one side moves that
# entry by one unit of the storage format, and the later steps inherit it, so V's bound is a
# small multiple of the storage unit roundoff and grows with the step.
@pytest.mark.parametrize("prec,v_tol,h_tol", [
    ("fp32", 1e-5, 1e-5), ("fp16", 1e-2, 1e-4), ("bf16", 5e-2, 3e-4)])
@pytest.mark.parametrize("which", list(LARGE))
def test_arnoldi_low_precision(g, torch, which, prec, v_tol, h_tol):
    p = LARGE[which]()
    steps = 50
    A, plan = _plan(g, p, prec, m=steps)
    v0 = oracle.splitmix64_uniform(5, p.n)
    V, H, k = plan.arnoldi(torch.tensor(v0, device="cuda"), steps)
    assert k == steps
    pm = oracle.Precision.for_inner(prec, p)
    Vg = _basis(V, pm)
    a_low = pm.matrix_values(p.vals)
    op = lambda v: pm.rw(pm.s_A * oracle.spmv(p, v, a_low))
    Vo, Ho, ko = oracle.arnoldi(op, v0, steps, pm)
    assert ko == k
    nA = _norm_inf(p)
    dV, dH = _column_errors(Vg, H, Vo, Ho, nA)
    assert dV.max() <= v_tol, dV
    assert dH.max() <= h_tol, dH
    # the GPU basis is orthonormal to the storage precision (CGS2) and satisfies the
    # Arnoldi relation with the stored copy of A; the oracle's emulated basis reaches
    # 1.7 u_s and 0.33 u_s on these problems
    u_s = oracle.unit_roundoff(prec)
    G = Vg.T @ Vg
    assert np.abs(np.eye(k + 1) - G).max() <= 16 * u_s
    AV = np.stack([pm.s_A * oracle.spmv(p, Vg[:, c], a_low) for c in range(k)], axis=1)
    assert np.linalg.norm(AV - Vg @ H) / (nA * np.sqrt(k)) <= 4 * u_s
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
    for form in ("register", "tma"):
        plan = g.Plan(A, kind, restart_m=steps, inner_prec=ip, cgs_kernel=form)
        V, H, k = plan.arnoldi(v0, steps)
        assert k == steps
        Hs.append(H)
        plan.close()
    nA = np.abs(oracle.dense(p)).sum(axis=1).max()
    # the first steps agree to the working precision; later ones drift apart at most as
    # fast as the Arnoldi process amplifies rounding in the low-precision basis
    for H in Hs[1:]:
        assert np.abs(Hs[0][:9, :8] - H[:9, :8]).max() <= tol * nA
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
