"""The C-ABI library loads on a machine without a GPU and exports every symbol that
include/gmres_ir.h declares; the ctypes structures match the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gmres_ir.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2109_01232_b300 import build
    build.build()
    import paper_2109_01232_b300 as g
    return g.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(gmres_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2109_01232_b300",
                                                                    "libgmres_ir.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(names) <= exported


def test_binding_covers_the_header(lib):
    import paper_2109_01232_b300 as g
    assert set(declared_functions()) == set(g.exported_symbols())


def test_struct_layout_matches_c(tmp_path, lib):
    import paper_2109_01232_b300 as g
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "gmres_ir.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(gmres_csr),"
        " sizeof(gmres_params), sizeof(gmres_stats), offsetof(gmres_params, seed),"
        " offsetof(gmres_stats, history), offsetof(gmres_params, record_history),"
        " offsetof(gmres_stats, rel_resid), offsetof(gmres_params, cgs_kernel)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    want = [ctypes.sizeof(g.csr_t), ctypes.sizeof(g.params_t), ctypes.sizeof(g.stats_t),
            g.params_t.seed.offset, g.stats_t.history.offset, g.params_t.record_history.offset,
            g.stats_t.rel_resid.offset, g.params_t.cgs_kernel.offset]
    assert got == want


def test_default_params_and_status_strings(lib):
    import paper_2109_01232_b300 as g
    p = g.default_params()
    assert (p.restart_m, p.rtol, p.inner_prec, p.poly_degree) == (50, 1e-10, 1, 0)
    assert p.cgs_kernel == g.CGS_KERNEL["register"]
    for code in range(9):
        assert lib.gmres_status_string(code)
    assert b"wait" in lib.gmres_status_string(g.ERR_DEVICE_TIMEOUT)
    assert g.MAX_RESTART == 512


def test_invalid_arguments_rejected_before_any_launch(lib):
    """Argument checks run on the host and need no device."""
    import paper_2109_01232_b300 as g
    p = g.default_params()
    st = g.stats_t()
    assert lib.gmres_solve(None, None, None, ctypes.byref(p), ctypes.byref(st), None) == g.ERR_INVALID
    c = g.csr_t(4, 4, 1, 1, 1)
    bad = g.default_params(restart_m=0)
    assert lib.gmres_ir_solve(ctypes.byref(c), 1, 1, ctypes.byref(bad), ctypes.byref(st), None) == g.ERR_INVALID
    big = g.default_params(restart_m=g.MAX_RESTART + 1)
    assert lib.gmres_ir_solve(ctypes.byref(c), 1, 1, ctypes.byref(big), ctypes.byref(st), None) == g.ERR_TOO_LARGE
    neg = g.default_params(rtol=-1.0)
    assert lib.gmres_solve(ctypes.byref(c), 1, 1, ctypes.byref(neg), ctypes.byref(st), None) == g.ERR_INVALID
    form = g.default_params(cgs_kernel=7)
    assert lib.gmres_solve(ctypes.byref(c), 1, 1, ctypes.byref(form), ctypes.byref(st), None) == g.ERR_INVALID
    for kw, code in ((dict(bj_block=-1), g.ERR_INVALID), (dict(bj_block=65), g.ERR_TOO_LARGE),
                     (dict(bj_block=4, poly_degree=5), g.ERR_INVALID),
                     (dict(max_outer=-1), g.ERR_INVALID)):
        q = g.default_params(**kw)
        assert lib.gmres_ir_solve(ctypes.byref(c), 1, 1, ctypes.byref(q), ctypes.byref(st), None) == code
    fd = g.default_params(bj_block=4)
    assert lib.gmres_fd_solve(ctypes.byref(c), 1, 1, ctypes.byref(fd), 50, None, None, None) == g.ERR_INVALID
    assert lib.gmres_plan_bj_apply(None, 1, 1, None) == g.ERR_INVALID
    assert lib.gmres_plan_perm(None, None, None) == g.ERR_INVALID
    empty = g.csr_t(0, 0, None, None, None)
    assert lib.gmres_ir_solve(ctypes.byref(empty), 1, 1, ctypes.byref(p), ctypes.byref(st), None) == g.OK


def test_batched_arguments_rejected_before_any_launch(lib):
    """Batched plan argument checks run on the host; an empty batch needs no device."""
    import numpy as np
    import paper_2109_01232_b300 as g
    plan = ctypes.c_void_p()
    p = g.default_params(restart_m=30)
    empty = g.csr_batch_t(0, None, None, None, None, None)
    assert lib.gmres_batch_plan_create(ctypes.byref(plan), ctypes.byref(empty), ctypes.byref(p), 1,
                                       None) == g.OK
    st = g.batch_stats_t(None, None, None, None, 0.0)
    assert lib.gmres_batch_plan_solve(plan, None, None, ctypes.byref(st), None) == g.OK
    assert lib.gmres_batch_plan_destroy(plan) == g.OK
    assert lib.gmres_ir_solve_batched(ctypes.byref(empty), None, None, ctypes.byref(p), None, None) == g.OK
    ro, no = np.array([0, 4], np.int64), np.array([0, 4], np.int64)
    one = g.csr_batch_t(1, ro.ctypes.data, no.ctypes.data, 1, 1, 1)
    for kw, code in ((dict(restart_m=g.BATCH_MAX_M + 1), g.ERR_TOO_LARGE),
                     (dict(inner_prec="fp16"), g.ERR_INVALID), (dict(poly_degree=3), g.ERR_INVALID),
                     (dict(bj_block=4), g.ERR_INVALID), (dict(max_outer=2), g.ERR_INVALID)):
        q = g.default_params(**{"restart_m": 30, **kw})
        assert lib.gmres_batch_plan_create(ctypes.byref(plan), ctypes.byref(one), ctypes.byref(q), 0,
                                           None) == code
    neg = g.csr_batch_t(-1, None, None, None, None, None)
    assert lib.gmres_batch_plan_create(ctypes.byref(plan), ctypes.byref(neg), ctypes.byref(p), 0,
                                       None) == g.ERR_INVALID
    bad_off = np.array([1, 4], np.int64)
    shifted = g.csr_batch_t(1, bad_off.ctypes.data, no.ctypes.data, 1, 1, 1)
    assert lib.gmres_batch_plan_create(ctypes.byref(plan), ctypes.byref(shifted), ctypes.byref(p), 0,
                                       None) == g.ERR_INVALID
    dec = np.array([0, 4, 3], np.int64)
    two = g.csr_batch_t(2, dec.ctypes.data, np.array([0, 4, 8], np.int64).ctypes.data, 1, 1, 1)
    assert lib.gmres_batch_plan_create(ctypes.byref(plan), ctypes.byref(two), ctypes.byref(p), 0,
                                       None) == g.ERR_INVALID
