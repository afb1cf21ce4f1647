"""Host-side checks of the C ABI (no GPU): the library builds, loads, exports every
symbol the header declares, validates arguments, and its host-only entry point
chase_cond_est agrees with the oracle's Eq. full-est."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chase_gb300.h")


@pytest.fixture(scope="module")
def cl():
    import paper_2603_10514_gb300 as P
    P.build()
    return P


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(chase_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["chase_solve", "chase_filter", "chase_qr", "chase_cond_est", "chase_create",
                 "chase_destroy", "chase_config_default", "chase_workspace_bytes",
                 "chase_status_string"]:
        assert want in names


def test_library_exports_every_declared_symbol(cl):
    out = subprocess.run(["nm", "-D", "--defined-only", cl.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (chase_[a-z_]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    L = cl.lib()
    for f in declared_functions():
        assert hasattr(L, f)


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "chase_gb300.h"\nint main(void){chase_config c; return chase_config_default(&c);}\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(tmp_path / "t.o")], check=True)


def test_documented_minimal_use_compiles_as_c(tmp_path):
    """The usage example in the header's introduction is valid C against the header."""
    lines = open(os.path.join(ROOT, "include", "chase_gb300.h")).read().splitlines()
    start = next(i for i, t in enumerate(lines) if "Minimal use" in t)
    body = []
    for t in lines[start + 1:]:
        if t.strip() == "*/":
            break
        body.append(t.strip()[1:].strip() if t.strip().startswith("*") else t)
    code = "\n".join(x for x in body if x and not x.startswith("device 0"))
    src = tmp_path / "use.c"
    src.write_text('#include "chase_gb300.h"\n'
                   "int use(int n, const void* dA, void* dV, int nev, int nex, double* evals,\n"
                   "        double* resid) {\n" + code + "\n  return rc;\n}\n")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(tmp_path / "use.o")], check=True)


def test_config_defaults(cl):
    cfg = cl.config_default()
    assert cfg.tol == 1e-10 and cfg.deg_init == 20 and cfg.deg_max == 36
    assert cfg.cond_hi == 1e8 and cfg.cond_lo == 20.0 and cfg.eta == 1.0


def test_status_strings(cl):
    assert cl.status_string(0) == "ok"
    assert "invalid" in cl.status_string(-3)
    assert "Cholesky" in cl.status_string(cl.CHASE_CHOL_FAILED)


def test_workspace_bytes_and_argument_checks(cl):
    L = cl.lib()
    b = ctypes.c_size_t()
    assert L.chase_workspace_bytes(1, 10000, 500, 100, 0, ctypes.byref(b)) == 0
    assert b.value > 5 * 10000 * 600 * 16
    assert L.chase_workspace_bytes(1, 10, 8, 5, 0, ctypes.byref(b)) == -4  # ell > n
    assert L.chase_workspace_bytes(5, 10, 8, 1, 0, ctypes.byref(b)) == -1
    # argument validation happens before any device work
    assert L.chase_solve(None, 0, 10, None, 10, 2, 1, None, None, None, 10, None, None, None, None, 0) == -1
    assert L.chase_qr(None, 0, 10, 2, None, 10, 1.0, 0, None, None) == -1
    assert L.chase_selftest_wait_timeout(None, 0.01) == -1


def test_cond_est_matches_oracle(cl):
    """chase_cond_est (host arithmetic of the library) against the oracle's Eq. full-est."""
    rng = np.random.default_rng(4)
    for trial in range(50):
        ell = int(rng.integers(2, 40))
        k = int(rng.integers(0, ell))
        ritz = np.sort(rng.uniform(-3, 0, ell))
        deg = np.sort(rng.integers(1, 40, ell)).astype(np.int32)
        lam1 = ritz[0] - rng.uniform(0, 0.5)
        c, e = rng.uniform(1, 3), rng.uniform(0.5, 2)
        eta = float(rng.uniform(1, 2))
        est, lest = cl.chase_cond_est(ritz, deg, k, lam1, c, e, eta)
        ref = oracle.log_cond_est(ritz[k], int(deg[k]), int(deg[-1]), lam1, c, e, eta)
        assert math.isclose(lest, ref, rel_tol=1e-14, abs_tol=1e-14)
        assert math.isclose(est, math.exp(ref), rel_tol=1e-13)


def test_cond_est_overflow_stays_finite_in_log(cl):
    est, lest = cl.chase_cond_est([-100.0, -1.0], [36, 2000], 0, -100.0, 1.0, 0.5)
    assert math.isinf(est) and math.isfinite(lest) and lest > 700


def test_struct_layouts_match_the_header(cl, tmp_path):
    """The binding's ctypes structures have the size and field offsets of the C header's
    (compiled here with gcc), so every field reaches the library where it expects it."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"chase_config": cl.Config, "chase_stats": cl.Stats, "chase_iter_log": cl.IterLog,
               "chase_bounds": cl.Bounds, "chase_problem": cl.Problem}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "chase_gb300.h"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(cl.LIB_PATH), "..", "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
