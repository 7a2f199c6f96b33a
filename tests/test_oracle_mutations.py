"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of the
oracle (a dropped term, a wrong sign, a shifted index, a transposed operand, a wrong
coefficient), runs ``tests/test_oracle_pins.py`` against that copy in a subprocess, and expects
it to fail.  A control run of the unmodified copy must pass.  CPU only; nothing here touches
the GPU path."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C = "oracle/tds_oracle.c"
PY = "oracle/oracle.py"

# (name, file, text, replacement): each text occurs exactly once in its file
MUTATIONS = [
    ("D1 drops its second tap pair", C,
     "r[-2] = -t2; r[-1] = -t1; r[0] = t0; r[1] = t1; r[2] = t2; }",
     "r[-2] = 0.0; r[-1] = -t1; r[0] = t0; r[1] = t1; r[2] = 0.0; }"),
    ("D2 second tap pair with the wrong sign", C,
     "else            { r[-2] =  t2;", "else            { r[-2] = -t2;"),
    ("D2 alpha 2/10 instead of 2/11", C, "alpha = 2.0 / 11.0;", "alpha = 2.0 / 10.0;"),
    ("Thomas forward step reads the previous row's sub-diagonal", C,
     "u[i] = w * (d[i] - a[i] * u[i - 1]);", "u[i] = w * (d[i] - a[i - 1] * u[i - 1]);"),
    ("Sherman-Morrison corner without 1/gamma", C,
     "bb[n - 1] = b[n - 1] - a[0] * c[n - 1] / gamma;", "bb[n - 1] = b[n - 1] - a[0] * c[n - 1];"),
    ("transposed band keeps the super-diagonal", C,
     "ct[i] = (i < n - 1) ? a[i + 1]", "ct[i] = (i < n - 1) ? c[i]"),
    ("B^T applied as B", C, "x[j] += coef * y[i];", "x[i] += coef * y[j];"),
    ("D1 closure at row 1: 1.4 for 1.5", C,
     "r1[-1] = -1.5 / (2.0 * h); r1[1] = 1.5 / (2.0 * h);", "r1[-1] = -1.5 / (2.0 * h); r1[1] = 1.4 / (2.0 * h);"),
    ("D2 closure at row 0: last tap with the wrong sign", C, "r0[3] = -1.0 / h2;", "r0[3] = 1.0 / h2;"),
    ("D1 closure at row n-1 not mirrored in sign", C, "rl[0] = 5.0 / (2.0 * h);", "rl[0] = -5.0 / (2.0 * h);"),
    ("filter centre tap 3/4 alpha_f -> 1/2 alpha_f", C,
     "a0 = 5.0 / 8.0 + 0.75 * af", "a0 = 5.0 / 8.0 + 0.5 * af"),
    ("filter closure row 1 centre 1/2 - alpha_f", C, "r1[0] = 0.5 + af;", "r1[0] = 0.5 - af;"),
    ("interpolation inner pair 1.4/2 for 3/2 / 2", C, "ha = 0.5 * 1.5", "ha = 0.5 * 1.4"),
    ("closed interpolation closure: coupling 4/3 for 5/3", C,
     "a[0] = 0.0; b[0] = 1.0; c[0] = 5.0 / 3.0;", "a[0] = 0.0; b[0] = 1.0; c[0] = 4.0 / 3.0;"),
    ("closed interpolation mirror row: taps not mirrored", C,
     "rm[1] = 5.0 / 24.0; rm[0] = 15.0 / 8.0;", "rm[1] = 15.0 / 8.0; rm[0] = 5.0 / 24.0;"),
    ("transport: conservative term subtracted", PY, "-0.5 * (conv + cons)", "-0.5 * (conv - cons)"),
    ("transport: viscous term of u_j", PY, "visc = deriv_lines(ui, 2, bc, h)", "visc = deriv_lines(uj, 2, bc, h)"),
    ("y lines taken in z-major order", PY,
     "return cart.transpose(0, 2, 1).reshape(nz * nx, ny)", "return cart.transpose(2, 0, 1).reshape(nz * nx, ny)"),
    ("interleaved layout with the line and row axes swapped", PY,
     "L.reshape(nl // sz, sz, n).transpose(0, 2, 1)", "L.reshape(nl // sz, n, sz)"),
]


def _copy_tree(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("__init__.py", "conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))


def _run_pins(dst):
    env = dict(os.environ)
    env["PYTHONPATH"] = dst
    env.pop("PYTEST_ADDOPTS", None)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join("tests", "test_oracle_pins.py")],
                          cwd=dst, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes(tmp_path):
    dst = str(tmp_path)
    _copy_tree(dst)
    r = _run_pins(dst)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name,path,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, path, old, new):
    dst = str(tmp_path)
    _copy_tree(dst)
    target = os.path.join(dst, path)
    with open(target) as fh:
        text = fh.read()
    assert text.count(old) == 1, "mutation anchor not unique or missing: %r" % old
    with open(target, "w") as fh:
        fh.write(text.replace(old, new))
    r = _run_pins(dst)
    # pytest exit code 1: tests ran and at least one failed (not an import or build error)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-2000:] + r.stderr[-2000:])
