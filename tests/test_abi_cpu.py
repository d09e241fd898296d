"""The C ABI library builds, loads and exports what include/*.h declares;
argument errors are reported without touching a GPU."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1406_5161_gb300 as pkg
from paper_1406_5161_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(svm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    assert "svm_train" in names and "svm_decision" in names


def test_library_exports_every_declared_symbol():
    lib = pkg.load()
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in declared_functions():
        assert name in exported, f"{name} declared but not exported"
        assert hasattr(lib, name)


def test_version_string():
    assert "sm_103a" in pkg.svm_version()


@pytest.mark.parametrize("kw,msg", [
    (dict(C=0.0), "C must be"),
    (dict(gamma=-1.0), "gamma must be"),
    (dict(tau=0.0), "tau must be"),
    (dict(precision=7), "unknown precision"),
])
def test_argument_errors_are_reported(kw, msg):
    p = synth.small_dense(10, 3, seed=1)
    args = dict(C=1.0, gamma=0.1, tau=1e-3)
    args.update(kw)
    r = pkg.svm_train(p.X, p.y, check=False, **args)
    assert r["status"] == pkg.SVM_ERR_ARG
    assert msg in pkg.svm_last_error()


def test_bad_shrink_policy_is_reported():
    p = synth.small_dense(10, 3, seed=1)
    r = pkg.svm_train(p.X, p.y, 1.0, 0.1, 1e-3, shrink=(9, 1, 0), check=False)
    assert r["status"] == pkg.SVM_ERR_ARG


def test_flag_constants_match_header():
    src = "".join(open(h).read() for h in glob.glob(os.path.join(ROOT, "include", "*.h")))
    defines = dict(re.findall(r"^#define (SVM_FLAG_\w+) (\d+)", src, flags=re.M))
    assert defines, "no SVM_FLAG_* in the header"
    for name, value in defines.items():
        assert getattr(pkg, name) == int(value), name


def test_ctypes_struct_sizes_match_header(tmp_path):
    """The Python binding's ctypes structures have the C header's sizes."""
    from paper_1406_5161_gb300 import _abi
    names = ["svm_csr", "svm_params", "svm_shrink_policy", "svm_stats"]
    prog = "#include <stdio.h>\n#include \"svm_gb300.h\"\nint main(void){\n" + "".join(
        f'printf("%zu\\n", sizeof({n}));\n' for n in names) + "return 0;}\n"
    (tmp_path / "sz.c").write_text(prog)
    exe = str(tmp_path / "sz")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(tmp_path / "sz.c"),
                    "-o", exe], check=True)
    sizes = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                            check=True).stdout.split()]
    import ctypes
    for n, s in zip(names, sizes):
        assert ctypes.sizeof(getattr(_abi, n)) == s, n


def test_shrink_presets_match_the_python_ones(tmp_path):
    """SVM_SHRINK_AGGRESSIVE / _AVERAGE / _LAZY initialise the C struct with
    the Table 3 classes the Python presets name."""
    prog = ("#include <stdio.h>\n#include \"svm_gb300.h\"\nint main(void){\n"
            "svm_shrink_policy p[3] = {SVM_SHRINK_AGGRESSIVE, SVM_SHRINK_AVERAGE, SVM_SHRINK_LAZY};\n"
            "for (int i = 0; i < 3; ++i) printf(\"%d %d %.17g %.17g\\n\", p[i].kind, p[i].recon, p[i].value,"
            " p[i].first_factor);\nreturn 0;}\n")
    (tmp_path / "pre.c").write_text(prog)
    exe = str(tmp_path / "pre")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(tmp_path / "pre.c"),
                    "-o", exe], check=True)
    rows = [line.split() for line in subprocess.run([exe], capture_output=True, text=True,
                                                     check=True).stdout.splitlines()]
    for row, py in zip(rows, (pkg.AGGRESSIVE, pkg.AVERAGE, pkg.LAZY)):
        kind, value, recon = py
        assert int(row[0]) == kind and int(row[1]) == recon and float(row[2]) == value
        assert float(row[3]) == 20.0


def test_fixed_workspace_rejects_huge_d_before_any_device_work():
    """d >= 2^31 cannot be carried by the row pass's 32-bit column layout; the
    fixed-workspace call must refuse it from its argument checks alone (the
    pointers below are never read, and no CUDA call is made on this host)."""
    import ctypes as ct
    from paper_1406_5161_gb300 import _abi
    lib = pkg.load()
    dummy = (ct.c_double * 16)()
    addr = ct.addressof(dummy)
    for d in (2 ** 31, 2 ** 32 + 5):
        X = _abi.svm_csr(10, d, addr, addr, addr, 1, 0)
        p = _abi.svm_params()
        p.C, p.gamma, p.tau, p.precision = 1.0, 0.1, 1e-3, pkg.SVM_FP64
        b = ct.c_double(0.0)
        it = ct.c_int64(0)
        rc = lib.svm_train_fixed_workspace(ct.byref(X), addr, ct.byref(p), addr, ct.byref(b),
                                           ct.byref(it))
        assert rc == pkg.SVM_ERR_ARG, d
        assert "d must be < 2^31" in pkg.svm_last_error()
