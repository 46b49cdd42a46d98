"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/s3ttv.h declares, its host-only helpers agree
with the oracle, and the product never touches the oracle."""
import ast
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "s3ttv.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(s3ttv_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_03313_gb300 import build as B
    B.build()
    import paper_2404_03313_gb300 as P
    return P.library()


def test_header_declares_the_boundary():
    fns = _declared_functions()
    for name in ("s3ttv_create", "s3ttv_solve", "s3ttv_destroy"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    import paper_2404_03313_gb300 as P
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in P.SIGNATURES, f"binding lacks {name}"


def test_host_helpers_match_oracle(lib):
    import oracle as O
    import paper_2404_03313_gb300 as P
    for N, sig, ps, pt in ((16384, 0.1, 0.05, 0.05), (8388608, 0.05, 0.05, 0.10), (100, 0.0, 0.0, 0.05)):
        np.testing.assert_allclose(P.radii(N, sig, ps, pt), O.radii(N, sig, ps, pt), rtol=1e-15)
    for pol, name in ((P.STEP_PAPER, "paper"), (P.STEP_PC_EXACT, "pc_exact")):
        g = P.step_sizes(256, 256, 5, pol)
        go = O.step_sizes(256, 256, 5, name)
        for key in go:
            assert g[key] == pytest.approx(go[key], rel=1e-15)


def test_invalid_arguments_rejected_on_host(lib):
    e = ctypes.c_double()
    assert lib.s3ttv_radii(0, 0.1, 0.05, 0.05, 0.95, ctypes.byref(e), ctypes.byref(e), ctypes.byref(e)) == -1
    assert lib.s3ttv_radii(10, 0.1, 1.5, 0.05, 0.95, ctypes.byref(e), ctypes.byref(e), ctypes.byref(e)) == -1
    g = (ctypes.c_double * 6)()
    assert lib.s3ttv_step_sizes(4, 4, 2, 7, g) == -1
    assert lib.s3ttv_create(None, 0, None) == -1
    assert lib.s3ttv_solve_batched(None, 1, None, 10, 0.0, None) == -1
    assert lib.s3ttv_strerror(-4).decode() == "NaN or Inf in the iterates"


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.s3ttv_create(ctypes.byref(h), 0, None)
    assert rc in (-1, -3) and not h.value


def _imports(path):
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def _py_files(d):
    for base, _, files in os.walk(os.path.join(ROOT, d)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_oracle_and_product_are_independent():
    for f in _py_files("oracle"):
        assert "paper_2404_03313_gb300" not in _imports(f), f
    for f in _py_files("paper_2404_03313_gb300"):
        mods = _imports(f)
        assert "oracle" not in mods and "synthetic" not in mods, f
    # the CUDA sources do not reach into oracle/ either
    csrc = os.path.join(ROOT, "paper_2404_03313_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower(), f


def test_header_is_plain_c(lib):
    """include/s3ttv.h compiles as strict C99 (no C++ or torch types in the
    boundary), and a C program that takes the address of every entry point it
    declares links against the library."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2404_03313_gb300 import LIB_PATH
    fns = _declared_functions()
    src = '#include "s3ttv.h"\n#include <stdio.h>\ntypedef void (*fn_t)(void);\n'
    src += "static fn_t table[] = {\n" + "".join(f"  (fn_t)&{name},\n" for name in fns) + "};\n"
    src += 'int main(void) {\n  printf("%d\\n", (int)(sizeof table / sizeof table[0]));\n  return 0;\n}\n'
    with tempfile.TemporaryDirectory() as d:
        c, o, exe = (os.path.join(d, x) for x in ("abi.c", "abi.o", "abi"))
        with open(c, "w") as f:
            f.write(src)
        p = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                            os.path.join(ROOT, "include"), "-c", c, "-o", o], capture_output=True, text=True)
        assert p.returncode == 0, p.stderr
        p = subprocess.run([gcc, o, "-o", exe, os.path.abspath(LIB_PATH)], capture_output=True, text=True)
        assert p.returncode == 0, p.stderr
