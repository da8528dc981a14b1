"""The C-ABI library builds, loads and exports every entry point that
include/eigref.h declares; host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2602_23778_gb300 import build
    build.build()
    import paper_2602_23778_gb300 as pkg
    return pkg.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "eigref.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eigref_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 9
    for name in names:
        assert hasattr(L, name), name
    import paper_2602_23778_gb300 as pkg
    assert sorted(pkg.SYMBOLS) == sorted(set(pkg.SYMBOLS) & set(names))


def test_params_default(L):
    import paper_2602_23778_gb300 as pkg
    p = pkg.Handle.params()
    assert (p.target, p.max_iters, p.tol, p.stop, p.precision, p.delta_c, p.sign_fix, p.use_graph) == \
        (0, 100, 0.0, 0, 0, 10.0, 1, 1)


def test_struct_layout_matches_header(tmp_path):
    """ctypes mirrors of eigref_params / eigref_report / eigref_problem agree with the C compiler's layout."""
    import subprocess
    import paper_2602_23778_gb300 as pkg
    fields = {"eigref_params": pkg.Params, "eigref_report": pkg.Report, "eigref_problem": pkg.Problem}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "eigref.h"', "int main(void) {"]
    for cname, cls in fields.items():
        src.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for f, _ in cls._fields_:
            src.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f))
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = []
    for cls in fields.values():
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert got == want


def test_status_strings(L):
    import paper_2602_23778_gb300 as pkg
    assert pkg.status_string(0) == "ok"
    assert "diverged" in pkg.status_string(5)
    assert pkg.status_string(99) == "unknown status"


def test_create_rejects_bad_arguments(L):
    h = ctypes.c_void_p()
    assert L.eigref_create(None, 0, None) == 1
    assert L.eigref_create(ctypes.byref(h), -1, None) == 1
    assert L.eigref_destroy(None) == 0


def test_oracle_evaluator_builds():
    from oracle import dd
    assert os.path.exists(dd.build())


def test_binding_refuses_mismatched_shapes_before_the_library(monkeypatch):
    """A narrow or mismatched P (or X, G, S) is refused in the binding, so no
    kernel can write past an output's end; the library is never reached."""
    import numpy as np
    import paper_2602_23778_gb300 as pkg

    def no_library():
        raise AssertionError("the library was called")

    monkeypatch.setattr(pkg, "lib", no_library)
    A = np.zeros((8, 8))
    X = np.zeros((8, 3), order="F")
    good = np.zeros((8, 3), order="F")
    for bad in (np.zeros((8, 2), order="F"), np.zeros((7, 3), order="F"), np.zeros((9, 3), order="F")):
        with pytest.raises(ValueError):
            pkg.product_dense_noalloc(A, X, bad)
        with pytest.raises(ValueError):
            pkg.Handle.product_dense(None, A, X, bad)
        with pytest.raises(ValueError):
            pkg.Handle.gram(None, X, bad, np.zeros((3, 3), order="F"), np.zeros((3, 3), order="F"))
    with pytest.raises(ValueError):
        pkg.product_dense_noalloc(A, np.zeros((7, 3), order="F"), good)
    with pytest.raises(ValueError):
        pkg.Handle.gram(None, X, good, np.zeros((2, 3), order="F"), np.zeros((3, 3), order="F"))
    rp = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8], dtype=np.int32)
    ci = np.arange(8, dtype=np.int32)
    val = np.ones(8)
    with pytest.raises(ValueError):
        pkg.Handle.product_csr(None, rp, ci, val, X, np.zeros((8, 2), order="F"))
