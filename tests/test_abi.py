"""The C-ABI library builds, loads and exports every entry point that
include/q2x.h declares; without a GPU it fails loudly (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "q2x.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(q2x_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def so():
    from paper_2107_10942_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("q2x_plan", "q2x_segments", "q2x_triangles_single", "q2x_triangles_double", "q2x_tetra",
                     "q2x_leaf_reduce"):
        assert required in names


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_no_cpu_fallback(so):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2107_10942_gb300 as q
    with pytest.raises(q.Q2XError) as ei:
        q.Plan(8)
    assert ei.value.status == 3  # Q2X_ERR_CUDA


def test_null_plan_is_an_argument_error(so):
    so.q2x_segments.restype = ctypes.c_int
    st = so.q2x_segments(None, ctypes.c_int64(0), ctypes.c_int64(0), None, None, None, ctypes.c_int64(0), None,
                         None, None, None, None, 0)
    assert st == 1
    so.q2x_last_error.restype = ctypes.c_char_p
    so.q2x_last_error.argtypes = [ctypes.c_void_p]
    assert so.q2x_last_error(None)  # a message is recorded


def test_null_plan_rejected_by_every_compute_entry(so):
    """Each compute entry point checks its plan before touching the device:
    called through the same ctypes signatures the binding uses, with a NULL
    plan and zero sizes, every one returns Q2X_ERR_ARG (1)."""
    from paper_2107_10942_gb300._lib import _SIGNATURES
    skip = {"q2x_plan", "q2x_last_error", "q2x_launch_count", "q2x_workspace_bytes", "q2x_plan_destroy",
            "q2x_batch_destroy", "q2x_batch_info", "q2x_device_errors", "q2x_plan_kernel_timing"}
    checked = []
    for name, argtypes in _SIGNATURES.items():
        if name in skip or not hasattr(so, name):
            continue
        f = getattr(so, name)
        f.restype = ctypes.c_int
        f.argtypes = argtypes
        args = [None if t is ctypes.c_void_p else t(0) if t in (ctypes.c_int, ctypes.c_int64) else None
                for t in argtypes]
        st = f(*args)
        assert st == 1, (name, st)
        checked.append(name)
    for required in ("q2x_nearfield", "q2x_segments_vector", "q2x_leaf_reduce_weighted", "q2x_translate",
                     "q2x_evaluate", "q2x_evaluate_curl", "q2x_galerkin_triangles"):
        assert required in checked


def test_header_is_plain_c(tmp_path):
    """include/q2x.h is a C header: a C99 translation unit that takes the
    address of every declared function compiles without warnings."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    src = tmp_path / "abi_check.c"
    src.write_text('#include "q2x.h"\n#include <stddef.h>\nvoid* q2x_abi_table[] = {\n' +
                   "".join("    (void*)&%s,\n" % n for n in names) + "    NULL\n};\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-Wno-pedantic",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "abi_check.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
