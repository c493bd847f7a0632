"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(msrcg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_math_9809043_gb300 import build as B
    try:
        return B.build()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc on this host
        if os.path.exists(B.LIB):
            return B.LIB
        pytest.skip(f"cannot build libmsrcg: {e}")


def test_header_declares_entry_points():
    names = _declared()
    for n in ("msrcg_build", "msrcg_solve", "msrcg_batch_solve", "msrcg_free", "msrcg_strerror"):
        assert n in names


def test_library_exports_all_declared(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(libpath):
    from paper_math_9809043_gb300 import msrcg as M
    o = M.default_opts()
    assert (o.scale, o.m, abs(o.f - 0.1) < 1e-15, o.maxit_outer) == (4, 4, True, 200)
    assert M.strerror(M.EBREAKDOWN).startswith("conjugate gradient")
    assert M.lib().msrcg_default_opts(None) == M.EINVAL


def test_set_trace_rejects_bad_arguments_on_the_host(libpath):
    # argument checks only: no hierarchy is built, nothing runs on a device
    from paper_math_9809043_gb300 import msrcg as M
    L = M.lib()
    assert L.msrcg_set_trace(None, None, 0) == M.EINVAL
    assert L.msrcg_set_trace(None, None, 16) == M.EINVAL
