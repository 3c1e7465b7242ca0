"""The bounds-checked build variant (-DQEQ_BOUNDS) compiles for sm_103a, exports
the same entry points and reports itself; the default build reports that it
has no checks (CPU: builds and loads, calls host-only entry points)."""

import ctypes
import subprocess

from paper_2503_21176_gb300 import _build


def _exported(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    return {ln.split()[-1] for ln in out.splitlines() if " T " in ln}


def _bounds_checked(path):
    b = ctypes.c_int32(-1)
    assert ctypes.CDLL(path).qeq_build_info(ctypes.byref(b)) == 0
    return b.value


def test_bounds_build_compiles_and_reports_itself():
    default, checked = _build.build(), _build.build(bounds=True)
    assert checked != default
    assert _bounds_checked(default) == 0
    assert _bounds_checked(checked) == 1
    assert _exported(checked) == _exported(default)
