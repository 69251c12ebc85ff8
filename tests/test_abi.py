"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no device calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

from conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(clbm3?_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2301_01868_gb300 import _build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        if not os.path.exists(_build.LIB):
            pytest.skip("no nvcc to build the library")
        return _build.LIB
    return _build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("clbm_create_grid", "clbm_set_case", "clbm_step", "clbm_moments",
                 "clbm_residual", "clbm_destroy", "clbm3_create_grid", "clbm3_step",
                 "clbm3_moments", "clbm3_totals"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_workspace_query_is_host_only(libpath):
    from paper_2301_01868_gb300 import clbm
    b21 = clbm.workspace_bytes(21, clbm.FP32, 64, 256)
    b9 = clbm.workspace_bytes(9, clbm.FP32, 64, 256)
    b64 = clbm.workspace_bytes(21, clbm.FP64, 64, 256)
    # two state buffers dominate: Q * (n1 + 2h) * ld * bytes each
    assert b21 >= 2 * 21 * 70 * 256 * 4 and b9 >= 2 * 9 * 66 * 256 * 4
    assert b64 > b21
    with pytest.raises(clbm.ClbmError):
        clbm.workspace_bytes(21, clbm.FP32, 2, 8)
