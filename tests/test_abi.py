"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/ds.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
            if f.endswith(".h")]
    names = set()
    for h in hdrs:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(ds_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2310_07551_gb300 import build as b
    if not os.path.exists(b.LIB) and shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["ds_phi_setup", "ds_tucker", "ds_step", "ds_integrate", "ds_plan_create",
                 "ds_plan_destroy", "ds_plan_sync", "ds_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    L.ds_version.restype = ctypes.c_char_p
    assert b"sm_103a" in L.ds_version()
