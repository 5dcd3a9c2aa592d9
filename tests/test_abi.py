"""The C-ABI library builds for sm_103a, loads, and exports every entry point the header declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(swm_\w+)\s*\(", src))
    # typedef'd function pointer types are not entry points
    names -= set(re.findall(r"typedef[^;]*\(\s*\*\s*(swm_\w+)\s*\)", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2410_03060_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("swm_create", "swm_set_cloud", "swm_build", "swm_solve", "swm_rcs_bistatic",
                     "swm_rcs_monostatic", "swm_far_field"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(swm_\w+)\b", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_the_header(libpath):
    from paper_2410_03060_gb300 import swm
    assert set(swm.EXPORTED) == set(declared_functions())
    assert swm.swm_version().startswith("swm")
