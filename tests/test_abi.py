"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/bindesc.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bindesc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(bd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2108_08380_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["bd_create", "bd_destroy", "bd_bad_params_create", "bd_hs_params_create",
                 "bd_integral", "bd_bad_describe", "bd_hashsift_describe", "bd_match"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(bd_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_header(libpath):
    import paper_2108_08380_gb300 as bd
    L = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(L, n)
    assert sorted(bd.exported_names()) == declared_functions()


def test_host_only_calls_without_a_gpu(libpath):
    """Pure host queries work without a device."""
    import paper_2108_08380_gb300 as bd
    assert bd.lib().bd_scratch_bytes_bad(640, 480) > 641 * 481 * 4
    assert bd.lib().bd_scratch_bytes_bad(0, 10) == 0
    assert bd.lib().bd_scratch_bytes_hashsift(1000) >= 1000 * 128 * 4
    assert bd.lib().bd_last_error(None) == b"null context"
