"""The C-ABI library builds, loads and exports every symbol its header declares (no GPU needed)."""
import ctypes
import glob
import os

import pytest

from paper_1012_2677_gb300 import ljmd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    lib = ljmd.load()
    headers = glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert headers
    for h in headers:
        names = ljmd.declared_symbols(h)
        assert names, h
        for name in names:
            assert hasattr(lib, name), "%s declared in %s but not exported" % (name, os.path.basename(h))


def test_host_only_entry_points():
    assert ljmd.ljmd_version() >= 100
    assert ljmd.ljmd_strerror(ljmd.LJ_EINVAL) == "invalid argument"
    assert ljmd.ljmd_strerror(12345) == "unknown status"


def test_argument_checks_before_any_device_work():
    lib = ljmd.load()
    p = ljmd.ljmd_params(1.0, 1.0, 2.5, 0.5, 0, 0, 1, 0)
    assert lib.ljmd_create(None, ctypes.byref(p), ljmd.LJ_MIXED, None) == ljmd.LJ_EINVAL
    h = ctypes.c_void_p()
    for bad in (ljmd.ljmd_params(1.0, 1.0, -2.5, 0.5, 0, 0, 1, 0), ljmd.ljmd_params(1.0, 1.0, 2.5, -0.1, 0, 0, 1, 0),
                ljmd.ljmd_params(1.0, 1.0, 2.5, 0.5, 7, 0, 1, 0), ljmd.ljmd_params(1.0, 1.0, 2.5, 0.5, 0, 0, 1, 3)):
        assert lib.ljmd_create(ctypes.byref(h), ctypes.byref(bad), ljmd.LJ_MIXED, None) == ljmd.LJ_EINVAL
    assert lib.ljmd_create(ctypes.byref(h), ctypes.byref(p), 5, None) == ljmd.LJ_EINVAL
    for fn, args in (("ljmd_step", (None, 0.005, 1)), ("ljmd_compute_forces", (None,)),
                     ("ljmd_build_pairlist", (None, 2.5, 0.5)), ("ljmd_get_stats", (None, None))):
        assert getattr(lib, fn)(*args) == ljmd.LJ_EINVAL
    assert lib.ljmd_set_wait_budget(-1) == ljmd.LJ_EINVAL


def test_product_path_has_no_oracle_dependency():
    """The CUDA library and its binding never import, include or link the oracle."""
    import re
    pkg = os.path.join(ROOT, "paper_1012_2677_gb300")
    pat = re.compile(r"(^\s*(import|from)\s+oracle\b|ljoracle|#include\s*[<\"][^>\"]*oracle)", re.M)
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            assert not pat.search(open(path).read()), path


def test_binding_constants_match_the_header():
    """Every #define LJ_* of include/ljmd.h has the same value in the binding."""
    import re
    hdr = open(os.path.join(ROOT, "include", "ljmd.h")).read()
    defs = dict(re.findall(r"^#define (LJ_[A-Z0-9_]+) \(?(-?\d+)\)?", hdr, flags=re.M))
    assert len(defs) >= 23  # status codes, device status bits, forms, list forms, rules, truncations
    for name, value in defs.items():
        assert getattr(ljmd, name) == int(value), name
