"""The C ABI library builds for sm_103a, loads, and exports every declared entry point (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(spalu_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_14193_gb300 import build, load_library
    build.build()
    return load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    from paper_2408_14193_gb300.spalu import SIGNATURES
    assert sorted(n for n, _, _ in SIGNATURES) == _declared()


def test_status_strings_and_defaults(lib):
    import ctypes

    from paper_2408_14193_gb300.spalu import Options
    assert lib.spalu_status_string(0) == b"ok"
    assert lib.spalu_status_string(-3) == b"zero pivot in an LU"
    o = Options.default()
    assert o.eps_id == 1e-8 and o.p_oversample == 5 and o.h0 == 16 and o.near_radius == 2
    assert o.gmres_tol == 1e-10 and o.spars_ctas == 4 and o.schur_tc == 1 and o.leaf_bwd == -1
    # argument checks that need no device: bad grid shape, bad leaf pitch, null output
    h = ctypes.c_void_p()
    assert lib.spalu_nd_build_grid(20, 31, 16, None, ctypes.byref(h)) == -1
    assert lib.spalu_nd_build_grid(31, 31, 8, None, ctypes.byref(h)) == -7
    assert lib.spalu_nd_build_grid(31, 31, 16, None, None) == -1
    assert lib.spalu_factor_create(None, None, None) == -1
    assert lib.spalu_solve(None, None, None, 1, 1, None) == -1


def test_library_is_built_for_sm103a():
    from paper_2408_14193_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
