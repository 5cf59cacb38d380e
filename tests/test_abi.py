"""The C ABI library on the CPU: it builds, loads, exports every function that
include/tm.h declares, and its host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_0905_3331_gb300 import build as libbuild
from paper_0905_3331_gb300 import tm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*\s+)+\**\s*(tm_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return tm.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ("tm_lattice_create", "tm_set_gauge", "tm_apply_D", "tm_apply_hopping_eo",
               "tm_apply_Mee_inv", "tm_solve_cg"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(tm.exported_symbols()) <= declared_functions()


def test_host_side_argument_checks(lib):
    h = ctypes.c_void_p()
    assert lib.tm_lattice_create(5, 4, 0.16, 0.01, ctypes.byref(h)) == 2  # TM_ERR_ODD_EXTENT
    assert b"must be even" in lib.tm_last_error()
    assert lib.tm_lattice_create(4, 0, 0.16, 0.01, ctypes.byref(h)) == 2
    assert lib.tm_lattice_create(4, 4, 0.16, 0.01, None) == 1  # TM_ERR_ARG
    assert lib.tm_lattice_create(4, 4, float("nan"), 0.01, ctypes.byref(h)) == 1
    assert lib.tm_apply_D(None, None, None, 1, 0, 1, None) == 1
    assert lib.tm_solve_cg(None, None, None, 1, None, None, None) == 1
    assert lib.tm_lattice_destroy(None) == 0
    assert lib.tm_volume(None) == 0
    assert lib.tm_set_hop_threads(None, 0, 18, 2) == 1
    assert lib.tm_get_hop_threads(None, 0, 18) == 0


def test_cg_params_defaults(lib):
    p = tm.CGParams()
    lib.tm_cg_params_default(ctypes.byref(p))
    assert (p.tol, p.max_iter, p.mode, p.sloppy_prec, p.sloppy_link, p.delta, p.use_x0,
            p.flavour, p.update_prec) == (1e-10, 100000, 0, 1, 12, 0.1, 0, 1, 0)


def test_launch_counter(lib):
    lib.tm_reset_launch_count()
    assert lib.tm_launch_count() == 0
