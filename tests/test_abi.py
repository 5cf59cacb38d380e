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


def test_every_entry_point_rejects_a_null_lattice_on_the_host(lib):
    """Each compute entry point checks its arguments before any CUDA call: a NULL lattice (or
    field) is TM_ERR_ARG with a message naming the function, on a machine without a GPU."""
    ERR_ARG = 1
    calls = {
        "tm_apply_D": lambda: lib.tm_apply_D(None, None, None, 1, 0, 1, None),
        "tm_apply_hopping_eo": lambda: lib.tm_apply_hopping_eo(None, 0, None, None, 0, 18, 1, None),
        "tm_apply_Mee_inv": lambda: lib.tm_apply_Mee_inv(None, None, None, 1, 0, 1, None),
        "tm_pack_half": lambda: lib.tm_pack_half(None, 0, None, None, 1, None),
        "tm_unpack_half": lambda: lib.tm_unpack_half(None, 0, None, None, 1, None),
        "tm_set_gauge": lambda: lib.tm_set_gauge(None, None, None),
        "tm_lattice_set_params": lambda: lib.tm_lattice_set_params(None, 0.16, 0.01),
        "tm_solve_cg": lambda: lib.tm_solve_cg(None, None, None, 1, None, None, None),
        "tm_solve_bicgstab": lambda: lib.tm_solve_bicgstab(None, None, None, 1, None, None, None),
        "tm_solve_mr": lambda: lib.tm_solve_mr(None, None, None, 1, None, None, None),
        "tm_solve_normal": lambda: lib.tm_solve_normal(None, None, None, None, None, None),
        "tm_chrono_guess": lambda: lib.tm_chrono_guess(None, None, None, 0, None, 1, None),
        "tm_apply_Dh": lambda: lib.tm_apply_Dh(None, None, None, 0.15, 0.19, 1, None),
        "tm_solve_doublet": lambda: lib.tm_solve_doublet(None, None, None, 0.15, 0.19, None, None, None),
        "tm_meson_contract": lambda: lib.tm_meson_contract(None, None, None, None),
        "tm_correlator": lambda: lib.tm_correlator(None, None, None, 1, None, None),
        "tm_solve_cg_batch": lambda: lib.tm_solve_cg_batch(None, 0, None, None, None),
    }
    for name, call in calls.items():
        assert call() == ERR_ARG, name
        assert name.encode() in lib.tm_last_error(), (name, lib.tm_last_error())
    fn = lib.tm_apply_D_noalloc
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 3 + [ctypes.c_void_p]
    fn.restype = ctypes.c_int
    assert fn(None, None, None, 1, 0, 1, None) == ERR_ARG
    assert b"tm_apply_D_noalloc" in lib.tm_last_error()


def test_batched_solver_checks_its_parameters_on_the_host(lib):
    """tm_solve_cg_batch rejects parameters it does not support before it reads a system: the
    mode (reliable updates only), the sloppy storage (FP32 or FP16) and link form (18/12/8), tol,
    max_iter, delta, and initial guesses."""
    ERR_ARG, UNSUPPORTED = 1, 10
    systems = (tm.TmSystem * 2)()

    def run(**kw):
        p = tm.CGParams()
        lib.tm_cg_params_default(ctypes.byref(p))
        p.mode = 2  # TM_CG_RELIABLE
        for k, v in kw.items():
            setattr(p, k, v)
        return lib.tm_solve_cg_batch(systems, 2, ctypes.byref(p), None, None), lib.tm_last_error()

    assert run(mode=0) == (UNSUPPORTED, b"tm_solve_cg_batch: mode must be TM_CG_RELIABLE")
    assert run(sloppy_prec=0)[0] == ERR_ARG
    assert run(sloppy_link=9)[0] == ERR_ARG
    assert run(tol=0.0)[0] == ERR_ARG
    assert run(max_iter=0)[0] == ERR_ARG
    assert run(delta=1.0)[0] == ERR_ARG
    assert run(use_x0=1)[0] == UNSUPPORTED
    # parameters accepted: the first system's NULL members are the next error
    st, msg = run()
    assert st == ERR_ARG and b"system 0 has a NULL member" in msg
