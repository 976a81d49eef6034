"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every declared symbol."""
import ctypes
import os
import re

import paper_1606_05474_b300 as hp
from paper_1606_05474_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "helios.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(helios_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    so = hp.build()
    lib = ctypes.CDLL(so)
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(_lib.EXPORTS) <= set(names)


def test_version_and_default_params():
    lib = _lib.load()
    assert lib.helios_version() == 100
    p = hp.default_params()
    assert (p.D, p.dtau_iso, p.w0_pure, p.tol, p.n_scat) == (2.0, 1e-4, 1e-6, 1e-7, 4)
    assert (p.fpre_num, p.fpre_exp, p.osc_down, p.osc_up) == (1e5, 0.9, 0.67, 1.1)


def test_null_arguments_are_rejected_without_a_device():
    lib = _lib.load()
    assert lib.helios_create(None, 0) == _lib.HELIOS_EINVAL
    assert lib.helios_plan_create(None, None, None, 0, None, None) == _lib.HELIOS_EINVAL
    assert b"null" in lib.helios_last_error()
    assert lib.helios_flux_sweep(None, None, 0, 0, None, None, None, None, None, None) == _lib.HELIOS_EINVAL
    assert lib.helios_solve_re(None, None, None, None, None) == _lib.HELIOS_EINVAL
