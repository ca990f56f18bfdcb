"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/stg.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "stg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_02690_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("stg_setup", "stg_vcycle", "stg_gmres_solve", "stg_apply_jacobian", "stg_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2210_02690_gb300 as pkg
    assert sorted(pkg.EXPORTED) == declared_symbols()


def test_options_default_without_gpu(lib):
    import paper_2210_02690_gb300 as pkg
    pkg.load_library()
    o = pkg.make_options()
    assert (o.nu1, o.nu2, o.omega, o.gamma1, o.gamma2, o.gmres_restart) == (4, 4, 0.7, 35.0, 35.0, 30)
    assert abs(o.gmres_rtol - 1e-8) < 1e-20
    assert lib.stg_options_default(None) == 1
