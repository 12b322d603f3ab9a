"""The C-ABI library builds, loads and exports every function the header declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for f in sorted(os.listdir(HEADER_DIR)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    b = __graft_entry__._builder()
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("fr_residual", "fr_jv", "ejacobi_factor", "ejacobi_apply", "gmres_solve",
                     "step_row", "step_esdirk", "step_bdf2", "fr_ctx_create", "fr_ctx_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_exposes_c_names(libpath):
    import paper_1904_04825_gb300 as fr
    for n in ("fr_residual", "fr_jv", "ejacobi_factor", "ejacobi_apply", "gmres_solve",
              "step_row", "step_esdirk", "step_bdf2"):
        assert callable(getattr(fr, n))


def test_defaults_and_argument_checks_without_gpu(libpath):
    """Option defaults and argument validation run on the host only."""
    import paper_1904_04825_gb300 as fr
    o = fr.default_opts()
    assert o.gamma == 1.4 and o.m_max == 30 and o.eps_rel == 1e-7 and o.precond == 1
    assert o.reorth_eta == 1.0 / 64.0
    po = fr.default_ptc_opts()
    assert po.dtau_max == 1e20 and po.tol_lin == 0.1 and po.reject_above == 0.1
    h = ctypes.c_void_p()
    # degree outside the compiled set / too-small mesh are rejected before any device call
    import numpy as np
    xe = np.linspace(0, 1, 3)
    desc = fr.fr_mesh_desc(2, 2, xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    assert fr.lib.fr_ctx_create(ctypes.byref(desc), 7, None, ctypes.byref(h)) == fr.FR_ERR_UNSUPPORTED
    desc1 = fr.fr_mesh_desc(1, 2, xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    assert fr.lib.fr_ctx_create(ctypes.byref(desc1), 2, None, ctypes.byref(h)) == fr.FR_ERR_INVALID_ARG
    bad = fr.default_opts(m_max=64)
    assert fr.lib.fr_ctx_create(ctypes.byref(desc), 2, ctypes.byref(bad), ctypes.byref(h)) == fr.FR_ERR_INVALID_ARG
    assert fr.lib.fr_residual(None, None, None, None) == fr.FR_ERR_INVALID_ARG
    assert fr.lib.fr_last_error(None) is not None
