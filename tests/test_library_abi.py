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
    assert o.block_columns == 0
    for kw, code in ((dict(block_columns=2), fr.FR_ERR_INVALID_ARG),
                     (dict(block_columns=1, block_precision=1), fr.FR_ERR_UNSUPPORTED)):   # FP32 columns: 3D only
        bad = fr.default_opts(**kw)
        assert fr.lib.fr_ctx_create(ctypes.byref(desc), 2, ctypes.byref(bad), ctypes.byref(h)) == code
    assert fr.lib.fr_residual(None, None, None, None) == fr.FR_ERR_INVALID_ARG
    assert fr.lib.fr_last_error(None) is not None


def test_3d_argument_checks_without_gpu(libpath):
    """fr_ctx_create_3d validates its mesh, degree and options on the host
    before any device call."""
    import numpy as np
    import paper_1904_04825_gb300 as fr
    h = ctypes.c_void_p()
    e3 = np.linspace(-1.0, 1.0, 3)
    dp = e3.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    desc = fr.fr_mesh3d_desc(2, 2, 2, dp, dp, dp)

    def create(d, p, **kw):
        o = fr.default_opts(**kw)
        return fr.lib.fr_ctx_create_3d(ctypes.byref(d), p, ctypes.byref(o), ctypes.byref(h))
    assert create(desc, 5, precond=0) == fr.FR_ERR_UNSUPPORTED          # degrees 1-4
    assert create(desc, 0, precond=0) == fr.FR_ERR_UNSUPPORTED
    assert create(desc, 3) == fr.FR_ERR_UNSUPPORTED                      # 320-row blocks: FP32/BF16 only
    assert create(desc, 4, block_precision=1) == fr.FR_ERR_UNSUPPORTED   # 625-row blocks not built
    assert create(desc, 2, block_columns=1) == fr.FR_ERR_UNSUPPORTED     # FP32 columns: reduced-precision blocks
    assert create(desc, 2, block_columns=1, precond=0, block_precision=1) == fr.FR_ERR_UNSUPPORTED
    assert create(desc, 2, block_columns=-1) == fr.FR_ERR_INVALID_ARG
    assert create(desc, 2, riemann=1) == fr.FR_ERR_UNSUPPORTED           # Rusanov only
    assert create(desc, 2, guess=2) == fr.FR_ERR_UNSUPPORTED
    assert create(desc, 2, body_force_x=0.1) == fr.FR_ERR_UNSUPPORTED
    assert create(desc, 2, m_max=64) == fr.FR_ERR_INVALID_ARG
    thin = fr.fr_mesh3d_desc(2, 2, 1, dp, dp, dp)
    assert create(thin, 2) == fr.FR_ERR_INVALID_ARG
    down = np.array([1.0, 0.0, -1.0])
    dd = down.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert create(fr.fr_mesh3d_desc(2, 2, 2, dp, dp, dd), 2) == fr.FR_ERR_INVALID_ARG
    assert fr.lib.fr_ctx_create_3d(None, 2, None, ctypes.byref(h)) == fr.FR_ERR_INVALID_ARG
    out = (ctypes.c_double * 3)()
    assert fr.lib.fr_dissipation_rate(None, None, 1.0, out, None) == fr.FR_ERR_INVALID_ARG
    assert fr.lib.fr_set_block_chunk(None, 1) == fr.FR_ERR_INVALID_ARG


def test_wrong_length_tensors_rejected_before_any_library_call(libpath):
    """The library takes vector lengths from the mesh and trusts the pointers,
    so the binding checks every tensor's length first (a shorter tensor would
    be read or written past its end).  Runs on the host: the check raises
    before any call into the library."""
    import types

    import numpy as np
    import torch

    import paper_1904_04825_gb300 as fr
    ne, np_ = 4, 9
    ctx = types.SimpleNamespace(handle=None, ndof=ne * 4 * np_, ne=ne, np=np_,
                                check=lambda rc, allow=(): rc)
    good = torch.zeros(ctx.ndof, dtype=torch.float64)
    short = torch.zeros(ctx.ndof - 1, dtype=torch.float64)
    # the first tensor argument is the wrong one (later ones would fail the
    # CUDA-tensor check on this GPU-less host)
    calls = [
        lambda: fr.fr_residual(ctx, short, good),
        lambda: fr.fr_jv(ctx, short, good, good, 0.0, good),
        lambda: fr.ejacobi_factor(ctx, short, None, 1.0),
        lambda: fr.ejacobi_apply(ctx, short, good),
        lambda: fr.gmres_solve(ctx, short, good, 0.0, good, good),
        lambda: fr.step_row(ctx, 3, 0.1, short),
        lambda: fr.step_esdirk(ctx, 3, 0.1, short),
        lambda: fr.step_bdf2(ctx, 0.1, short, good, False),
        lambda: fr.step_ssprk3(ctx, 0.1, short),
        lambda: fr.fr_vortex_error(ctx, short, 0.0),
    ]
    for call in calls:
        with pytest.raises(ValueError):
            call()
    xe = np.linspace(0.0, 1.0, 3)   # 2 x 2 elements, p = 2: 144 values
    s2 = torch.zeros(143, dtype=torch.float64)
    g2 = torch.zeros(144, dtype=torch.float64)
    with pytest.raises(ValueError):
        fr.fr_jv_noalloc(xe, xe, 2, s2, g2, g2, 0.0, g2)
    with pytest.raises(ValueError):       # degree 3 needs 256 values
        fr.fr_jv_noalloc(xe, xe, 3, g2, g2, g2, 0.0, g2)
