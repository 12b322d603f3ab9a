"""Resume from a checkpoint on the GPU: stepping on from a saved and
reloaded state (with BDF2's previous state) in a fresh context reproduces
the uninterrupted run bit for bit."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    import paper_1904_04825_gb300 as mod
    return mod


def _setup():
    import torch
    p = 2
    xe, ye = S.uniform_mesh(8)
    X, Y = S.point_coords(xe, ye, p)
    return p, (xe, ye), torch.from_numpy(S.Vortex().state(X, Y)).cuda()


def test_bdf2_resume_is_bit_identical(fr, tmp_path):
    import torch
    from paper_1904_04825_gb300 import checkpoint as ck
    p, edges, U0 = _setup()
    po = fr.default_ptc_opts(tol_nl=1e-8, tol_lin=1e-2)
    dt = 0.1
    # uninterrupted: three steps
    ctx = fr.Context(*edges, p)
    U, Up = U0.clone(), torch.empty_like(U0)
    for k in range(3):
        fr.step_bdf2(ctx, dt, U, Up, k == 0, po)
    ctx.close()
    # one step, checkpoint, a fresh context, two more steps
    ctx = fr.Context(*edges, p)
    V, Vp = U0.clone(), torch.empty_like(U0)
    fr.step_bdf2(ctx, dt, V, Vp, True, po)
    ctx.close()
    ck.save(str(tmp_path / "c"), V, t=dt, step=1, scheme="BDF2", p=p, edges=edges, U_prev=Vp)
    del V, Vp
    W, Wp, h = ck.load(str(tmp_path / "c"))
    assert h["step"] == 1 and Wp is not None
    ctx = fr.Context(*edges, p)
    for _ in range(2):
        fr.step_bdf2(ctx, dt, W, Wp, False, po)
    assert torch.equal(W, U) and torch.equal(Wp, Up)


def test_row3_resume_is_bit_identical(fr, tmp_path):
    import torch
    from paper_1904_04825_gb300 import checkpoint as ck
    p, edges, U0 = _setup()
    dt = 0.1
    ctx = fr.Context(*edges, p, fr.default_opts(tol_lin=1e-8))
    U = U0.clone()
    for _ in range(2):
        fr.step_row(ctx, 3, dt, U)
    ctx2 = fr.Context(*edges, p, fr.default_opts(tol_lin=1e-8))
    V = U0.clone()
    fr.step_row(ctx2, 3, dt, V)
    ck.save(str(tmp_path / "r"), V, t=dt, step=1, scheme="ROW3", p=p, edges=edges)
    W, none, _ = ck.load(str(tmp_path / "r"))
    ctx3 = fr.Context(*edges, p, fr.default_opts(tol_lin=1e-8))
    fr.step_row(ctx3, 3, dt, W)
    assert none is None and torch.equal(W, U)
    assert float((U - U0).abs().max()) > 0.0
