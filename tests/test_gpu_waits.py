"""Bounded waits: a wait of the element-Jacobi apply that runs out ends in
FR_ERR_TIMEOUT on the host, with nothing left in flight on the GPU.

The apply's CTAs wait on shared-memory barriers for the bulk copies of their
elements.  The test hook fr_set_wait_test makes CTA 0 leave its first
element's copies unissued (a barrier that nothing completes) and lowers the
poll limit, so the wait runs out quickly; the CTA flags the context, waits
(bounded) for the copies it did issue and leaves.  The GMRES call then
reports FR_ERR_TIMEOUT.  A fresh context on the same GPU afterwards solves
normally, which shows the GPU is left clean.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _problem(fr, prec=0):
    import torch
    xe, ye = S.uniform_mesh(8)
    X, Y = S.point_coords(xe, ye, 2)
    U = torch.from_numpy(S.Vortex().state(X, Y)).cuda()
    ctx = fr.Context(xe, ye, 2, fr.default_opts(block_precision=prec))
    R0 = ctx.empty()
    fr.fr_residual(ctx, U, R0)
    shift = 20.0
    fr.ejacobi_factor(ctx, U, R0, shift)
    b = torch.from_numpy(S.random_vector(ctx.shape, 3)).cuda()
    return ctx, U, R0, shift, b


@pytest.mark.parametrize("prec", [0, 2])
def test_apply_wait_runs_out_and_gmres_reports_timeout(prec):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1904_04825_gb300 as fr
    ctx, U, R0, shift, b = _problem(fr, prec)
    fr.fr_set_wait_test(ctx, polls=2000, skip_first_copy=True)
    x = torch.zeros_like(b)
    with pytest.raises(fr.FrError) as e:
        fr.gmres_solve(ctx, U, R0, shift, b, x, m=10, rtol=1e-10, max_restarts=2)
    assert e.value.code == fr.FR_ERR_TIMEOUT
    torch.cuda.synchronize()
    ctx.close()

    ctx, U, R0, shift, b = _problem(fr, prec)
    x = torch.zeros_like(b)
    info = fr.gmres_solve(ctx, U, R0, shift, b, x, m=30, rtol=1e-10, max_restarts=20)
    assert info.converged and np.all(np.isfinite(x.cpu().numpy()))
    ctx.close()


def test_wait_test_hook_rejects_bad_arguments():
    import paper_1904_04825_gb300 as fr
    xe, ye = S.uniform_mesh(4)
    ctx = fr.Context(xe, ye, 2)
    assert fr.lib.fr_set_wait_test(ctx.handle, 10, 2) == fr.FR_ERR_INVALID_ARG
    assert fr.fr_set_wait_test(ctx, 0, False) == 0
    ctx.close()
