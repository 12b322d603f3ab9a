"""fr_jv_noalloc, the allocation-free form of fr_jv.

Some callers cannot allocate device memory where they need the product (an
application whose allocator reserved the GPU up front, or code that must not
call cudaMalloc after start-up).  fr_jv_noalloc serves them from a fixed
static working array inside the library.  This test calls it through the C
ABI twice in a row, with different inputs, and checks each result against
the context-based fr_jv on the same inputs, within the FD-product tolerance
the other GPU tests use.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TOL_FD = 1e-6


def test_noalloc_jv_matches_fr_jv_on_two_calls():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1904_04825_gb300 as fr

    cases = [(3, 0, 7.5, 11), (2, 1, 0.0, 12)]   # (p, mesh seed, shift, z seed)
    for p, mseed, shift, zseed in cases:
        xe, ye = S.stretched_mesh(9, 7, seed=mseed)
        X, Y = S.point_coords(xe, ye, p)
        U0 = S.smooth_random_state(X, Y, seed=40 + p, amp=0.1)
        z0 = S.random_vector(U0.shape, zseed)
        ctx = fr.Context(xe, ye, p)
        U = torch.from_numpy(U0).cuda()
        z = torch.from_numpy(z0).cuda()
        R0 = ctx.empty()
        fr.fr_residual(ctx, U, R0)
        y_ref = ctx.empty()
        fr.fr_jv(ctx, U, R0, z, shift, y_ref)
        y = torch.full_like(y_ref, float("nan"))
        fr.fr_jv_noalloc(xe, ye, p, U, R0, z, shift, y)
        torch.cuda.synchronize()
        yr = y_ref.cpu().numpy()
        yn = y.cpu().numpy()
        assert np.all(np.isfinite(yn))
        assert np.linalg.norm(yn - yr) <= TOL_FD * np.linalg.norm(yr)
        ctx.close()


def test_noalloc_rejects_meshes_beyond_its_fixed_size():
    import torch
    import paper_1904_04825_gb300 as fr
    xe = np.linspace(0.0, 1.0, 4098)           # 4097 cells: one more than the limit
    ye = np.linspace(0.0, 1.0, 3)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(fr.FrError) as ei:
        fr.fr_jv_noalloc(xe, ye, 2, t, t.clone(), t.clone(), 0.0, t.clone())
    assert ei.value.code == fr.FR_ERR_INVALID_ARG
    assert "4096" in str(ei.value)
