"""fr_jv_noalloc, the allocation-free form of fr_jv.

Some callers cannot allocate device memory where they need the product (an
application whose allocator reserved the GPU up front, or code that must not
call cudaMalloc after start-up).  fr_jv_noalloc serves them from a fixed
static working array inside the library.  This test calls it through the C
ABI several times in a row, with different inputs and options, and checks
each result against the FP64 oracle's FD product and against the
context-based fr_jv on the same inputs, within the FD-product tolerance the
other GPU tests use.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import Problem, fd_jv

pytestmark = pytest.mark.gpu

TOL_FD = 1e-6


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_noalloc_jv_matches_oracle_and_fr_jv_on_calls_in_a_row():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1904_04825_gb300 as fr

    # (p, mesh seed, shift, z seed, options): the scaled FD step with the
    # Rusanov flux twice, the paper's Roe flux, and a fixed FD step
    cases = [(3, 0, 7.5, 11, {}), (2, 1, 0.0, 12, {}), (4, 2, 3.0, 13, {"riemann": 1}),
             (3, 3, 1.0, 14, {"eps_fixed": 1e-6})]
    for p, mseed, shift, zseed, kw in cases:
        xe, ye = S.stretched_mesh(9, 7, seed=mseed)
        X, Y = S.point_coords(xe, ye, p)
        U0 = S.smooth_random_state(X, Y, seed=40 + p, amp=0.1)
        z0 = S.random_vector(U0.shape, zseed)
        opts = fr.default_opts(**kw)
        prob = Problem(Mesh(xe, ye), p, riemann="roe" if kw.get("riemann") == 1 else "rusanov")
        R0o = prob.R(U0)
        yo = fd_jv(prob, U0, R0o, z0, shift, eps_fixed=kw.get("eps_fixed") or None)

        ctx = fr.Context(xe, ye, p, opts)
        U = torch.from_numpy(U0).cuda()
        z = torch.from_numpy(z0).cuda()
        R0 = ctx.empty()
        fr.fr_residual(ctx, U, R0)
        y_ref = ctx.empty()
        fr.fr_jv(ctx, U, R0, z, shift, y_ref)
        y = torch.full_like(y_ref, float("nan"))
        fr.fr_jv_noalloc(xe, ye, p, U, R0, z, shift, y, opts=opts)
        torch.cuda.synchronize()
        yn = y.cpu().numpy()
        assert np.all(np.isfinite(yn))
        assert _rel(yn, yo) <= TOL_FD, (p, kw, _rel(yn, yo))
        assert _rel(yn, y_ref.cpu().numpy()) <= TOL_FD
        ctx.close()


def test_noalloc_rejects_meshes_beyond_its_fixed_size_and_other_operators():
    import torch
    import paper_1904_04825_gb300 as fr
    xe = np.linspace(0.0, 1.0, 4098)           # 4097 cells: one more than the limit
    ye = np.linspace(0.0, 1.0, 3)
    n = 4097 * 2 * 4 * 9
    t = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(4)]
    with pytest.raises(fr.FrError) as ei:
        fr.fr_jv_noalloc(xe, ye, 2, t[0], t[1], t[2], 0.0, t[3])
    assert ei.value.code == fr.FR_ERR_INVALID_ARG
    assert "4096" in str(ei.value)
    # viscous or FP32-linear-parts options name another operator than this product
    xe = np.linspace(0.0, 1.0, 5)
    n = 16 * 4 * 9
    t = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(4)]
    for kw in ({"mu": 1e-3}, {"jv_precision": 1}):
        with pytest.raises(fr.FrError) as ei:
            fr.fr_jv_noalloc(xe, xe, 2, t[0], t[1], t[2], 0.0, t[3], opts=fr.default_opts(**kw))
        assert ei.value.code == fr.FR_ERR_UNSUPPORTED


def test_noalloc_refuses_stream_capture():
    """The call copies host edge arrays on the stream, which a captured graph
    could not replay: on a capturing stream it returns FR_ERR_UNSUPPORTED
    and records nothing."""
    import torch
    import paper_1904_04825_gb300 as fr
    xe = np.linspace(0.0, 1.0, 5)
    n = 16 * 4 * 9
    t = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(4)]
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(g):
        try:
            fr.fr_jv_noalloc(xe, xe, 2, t[0], t[1], t[2], 0.0, t[3])
        except fr.FrError as e:
            codes.append(e.code)
        t[3].add_(1.0)   # one captured kernel, so the graph is not empty
    assert codes == [fr.FR_ERR_UNSUPPORTED]
