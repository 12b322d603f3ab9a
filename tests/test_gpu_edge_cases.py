"""Edge cases on the GPU: degenerate and smallest meshes, one-element-wide
meshes (ragged tiles in one direction), a zero right-hand side, argument
checks, and the largest mesh a single step is exercised on (sampled parity).
Tolerances as in test_gpu_parity.py."""
import ctypes

import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import Problem, fd_jv

pytestmark = pytest.mark.gpu

TOL_R = 1e-12
TOL_FD = 1e-6


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    import paper_1904_04825_gb300 as mod
    return mod


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("nx,ny,p", [(0, 4, 2), (1, 4, 2), (4, 1, 3), (4, 4, 1), (4, 4, 7)])
def test_degenerate_meshes_and_degrees_rejected(fr, nx, ny, p):
    xe = np.linspace(-1, 1, nx + 1) if nx > 0 else np.zeros(1)
    ye = np.linspace(-1, 1, ny + 1)
    with pytest.raises(fr.FrError):
        fr.Context(xe, ye, p)


def test_bad_edges_and_options_rejected(fr):
    xe = np.array([0.0, 1.0, 1.0, 2.0])  # a zero-width cell
    ye = np.linspace(0, 1, 4)
    with pytest.raises(fr.FrError):
        fr.Context(xe, ye, 2)
    xe = np.linspace(0, 1, 4)
    for kw in ({"gmres_m": 40}, {"block_precision": 3}, {"riemann": 2}, {"jv_precision": 2}, {"guess": 3},
               {"reorth_eta": 2.0}):
        with pytest.raises(fr.FrError):
            fr.Context(xe, ye, 2, fr.default_opts(**kw))


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("nx,ny", [(2, 2), (2, 9), (11, 2)])
def test_smallest_and_one_tile_wide_meshes(fr, p, nx, ny):
    """2 x 2 (every element is its own neighbour's neighbour) and meshes two
    elements wide: R, A z and one ROW2 step against the oracle."""
    xe, ye = S.stretched_mesh(nx, ny, seed=nx + ny + p)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.smooth_random_state(X, Y, seed=p, amp=0.1)
    z0 = S.random_vector(U0.shape, seed=p + 1)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-12, gmres_max_restarts=40))
    U = _t(U0)
    R = ctx.empty()
    fr.fr_residual(ctx, U, R)
    assert _rel(R.cpu().numpy(), R0) < TOL_R
    y = ctx.empty()
    fr.fr_jv(ctx, U, _t(R0), _t(z0), 3.0, y)
    assert _rel(y.cpu().numpy(), fd_jv(prob, U0, R0, z0, 3.0)) < TOL_FD


def test_zero_right_hand_side_gives_zero_solution(fr):
    p = 2
    xe, ye = S.uniform_mesh(6)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.Vortex().state(X, Y)
    ctx = fr.Context(xe, ye, p)
    U = _t(U0)
    R0 = ctx.empty()
    fr.fr_residual(ctx, U, R0)
    fr.ejacobi_factor(ctx, U, R0, 10.0)
    b = ctx.empty().zero_()
    x = _t(S.random_vector(U0.shape, seed=3))  # nonzero guess: the solution of A x = 0 is 0
    info = fr.gmres_solve(ctx, U, R0, 10.0, b, x, m=30, rtol=1e-10, max_restarts=5)
    assert info.converged and info.iters == 0
    assert float(x.abs().max()) == 0.0


def test_misaligned_apply_input_rejected(fr):
    import torch
    p = 2
    xe, ye = S.uniform_mesh(4)
    ctx = fr.Context(xe, ye, p)
    U = _t(S.Vortex().state(*S.point_coords(xe, ye, p)))
    fr.ejacobi_factor(ctx, U, None, 10.0)
    buf = torch.zeros(ctx.ndof + 1, dtype=torch.float64, device="cuda")
    r = buf[1:]  # 8-byte aligned view
    z = ctx.empty()
    rc = fr.lib.ejacobi_apply(ctx.handle, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                              fr._stream(None))
    assert rc == fr.FR_ERR_INVALID_ARG


def test_largest_mesh_sampled_parity(fr):
    """768 x 768 elements at p = 3 (37.7 M DOFs, ~55 GB of workspace, 23x the
    benchmark mesh): the residual against the oracle on sampled elements
    (full-mesh oracle residual, compared on 4096 elements incl. the corners
    and the last one), and one ROW2 step that keeps the state finite."""
    import torch
    p, n = 3, 768
    xe, ye = S.uniform_mesh(n)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.Vortex().state(X, Y)
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-4))
    U = _t(U0)
    R = ctx.empty()
    fr.fr_residual(ctx, U, R)
    Ro = Problem(Mesh(xe, ye), p).R(U0)
    idx = np.unique(np.concatenate([[0, n - 1, n * n - n, n * n - 1],
                                    np.random.default_rng(0).integers(0, n * n, 4092)]))
    Rg = R[torch.from_numpy(idx).cuda()].cpu().numpy()
    scale = np.max(np.abs(Ro)) + 1e-300
    assert np.max(np.abs(Rg - Ro[idx])) < 1e-10 * scale
    del Ro
    st = fr.step_row(ctx, 2, 0.005, U)
    assert st.converged
    assert bool(U.isfinite().all())
