"""Reduced-precision element-Jacobi blocks (FP32 inversion, FP32 or BF16
storage) against the FP64 oracle.

The preconditioner's own error is stated against the oracle's FP64 blocks.
The FP32-class inversion runs its trailing updates on the tensor cores with
every operand split into two TF32 halves (about 22 bits of it, an effective
unit roundoff of 2^-23 = 1.2e-7, twice that of FP32); it leaves about
n u cond(M) relative error in M^-1 r, bound 2e-4 (measured 1.0e-4 on the
walled channel's blocks of condition 4e5); BF16 storage rounds every entry
to 8 bits (u_bf16 = 3.9e-3), bound 3e-2.  The converged linear solves and the
end-of-run state do not depend on the preconditioner: with tol_lin = 1e-12
they match the FP64 oracle to 1e-9 like the FP64 path."""
import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import ElementJacobi, Problem, element_blocks
from oracle.steppers import SolverOpts
from oracle.steppers import step_row as o_row
from oracle.tableaus import ROW

pytestmark = pytest.mark.gpu

PREC_TOL = {1: 2e-4, 2: 3e-2}


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    import paper_1904_04825_gb300 as mod
    return mod


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_reduced_precision_apply_error(fr, prec, p):
    xe, ye = S.stretched_mesh(6, 5, seed=p)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.smooth_random_state(X, Y, seed=21, amp=0.1)
    r0 = S.random_vector(U0.shape, 22)
    shift = 40.0
    ctx = fr.Context(xe, ye, p, fr.default_opts(block_precision=prec))
    fr.ejacobi_factor(ctx, _t(U0), None, shift)
    z = ctx.empty()
    fr.ejacobi_apply(ctx, _t(r0), z)
    zo = ElementJacobi(element_blocks(Problem(Mesh(xe, ye), p), U0, shift))(r0)
    err = np.linalg.norm(z.cpu().numpy() - zo) / np.linalg.norm(zo)
    assert err < PREC_TOL[prec], err


@pytest.mark.parametrize("prec", [1, 2])
def test_reduced_precision_run_matches_fp64_oracle(fr, prec):
    """20 x 20, p = 2 vortex, 10 ROW2 steps of 0.05 at tol_lin = 1e-12."""
    p = 2
    xe, ye = S.uniform_mesh(20)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-12, gmres_max_restarts=60,
                                                block_precision=prec))
    U = _t(U0)
    Uo = U0.copy()
    it = 0
    for _ in range(10):
        st = fr.step_row(ctx, 2, 0.05, U)
        assert st.converged
        it += st.gmres_iters
        Uo, _ = o_row(prob, ROW[2](), 0.05, Uo, SolverOpts(tol_lin=1e-12, m=30, max_restarts=60))
    assert np.linalg.norm(U.cpu().numpy() - Uo) / np.linalg.norm(Uo) < 1e-9


# ------------------------------------------------- FP32 linear parts of A z --
# jv_precision = 1: the divergence, correction and z-traces of
# R(U + eps z) - R(U) run in FP32 on the flux differences.  Their rounding
# (u_32 = 6e-8) is amplified by the cancellation inside the derivative
# (coefficients up to (p+1)^2/2, smooth differences) by at most ~100, so A z
# matches the oracle's FP64 finite-difference product to 1e-5 relative L2;
# a wrong sign, index or missing term errs by O(1).
TOL_JV32 = 1e-5


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("nx,ny", [(5, 4), (13, 11), (24, 7)])
def test_mixed_jv_matches_oracle(fr, p, nx, ny):
    from oracle.jfnk import fd_jv
    xe, ye = S.stretched_mesh(nx, ny, seed=nx * p)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.smooth_random_state(X, Y, seed=p, amp=0.1)
    z0 = S.random_vector(U0.shape, seed=nx + p)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    ctx = fr.Context(xe, ye, p, fr.default_opts(jv_precision=1))
    U, z, Rg = _t(U0), _t(z0), _t(R0)
    y = ctx.empty()
    for shift in (0.0, 7.5):
        fr.fr_jv(ctx, U, Rg, z, shift, y)
        yo = fd_jv(prob, U0, R0, z0, shift)
        assert np.linalg.norm(y.cpu().numpy() - yo) / np.linalg.norm(yo) < TOL_JV32
    # a zero direction gives zero
    fr.fr_jv(ctx, U, Rg, _t(np.zeros_like(z0)), 3.0, y)
    assert np.array_equal(y.cpu().numpy(), np.zeros_like(z0))


def test_mixed_jv_run_within_tolerance(fr):
    """ROW3 steps of the 20 x 20 p = 3 vortex with the mixed A z at
    tol_lin = 1e-8 against the FP64 oracle at tol_lin = 1e-12: the stage
    solves converge to the mixed operator's solution, which differs from the
    FP64 one by the A z error (1e-7 relative) times the step, so the states
    agree to 1e-7 relative."""
    p = 3
    xe, ye = S.uniform_mesh(20)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-8, gmres_max_restarts=60, jv_precision=1))
    ref = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-8, gmres_max_restarts=60))
    U, V = _t(U0), _t(U0)
    Uo = U0.copy()
    for _ in range(3):
        st = fr.step_row(ctx, 3, 0.05, U)
        sr = fr.step_row(ref, 3, 0.05, V)
        assert st.converged and sr.converged
        assert abs(st.gmres_iters - sr.gmres_iters) <= 0.1 * sr.gmres_iters + 2
        Uo, _ = o_row(prob, ROW[3](), 0.05, Uo, SolverOpts(tol_lin=1e-12, m=30, max_restarts=60))
    assert np.linalg.norm(U.cpu().numpy() - Uo) / np.linalg.norm(Uo) < 1e-7


def test_mixed_jv_rejected_for_navier_stokes(fr):
    ch = S.Channel()
    xe = np.linspace(0.0, 2.0, 5)
    ye = S.channel_y_edges(4)
    with pytest.raises(fr.FrError):
        fr.Context(xe, ye, 2, fr.default_opts(jv_precision=1, mu=ch.mu, wall_temperature=ch.temperature),
                   wall_y=True)
