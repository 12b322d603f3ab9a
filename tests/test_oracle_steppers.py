"""Pins of the oracle time integrators (oracle/steppers.py) on the FR vortex."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import Problem
from oracle.steppers import PtcOpts, SolverOpts, step_bdf2, step_esdirk, step_row, step_ssprk3
from oracle.tableaus import ESDIRK, ROW


@pytest.fixture(scope="module")
def vortex():
    p = 2
    xe, ye = S.uniform_mesh(4)
    prob = Problem(Mesh(xe, ye), p)
    X, Y = S.point_coords(xe, ye, p)
    return prob, S.Vortex().state(X, Y)


TIGHT = SolverOpts(tol_lin=1e-12, m=30, max_restarts=40)
TIGHT_PTC = PtcOpts(tol_nl=1e-12, tol_lin=1e-3)


def _run(step, U0, T, n):
    U = U0.copy()
    Up = None
    for k in range(n):
        U, Up = step(U, Up, T / n, k)
    return U


def _rate(step, U0, T, ns, nref):
    ref = _run(step, U0, T, nref)
    errs = [np.linalg.norm(_run(step, U0, T, n) - ref) for n in ns]
    return errs, [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("order", [2, 3, 4])
def test_row_temporal_order(vortex, order):
    prob, U0 = vortex
    tab = ROW[order]()
    step = lambda U, Up, dt, k: (step_row(prob, tab, dt, U, TIGHT)[0], None)
    errs, rates = _rate(step, U0, 0.4, (2, 4, 8), 32)
    # at least the nominal order (ROW2's linear error is third order, so its
    # pre-asymptotic rate may exceed 2)
    assert rates[-1] > order - 0.35, (errs, rates)
    assert rates[-1] < order + 0.95, (errs, rates)


@pytest.mark.slow
@pytest.mark.parametrize("order", [2, 3, 4])
def test_esdirk_temporal_order(vortex, order):
    prob, U0 = vortex
    tab = ESDIRK[order]()
    step = lambda U, Up, dt, k: (step_esdirk(prob, tab, dt, U, TIGHT_PTC, TIGHT)[0], None)
    errs, rates = _rate(step, U0, 0.4, (2, 4, 8), 32)
    assert rates[-1] > order - 0.35, (errs, rates)
    assert rates[-1] < order + 0.95, (errs, rates)


def test_bdf2_temporal_order(vortex):
    prob, U0 = vortex

    def step(U, Up, dt, k):
        Un, Uo, _ = step_bdf2(prob, dt, U, Up, first_step=(k == 0), popts=TIGHT_PTC, sopts=TIGHT)
        return Un, Uo
    errs, rates = _rate(step, U0, 0.4, (4, 8, 16), 64)
    assert abs(rates[-1] - 2.0) < 0.3, (errs, rates)


def test_row_and_esdirk_agree_to_their_error(vortex):
    prob, U0 = vortex
    dt = 0.05
    Ur, sr = step_row(prob, ROW[4](), dt, U0, TIGHT)
    Ue, se = step_esdirk(prob, ESDIRK[4](), dt, U0, TIGHT_PTC, TIGHT)
    assert np.linalg.norm(Ur - Ue) / np.linalg.norm(U0) < 1e-6
    assert sr.converged and se.converged
    assert sr.gmres_iters > 0 and se.ptc_iters > 0


def test_ptc_rejection_halves_dtau_max(vortex):
    """A GMRES that cannot cut its residual by one decade (a single Krylov
    iteration, no preconditioner) rejects pseudo steps (Sec. 4.4)."""
    prob, U0 = vortex
    weak = SolverOpts(m=1, max_restarts=0, precond=False)
    popts = PtcOpts(tol_nl=1e-8, tol_lin=1e-1, max_rejections=3, max_iters=5)
    _, st = step_esdirk(prob, ESDIRK[2](), 0.5, U0, popts, weak)
    assert st.rejections > 0
    assert not st.converged


def test_ptc_converges_loose_tolerances(vortex):
    prob, U0 = vortex
    popts = PtcOpts(tol_nl=1e-6, tol_lin=1e-1)
    U1, st = step_esdirk(prob, ESDIRK[3](), 0.1, U0, popts, SolverOpts())
    assert st.converged and st.rejections == 0
    assert np.all(np.isfinite(U1))


class _Linear:
    """R(u) = A u (a fixed non-normal matrix)."""

    def __init__(self, A):
        self.A = A

    def R(self, U):
        return self.A @ U


def test_ssprk3_is_the_third_order_taylor_polynomial_on_linear_problems():
    """Any three-stage third-order Runge-Kutta scheme advances u' = A u by
    exactly (I + hA + (hA)^2/2 + (hA)^3/6) u."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((6, 6)) + np.triu(rng.standard_normal((6, 6)), 1) * 3.0
    u = rng.standard_normal(6)
    h = 0.07
    hA = h * A
    want = u + hA @ u + hA @ (hA @ u) / 2.0 + hA @ (hA @ (hA @ u)) / 6.0
    got = step_ssprk3(_Linear(A), h, u)
    assert np.allclose(got, want, rtol=1e-14, atol=1e-14)


def test_ssprk3_temporal_order(vortex):
    prob, U0 = vortex
    step = lambda U, Up, dt, k: (step_ssprk3(prob, dt, U), None)
    errs, rates = _rate(step, U0, 0.4, (16, 32, 64), 512)
    assert 2.7 < rates[-1] < 3.4, (errs, rates)


def test_frozen_stage_preconditioner_reaches_the_same_stage_solution(vortex):
    """refresh = "frozen" keeps each stage's first element-Jacobi blocks (and
    their shift) for all its pseudo steps: a different right preconditioner,
    so a different Krylov path, but PTC converges to the same stage values."""
    prob, U0 = vortex
    tab = ESDIRK[3]()
    base = step_esdirk(prob, tab, 0.2, U0, PtcOpts(tol_nl=1e-11, tol_lin=1e-3), TIGHT)[0]
    frz = step_esdirk(prob, tab, 0.2, U0, PtcOpts(tol_nl=1e-11, tol_lin=1e-3, refresh="frozen"), TIGHT)[0]
    assert np.linalg.norm(frz - base) / np.linalg.norm(base) < 1e-9
