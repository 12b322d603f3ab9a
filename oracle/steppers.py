"""Time integrators of Sec. 4 on top of the JFNK pieces.

* ``step_row``: Eq. Rosenbrock_General.  The operator (I/(omega dt) - dR/dq)
  is frozen at q^n for all stages (the Jacobian is evaluated once per step,
  Sec. 4.3), applied Jacobian-free with base point (q^n, R(q^n)); each stage
  solves it with GMRES from a zero guess to ``tol_lin``.  The element-Jacobi
  blocks are formed once per step at q^n with shift 1/(omega dt).
* ``step_esdirk``: Eq. ESDIRK2 with the stage equations of Eq. SDIRK_newton
  solved by pseudo-transient continuation (Eq. linearized_pseudo_transient_final):
  (I/dtau + I/(omega dt) - dR/dq)^k dq = -F(q^k).  Each pseudo step forms
  the element-Jacobi blocks at q^k and solves with GMRES to ``tol_lin``.
  SER update dtau <- min(dtau ||F^{k}|| / ||F^{k+1}||, dtau_max) after every
  accepted step, dtau_init = dt and dtau_max = 1e20 unless given (Sec. 4.4).
  When GMRES fails to cut its residual by one decade the pseudo step is
  rejected, dtau_max is halved and dtau = min(dtau, dtau_max).  The stage
  iterate starts from the previous stage value; convergence is
  ||F^k|| / ||F^0|| < tol_nl (relative to the first pseudo step, Sec. 5.1).
* ``step_bdf2``: Eq. BDF with omega = 2/3, a = (4/3, -1/3), Eq. BDF_newton
  solved by the same continuation.  The paper does not say how the first step
  is started; ``first_step=True`` takes one backward-Euler step
  (omega = 1, a = (1, 0)).

* ``step_ssprk3``: the explicit three-stage, third-order strong-stability-
  preserving Runge-Kutta scheme the paper's introduction contrasts the
  implicit schemes with (Shu-Osher form: u1 = u + dt R(u),
  u2 = 3/4 u + 1/4 (u1 + dt R(u1)), u_new = 1/3 u + 2/3 (u2 + dt R(u2))).

Pins (tests/test_oracle_steppers.py): observed temporal order of every
scheme on a smooth vortex problem at tight tolerances, BDF2 coefficients,
rejection / halving path, agreement of ROW at tight tolerance with ESDIRK
of the same order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .jfnk import ElementJacobi, Problem, diagonal_blocks, element_blocks, fd_jv, gmres
from .tableaus import BDF2_A, BDF2_OMEGA, EsdirkTableau, RowTableau


@dataclass
class SolverOpts:
    m: int = 30
    max_restarts: int = 20
    tol_lin: float = 1e-8
    precond: bool = True
    eps_rel: float = 1e-7
    eps_fixed: float | None = None


@dataclass
class PtcOpts:
    tol_nl: float = 1e-6
    tol_lin: float = 1e-1
    dtau_init: float | None = None   # None -> dt
    dtau_max: float = 1e20
    max_iters: int = 200
    max_rejections: int = 30
    reject_above: float = 0.1        # GMRES relres above this -> reject
    refresh: str = "stage"           # "stage", "iterate" or "frozen" (element-Jacobi blocks)


@dataclass
class StepStats:
    gmres_iters: int = 0
    gmres_calls: int = 0
    ptc_iters: int = 0
    rejections: int = 0
    residual_evals: int = 0
    converged: bool = True
    per_stage_iters: list = field(default_factory=list)


def _linear_solve(prob, U, R0, shift, b, opts: SolverOpts, tol, stats: StepStats, blocks=None):
    Minv = ElementJacobi(blocks) if (opts.precond and blocks is not None) else None
    A = lambda z: fd_jv(prob, U, R0, z, shift, opts.eps_rel, opts.eps_fixed)
    x, info = gmres(A, b, None, opts.m, tol, opts.max_restarts, Minv)
    stats.gmres_iters += info.iters
    stats.gmres_calls += 1
    stats.per_stage_iters.append(info.iters)
    return x, info


def step_row(prob: Problem, tab: RowTableau, dt, U, opts: SolverOpts = SolverOpts()):
    """One ROW step q^n -> q^{n+1} (Eq. Rosenbrock_General)."""
    stats = StepStats()
    n0 = prob.n_residuals
    shift = 1.0 / (tab.gamma * dt)
    R0 = prob.R(U)
    blocks = element_blocks(prob, U, shift, eps_rel=opts.eps_rel) if opts.precond else None
    Y = []
    for i in range(tab.stages):
        if i == 0 or not np.any(tab.a[i, :i]):
            Ri = R0
        else:
            Ui = U + sum(tab.a[i, j] * Y[j] for j in range(i))
            Ri = prob.R(Ui)
        b = Ri + sum(tab.c[i, j] * Y[j] for j in range(i)) / dt if i > 0 else Ri
        Yi, info = _linear_solve(prob, U, R0, shift, b, opts, opts.tol_lin, stats, blocks)
        stats.converged &= info.converged
        Y.append(Yi)
    Unew = U + sum(tab.m[j] * Y[j] for j in range(tab.stages))
    stats.residual_evals = prob.n_residuals - n0
    return Unew, stats


def ptc_solve(prob: Problem, rhs_const, omega_dt, q0, dt, popts: PtcOpts, sopts: SolverOpts,
              stats: StepStats):
    """Solve F(q) = q/(omega dt) - R(q) - rhs_const/(omega dt) = 0 by
    pseudo-transient continuation with SER (Sec. 4.4).  Returns (q, R(q))."""
    def F_of(q):
        Rq = prob.R(q)
        return (q - rhs_const) / omega_dt - Rq, Rq

    q = q0.copy()
    F, Rq = F_of(q)
    F0 = np.linalg.norm(F)
    Fn = F0
    dtau = dt if popts.dtau_init is None else popts.dtau_init
    dtau_max = popts.dtau_max
    k = 0
    rejections = 0
    J = None
    J_k = -1
    while F0 > 0.0 and Fn / F0 >= popts.tol_nl:
        if k >= popts.max_iters:
            stats.converged = False
            break
        shift = 1.0 / dtau + 1.0 / omega_dt
        blocks = None
        if sopts.precond:
            if J is None or (popts.refresh == "iterate" and J_k != k):
                J = diagonal_blocks(prob, q, eps_rel=sopts.eps_rel)
                J_k = k
                shift0 = shift
            # "frozen": the blocks keep the stage's first shift (any fixed
            # right preconditioner leaves the converged answer unchanged)
            blocks = (shift0 if popts.refresh == "frozen" else shift) * np.eye(J.shape[1])[None] - J
        dq, info = _linear_solve(prob, q, Rq, shift, -F, sopts, popts.tol_lin, stats, blocks)
        if info.relres > popts.reject_above:
            rejections += 1
            stats.rejections += 1
            if rejections > popts.max_rejections:
                stats.converged = False
                break
            dtau_max *= 0.5
            dtau = min(dtau, dtau_max)
            continue
        q = q + dq
        Fnew, Rq = F_of(q)
        Fnew_n = np.linalg.norm(Fnew)
        dtau = min(dtau * Fn / Fnew_n, dtau_max) if Fnew_n > 0 else dtau_max
        F, Fn = Fnew, Fnew_n
        k += 1
        stats.ptc_iters += 1
    return q, Rq


def step_esdirk(prob: Problem, tab: EsdirkTableau, dt, U, popts: PtcOpts = PtcOpts(),
                sopts: SolverOpts = SolverOpts()):
    """One ESDIRK step (Eq. ESDIRK2 with Eq. SDIRK_newton)."""
    stats = StepStats()
    n0 = prob.n_residuals
    omega_dt = tab.omega * dt
    Rs = [prob.R(U)]
    q = U
    for i in range(1, tab.stages):
        rhs = U + dt * sum(tab.A[i, j] * Rs[j] for j in range(i))
        q, Rq = ptc_solve(prob, rhs, omega_dt, q, dt, popts, sopts, stats)
        Rs.append(Rq)
    Unew = U + dt * sum(tab.b[i] * Rs[i] for i in range(tab.stages))
    stats.residual_evals = prob.n_residuals - n0
    return Unew, stats


def step_bdf2(prob: Problem, dt, U, U_prev, first_step=False, popts: PtcOpts = PtcOpts(),
              sopts: SolverOpts = SolverOpts()):
    """One BDF2 step (Eq. BDF / BDF_newton); returns (q^{n+1}, q^n, stats)."""
    stats = StepStats()
    n0 = prob.n_residuals
    if first_step:
        omega, a1, a2 = 1.0, 1.0, 0.0
    else:
        omega, (a1, a2) = BDF2_OMEGA, BDF2_A
    rhs = a1 * U + (a2 * U_prev if a2 != 0.0 else 0.0)
    q, _ = ptc_solve(prob, rhs, omega * dt, U, dt, popts, sopts, stats)
    stats.residual_evals = prob.n_residuals - n0
    return q, U.copy(), stats


def step_ssprk3(prob, dt, U):
    """One explicit SSPRK3 step (Shu-Osher form); ``prob`` needs only ``R``."""
    u1 = U + dt * prob.R(U)
    u2 = 0.75 * U + 0.25 * (u1 + dt * prob.R(u1))
    return U / 3.0 + (2.0 / 3.0) * (u2 + dt * prob.R(u2))
