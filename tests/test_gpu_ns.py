"""Viscous BR2 residual, FD operator, element blocks and steps on the GPU
against the FP64 oracle (oracle/ns2d.py) and the Poiseuille closed form.
Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

import synthetic as S
from oracle.basis import Basis
from oracle.fr2d import Mesh
from oracle.jfnk import ElementJacobi, Problem, element_blocks, fd_jv
from oracle.ns2d import Viscous, ns_residual
from oracle.steppers import PtcOpts, SolverOpts
from oracle.steppers import step_esdirk as o_esdirk
from oracle.steppers import step_row as o_row
from oracle.tableaus import ESDIRK, ROW

pytestmark = pytest.mark.gpu


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


def _channel(nx, ny, p, seed=0):
    xe = np.linspace(0.0, 2.0, nx + 1)
    ye = S.channel_y_edges(ny, first=0.02, ratio=1.3)
    X, Y = S.point_coords(xe, ye, p)
    rho = 1.0
    T = 1.0 / (1.4 * 0.2 ** 2)          # M = 0.2 on the centreline speed 1 (R = 1)
    u = 4 * Y * (1 - Y)
    U = S.conserved(rho * np.ones_like(X), u, np.zeros_like(X), rho * T * np.ones_like(X))
    pert = S.smooth_random_state(X, Y, seed=seed, amp=0.01, box=(0, 2, 0, 1), base=(0.0, 0.0, 0.0, 0.0))
    U = U + pert * (Y * (1 - Y))[:, None, :] * 4
    return xe, ye, U, T


def _opts(fr, mu, gx=0.0, tw=1.0, **kw):
    return fr.default_opts(mu=mu, prandtl=0.72, body_force_x=gx, wall_temperature=tw, **kw)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_ns_residual_periodic_matches_oracle(fr, p):
    xe, ye = S.stretched_mesh(7, 5, seed=p)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.smooth_random_state(X, Y, seed=30 + p, amp=0.1)
    mu = 0.05
    ctx = fr.Context(xe, ye, p, _opts(fr, mu))
    R = ctx.empty()
    fr.fr_residual(ctx, _t(U0), R)
    Ro = ns_residual(U0, Mesh(xe, ye), p, Viscous(mu=mu))
    assert _rel(R.cpu().numpy(), Ro) < 1e-12


@pytest.mark.parametrize("p", [3, 4])
def test_ns_residual_channel_walls_matches_oracle(fr, p):
    xe, ye, U0, T = _channel(6, 8, p, seed=p)
    mu, gx = 0.002, 8 * 0.002
    ctx = fr.Context(xe, ye, p, _opts(fr, mu, gx, T), wall_y=True)
    R = ctx.empty()
    fr.fr_residual(ctx, _t(U0), R)
    Ro = ns_residual(U0, Mesh(xe, ye, wall_y=True), p, Viscous(mu=mu, gx=gx, t_wall=T))
    # the residual is a small difference of O(1/h) terms near the walls
    assert np.max(np.abs(R.cpu().numpy() - Ro)) < 1e-11 * max(1.0, np.max(np.abs(Ro)))


def test_ns_poiseuille_closed_form_on_gpu(fr):
    p = 4
    xe = np.linspace(0.0, 2.0, 4)
    ye = S.channel_y_edges(6, first=0.05, ratio=1.3)
    X, Y = S.point_coords(xe, ye, p)
    mu, T = 0.002, 17.857
    u = 4 * Y * (1 - Y)
    U0 = S.conserved(np.ones_like(X), u, np.zeros_like(X), T * np.ones_like(X))
    ctx = fr.Context(xe, ye, p, _opts(fr, mu, 8 * mu, T), wall_y=True)
    R = ctx.empty()
    fr.fr_residual(ctx, _t(U0), R)
    Rg = R.cpu().numpy()
    heat = mu * (4 * (1 - 2 * Y)) ** 2
    assert np.max(np.abs(Rg[:, :3])) < 1e-10
    assert np.max(np.abs(Rg[:, 3] - heat)) < 1e-9


def test_ns_conservation_periodic(fr):
    p = 3
    xe, ye = S.stretched_mesh(6, 5, seed=9)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.smooth_random_state(X, Y, seed=2, amp=0.1)
    ctx = fr.Context(xe, ye, p, _opts(fr, 0.05))
    R = ctx.empty()
    fr.fr_residual(ctx, _t(U0), R)
    Rg = R.cpu().numpy()
    m = Mesh(xe, ye)
    b = Basis(p)
    w2 = np.outer(b.w, b.w).reshape(-1)
    detJ = (0.25 * m.hx * m.hy).reshape(-1)
    tot = np.einsum("evp,p,e->v", Rg, w2, detJ)
    scale = np.einsum("evp,p,e->v", np.abs(Rg), w2, detJ)
    assert np.all(np.abs(tot) < 1e-13 * np.maximum(scale, 1.0))


@pytest.mark.parametrize("p", [2, 3])
def test_ns_jv_matches_oracle(fr, p):
    xe, ye, U0, T = _channel(4, 6, p, seed=1)
    mu, gx = 0.002, 0.016
    ph = Viscous(mu=mu, gx=gx, t_wall=T)
    prob = Problem(Mesh(xe, ye, wall_y=True), p, viscous=ph)
    R0 = prob.R(U0)
    z0 = S.random_vector(U0.shape, 5)
    ctx = fr.Context(xe, ye, p, _opts(fr, mu, gx, T), wall_y=True)
    y = ctx.empty()
    fr.fr_jv(ctx, _t(U0), _t(R0), _t(z0), 12.0, y)
    yo = fd_jv(prob, U0, R0, z0, 12.0)
    assert _rel(y.cpu().numpy(), yo) < 1e-6


# FP32 blocks: tensor-core inversion with TF32-split operands (effective unit
# roundoff 2^-23), bound 2e-4; the wall-clustered blocks here have condition
# numbers up to 4e5 (see tests/test_gpu_mixed_precision.py)
@pytest.mark.parametrize("prec,tol", [(0, 1e-6), (1, 2e-4), (2, 3e-2)])
def test_ns_element_jacobi_matches_oracle(fr, prec, tol):
    p = 2
    xe, ye, U0, T = _channel(4, 4, p, seed=2)
    mu, gx = 0.002, 0.016
    ph = Viscous(mu=mu, gx=gx, t_wall=T)
    prob = Problem(Mesh(xe, ye, wall_y=True), p, viscous=ph)
    shift = 50.0
    ctx = fr.Context(xe, ye, p, _opts(fr, mu, gx, T, block_precision=prec), wall_y=True)
    fr.ejacobi_factor(ctx, _t(U0), None, shift)
    r0 = S.random_vector(U0.shape, 8)
    z = ctx.empty()
    fr.ejacobi_apply(ctx, _t(r0), z)
    zo = ElementJacobi(element_blocks(prob, U0, shift))(r0)
    assert _rel(z.cpu().numpy(), zo) < tol


@pytest.mark.parametrize("prec", [0, 2])
def test_ns_row3_step_matches_oracle(fr, prec):
    p = 2
    xe, ye, U0, T = _channel(4, 4, p, seed=3)
    mu, gx = 0.002, 0.016
    ph = Viscous(mu=mu, gx=gx, t_wall=T)
    prob = Problem(Mesh(xe, ye, wall_y=True), p, viscous=ph)
    ctx = fr.Context(xe, ye, p, _opts(fr, mu, gx, T, tol_lin=1e-12, gmres_max_restarts=60,
                                      block_precision=prec), wall_y=True)
    U = _t(U0)
    st = fr.step_row(ctx, 3, 0.02, U)
    Uo, so = o_row(prob, ROW[3](), 0.02, U0, SolverOpts(tol_lin=1e-12, m=30, max_restarts=60))
    assert st.converged and so.converged
    assert _rel(U.cpu().numpy(), Uo) < 1e-9


def test_ns_esdirk3_step_matches_oracle(fr):
    p = 2
    xe, ye, U0, T = _channel(4, 4, p, seed=4)
    mu, gx = 0.002, 0.016
    ph = Viscous(mu=mu, gx=gx, t_wall=T)
    prob = Problem(Mesh(xe, ye, wall_y=True), p, viscous=ph)
    ctx = fr.Context(xe, ye, p, _opts(fr, mu, gx, T, gmres_max_restarts=60), wall_y=True)
    po = fr.default_ptc_opts(tol_nl=1e-12, tol_lin=1e-3)
    U = _t(U0)
    st = fr.step_esdirk(ctx, 3, 0.02, U, po)
    Uo, so = o_esdirk(prob, ESDIRK[3](), 0.02, U0, PtcOpts(tol_nl=1e-12, tol_lin=1e-3),
                      SolverOpts(m=30, max_restarts=60))
    assert st.converged and so.converged
    assert _rel(U.cpu().numpy(), Uo) < 1e-9


def test_ns_residual_channel_full_size(fr):
    """The channel workload at its full size (256 x 128, p = 3, 2.1 M DOFs,
    first cell 1e-3, ratio 1.15) in the bench's launch configuration: every
    output against the oracle.  R is a small difference (|R| <= 0.05) of
    flux-derivative terms that reach 1e5-1e6 next to the walls (2/h = 2000,
    pressure ~18), so, as for the Euler residual at full size, 1e-12 is
    measured against the magnitude of those terms."""
    ch = S.Channel()
    p = 3
    xe = np.linspace(0.0, ch.lx, 257)
    ye = S.channel_y_edges(128, first=1e-3, ratio=1.15)
    X, Y = S.point_coords(xe, ye, p)
    U0 = ch.state(X, Y, seed=0)
    ctx = fr.Context(xe, ye, p, _opts(fr, ch.mu, ch.body_force, ch.temperature), wall_y=True)
    R = ctx.empty()
    fr.fr_residual(ctx, _t(U0), R)
    Ro = ns_residual(U0, Mesh(xe, ye, wall_y=True), p,
                     Viscous(mu=ch.mu, prandtl=ch.prandtl, gx=ch.body_force, t_wall=ch.temperature))
    d = R.cpu().numpy() - Ro
    scale = _term_scale(U0, xe, ye, p)
    assert np.linalg.norm(d) < 1e-12 * np.linalg.norm(scale)
    assert np.max(np.abs(d)) < 1e-12 * np.max(scale)


def _term_scale(U0, xe, ye, p):
    """sJ (|D| |F| + |D| |G|) per point with the inviscid fluxes: the size of
    the terms whose difference is R (oracle-side fluxes, test only)."""
    from oracle.fr2d import as_grid, flux_x, flux_y, from_grid
    m = Mesh(xe, ye)
    b = Basis(p)
    Q = as_grid(U0, m, p)
    hx = m.hx[None, :, :, None, None]
    hy = m.hy[None, :, :, None, None]
    F = np.abs(0.5 * hy * flux_x(Q))
    G = np.abs(0.5 * hx * flux_y(Q))
    aD = np.abs(b.D)
    Sg = np.einsum("ik,...jk->...ji", aD, F) + np.einsum("jk,...ki->...ji", aD, G)
    return from_grid(Sg * 4.0 / (hx * hy), m, p)
