"""3D hexahedral Navier-Stokes path on the GPU against the FP64 oracle
(oracle/fr3d.py): residual (Euler and BR2, degrees 1-4, ragged element
tiles), FD operator, element-Jacobi blocks (degrees 1-3), ROW / ESDIRK /
SSPRK3 steps, the Taylor-Green dissipation rate, and properties of the
64^3 p = 3 Taylor-Green workload.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

import synthetic as S
from oracle.basis import Basis
from oracle.fr3d import Gas3D, Mesh3D, Problem3D, dissipation_rate, residual3d
from oracle.jfnk import ElementJacobi, element_blocks, fd_jv
from oracle.steppers import PtcOpts, SolverOpts
from oracle.steppers import step_esdirk as o_esdirk
from oracle.steppers import step_row as o_row
from oracle.steppers import step_ssprk3 as o_ssprk3
from oracle.tableaus import ESDIRK, ROW

pytestmark = pytest.mark.gpu

TG = S.TaylorGreen()
JV32_TOL = 1e-6   # relative error of the FP32-linear-parts A z: measured 6e-8 .. 9e-8 (p = 1-4)


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


def _opts(fr, mu, **kw):
    kw.setdefault("precond", 0)
    return fr.default_opts(mu=mu, prandtl=0.71, **kw)


def _random_case(p, dims=(5, 3, 4), seed=0):
    edges = S.stretched_mesh3d(*dims, seed=seed)
    X, Y, Z = S.point_coords3d(*edges, p)
    return edges, S.smooth_random_state3d(X, Y, Z, seed=seed + 1, amp=0.1)


def _tgv_case(n, p):
    edges = S.uniform_mesh3d(n)
    X, Y, Z = S.point_coords3d(*edges, p)
    return edges, TG.state(X, Y, Z)


@pytest.mark.parametrize("mu", [0.0, 0.05])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_residual_matches_oracle(fr, p, mu):
    """60 elements: the element tiles of every degree (16, 8, 4, 2 per CTA)
    end in a ragged tile for p = 1 and 2."""
    edges, U0 = _random_case(p, seed=p)
    ctx = fr.Context3D(*edges, p, _opts(fr, mu))
    R = ctx.empty()
    fr.fr_residual(ctx, _t(U0), R)
    Ro = residual3d(U0, Mesh3D(*edges), p, Gas3D(mu=mu, prandtl=0.71))
    assert _rel(R.cpu().numpy(), Ro) < 1e-12


def test_free_stream_and_conservation(fr):
    p = 3
    edges, U0 = _random_case(p, seed=7)
    ctx = fr.Context3D(*edges, p, _opts(fr, 0.05))
    R = ctx.empty()
    one = np.ones(U0.shape[::2])
    Uf = S.conserved3d(1.2 * one, 0.3 * one, -0.2 * one, 0.4 * one, 2.0 * one)
    fr.fr_residual(ctx, _t(Uf), R)
    assert float(R.abs().max()) < 1e-12
    fr.fr_residual(ctx, _t(U0), R)
    Rg = R.cpu().numpy()
    m = Mesh3D(*edges)
    b = Basis(p)
    w3 = np.einsum("k,j,i->kji", b.w, b.w, b.w).reshape(-1)
    vol = np.einsum("z,y,x->zyx", m.hz, m.hy, m.hx).reshape(-1) / 8.0
    tot = np.einsum("evp,p,e->v", Rg, w3, vol)
    scale = np.einsum("evp,p,e->v", np.abs(Rg), w3, vol)
    assert np.all(np.abs(tot) < 1e-13 * np.maximum(scale, 1.0))


@pytest.mark.parametrize("p", [1, 3])
def test_jv_matches_oracle(fr, p):
    edges, U0 = _random_case(p, dims=(4, 3, 3), seed=11)
    gas = Gas3D(mu=0.03, prandtl=0.71)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    R0 = prob.R(U0)
    z0 = S.random_vector(U0.shape, 5)
    ctx = fr.Context3D(*edges, p, _opts(fr, 0.03))
    y = ctx.empty()
    fr.fr_jv(ctx, _t(U0), _t(R0), _t(z0), 12.0, y)
    yo = fd_jv(prob, U0, R0, z0, 12.0)
    assert _rel(y.cpu().numpy(), yo) < 1e-6


@pytest.mark.parametrize("p,mu", [(1, 0.03), (2, 0.03), (3, 0.03), (4, 0.03), (3, 0.0)])
def test_jv_fp32_linear_parts_matches_oracle(fr, p, mu):
    """A z with FP32 linear parts (jv_precision = 1) against the oracle's FP64
    FD product: the FP32 rounding of z and of the derivatives, traces,
    liftings and divergence acts on (R(U + eps z) - R(U)) / eps, not on R,
    so it leaves a relative error of a few FP32 unit roundoffs (6e-8 to 9e-8
    measured for p = 1-4); z = 0 gives shift z = 0 exactly."""
    edges, U0 = _random_case(p, dims=(4, 3, 3), seed=11)
    gas = Gas3D(mu=mu, prandtl=0.71)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    R0 = prob.R(U0)
    z0 = S.random_vector(U0.shape, 5)
    ctx = fr.Context3D(*edges, p, _opts(fr, mu, jv_precision=1))
    y = ctx.empty()
    fr.fr_jv(ctx, _t(U0), _t(R0), _t(z0), 12.0, y)
    yo = fd_jv(prob, U0, R0, z0, 12.0)
    err = _rel(y.cpu().numpy(), yo)
    assert err < JV32_TOL, err
    fr.fr_jv(ctx, _t(U0), _t(R0), _t(np.zeros_like(z0)), 12.0, y)
    assert np.all(y.cpu().numpy() == 0.0)


def test_row3_step_with_fp32_linear_parts_matches_oracle(fr):
    """ROW3 with the FP32-linear-parts A z at tol_lin 1e-8 (the operator's
    own relative error is ~1e-6, so GMRES converges to the FP64 step to about
    that level)."""
    p = 2
    edges, U0 = _tgv_case(4, p)
    gas = Gas3D(mu=TG.mu, prandtl=TG.prandtl)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    dt = 0.1
    ctx = fr.Context3D(*edges, p, _opts(fr, TG.mu, precond=1, tol_lin=1e-8, gmres_max_restarts=100,
                                        jv_precision=1))
    U = _t(U0)
    st = fr.step_row(ctx, 3, dt, U)
    Uo, so = o_row(prob, ROW[3](), dt, U0, SolverOpts(tol_lin=1e-12, m=30, max_restarts=200, precond=True))
    assert st.converged and so.converged
    err = _rel(U.cpu().numpy(), Uo)
    assert err < 1e-7, err


@pytest.mark.parametrize("p,prec,tol", [(1, 0, 1e-6), (1, 2, 3e-2), (2, 0, 1e-6), (2, 1, 1e-4), (3, 1, 1e-4),
                                        (3, 2, 3e-2)])
def test_element_jacobi_matches_oracle(fr, p, prec, tol):
    """Blocks of 40 rows (bulk-copy apply), 135 rows (row apply) and 320
    rows (FP32 Gauss-Jordan over a two-CTA cluster, row apply)."""
    edges, U0 = _random_case(p, dims=(2, 4, 2), seed=13)
    gas = Gas3D(mu=0.03, prandtl=0.71)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    shift = 40.0
    ctx = fr.Context3D(*edges, p, _opts(fr, 0.03, precond=1, block_precision=prec))
    fr.ejacobi_factor(ctx, _t(U0), None, shift)
    r0 = S.random_vector(U0.shape, 8)
    z = ctx.empty()
    fr.ejacobi_apply(ctx, _t(r0), z)
    zo = ElementJacobi(element_blocks(prob, U0, shift))(r0)
    assert _rel(z.cpu().numpy(), zo) < tol


@pytest.mark.parametrize("p,prec,tol", [(2, 1, 2e-3), (3, 1, 2e-3), (3, 2, 3e-2)])
def test_fp32_columns_match_oracle(fr, p, prec, tol):
    """Element-Jacobi columns formed in FP32 (block_columns = 1: step
    2^-12 (1 + |q|), the element-local R(U) by the same FP32 arithmetic)
    against the oracle's FP64 blocks: the FD columns carry ~1e-3 relative
    error (truncation of the larger step plus FP32 rounding of the residual
    over the step), so the apply agrees to that level."""
    edges, U0 = _random_case(p, dims=(2, 4, 2), seed=13)
    gas = Gas3D(mu=0.03, prandtl=0.71)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    shift = 40.0
    ctx = fr.Context3D(*edges, p, _opts(fr, 0.03, precond=1, block_precision=prec, block_columns=1))
    fr.fr_set_block_chunk(ctx, 5)            # chunks of 5 elements, ragged last chunk
    fr.ejacobi_factor(ctx, _t(U0), None, shift)
    r0 = S.random_vector(U0.shape, 8)
    z = ctx.empty()
    fr.ejacobi_apply(ctx, _t(r0), z)
    zo = ElementJacobi(element_blocks(prob, U0, shift))(r0)
    err = _rel(z.cpu().numpy(), zo)
    assert err < tol, err


def test_degree3_blocks_staged_in_chunks(fr):
    """320-row blocks staged and inverted a few elements at a time (ragged
    last chunk) give the same preconditioner, bit for bit, as one chunk."""
    p = 3
    edges, U0 = _random_case(p, dims=(2, 4, 2), seed=17)
    shift = 25.0
    r0 = _t(S.random_vector(U0.shape, 9))
    zs = []
    for chunk in (None, 5, 1):
        ctx = fr.Context3D(*edges, p, _opts(fr, 0.03, precond=1, block_precision=1))
        if chunk:
            fr.fr_set_block_chunk(ctx, chunk)
        fr.ejacobi_factor(ctx, _t(U0), None, shift)
        z = ctx.empty()
        fr.ejacobi_apply(ctx, r0, z)
        zs.append(z.cpu().numpy())
        ctx.close()
    assert np.array_equal(zs[0], zs[1]) and np.array_equal(zs[0], zs[2])
    with pytest.raises(fr.FrError):
        ctx = fr.Context3D(*edges, p, _opts(fr, 0.03, precond=1, block_precision=1))
        fr.fr_set_block_chunk(ctx, 17)      # more than the 16 elements


def test_ssprk3_steps_match_oracle(fr):
    p = 2
    edges, U0 = _tgv_case(4, p)
    gas = Gas3D(mu=TG.mu, prandtl=TG.prandtl)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    ctx = fr.Context3D(*edges, p, _opts(fr, TG.mu))
    U = _t(U0)
    Uo = U0.copy()
    for _ in range(3):
        fr.step_ssprk3(ctx, 0.01, U)
        Uo = o_ssprk3(prob, 0.01, Uo)
    assert _rel(U.cpu().numpy(), Uo) < 1e-12


@pytest.mark.parametrize("p,precond,cols", [(1, 1, 0), (2, 1, 0), (3, 0, 0), (3, 1, 0), (3, 1, 1)])
def test_row3_step_matches_oracle(fr, p, precond, cols):
    """cols = 1: FP32 block columns; the preconditioner changes, the
    converged step does not."""
    n = 4 if p < 3 else (2 if precond else 3)   # the oracle's blocks need even nx, ny, nz
    edges, U0 = _tgv_case(n, p)
    gas = Gas3D(mu=TG.mu, prandtl=TG.prandtl)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    dt = 0.1
    prec = 1 if p == 3 and precond else 0       # 320-row blocks are stored in FP32
    ctx = fr.Context3D(*edges, p, _opts(fr, TG.mu, precond=precond, block_precision=prec, tol_lin=1e-12,
                                        gmres_max_restarts=200, block_columns=cols))
    U = _t(U0)
    st = fr.step_row(ctx, 3, dt, U)
    Uo, so = o_row(prob, ROW[3](), dt, U0, SolverOpts(tol_lin=1e-12, m=30, max_restarts=200,
                                                       precond=bool(precond)))
    assert st.converged and so.converged
    assert _rel(U.cpu().numpy(), Uo) < 1e-9


def test_esdirk3_step_matches_oracle(fr):
    p = 2
    edges, U0 = _tgv_case(4, p)
    gas = Gas3D(mu=TG.mu, prandtl=TG.prandtl)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    dt = 0.1
    ctx = fr.Context3D(*edges, p, _opts(fr, TG.mu, precond=1, gmres_max_restarts=60))
    po = fr.default_ptc_opts(tol_nl=1e-12, tol_lin=1e-3)
    U = _t(U0)
    st = fr.step_esdirk(ctx, 3, dt, U, po)
    Uo, so = o_esdirk(prob, ESDIRK[3](), dt, U0, PtcOpts(tol_nl=1e-12, tol_lin=1e-3),
                      SolverOpts(m=30, max_restarts=60))
    assert st.converged and so.converged
    assert _rel(U.cpu().numpy(), Uo) < 1e-9


def test_esdirk3_degree3_step_with_chunked_blocks_matches_oracle(fr):
    """ESDIRK3 with 320-row FP32 blocks staged three elements at a time: a
    new pseudo-time shift forms the blocks again at the current iterate
    (the oracle re-inverts the stage's first blocks); both converge to the
    same stage solutions."""
    p = 3
    edges, U0 = _tgv_case(2, p)
    gas = Gas3D(mu=TG.mu, prandtl=TG.prandtl)
    prob = Problem3D(Mesh3D(*edges), p, gas)
    dt = 0.1
    ctx = fr.Context3D(*edges, p, _opts(fr, TG.mu, precond=1, block_precision=1, gmres_max_restarts=60))
    fr.fr_set_block_chunk(ctx, 3)
    po = fr.default_ptc_opts(tol_nl=1e-12, tol_lin=1e-3)
    U = _t(U0)
    st = fr.step_esdirk(ctx, 3, dt, U, po)
    Uo, so = o_esdirk(prob, ESDIRK[3](), dt, U0, PtcOpts(tol_nl=1e-12, tol_lin=1e-3),
                      SolverOpts(m=30, max_restarts=60))
    assert st.converged and so.converged
    assert _rel(U.cpu().numpy(), Uo) < 1e-9


@pytest.mark.parametrize("p", [2, 3])
def test_dissipation_rate_matches_oracle(fr, p):
    edges, U0 = _tgv_case(5, p)
    gas = Gas3D(mu=TG.mu, prandtl=TG.prandtl)
    ctx = fr.Context3D(*edges, p, _opts(fr, TG.mu))
    U = _t(U0)
    Ue = U0.copy()
    # a state with div v != 0 and a non-constant pressure, so eps3 is exercised too
    edges2, Ur = _random_case(p, dims=(3, 4, 5), seed=21)
    ctx2 = fr.Context3D(*edges2, p, _opts(fr, TG.mu))
    for c, V, E, m in ((ctx, U, Ue, Mesh3D(*edges)), (ctx2, _t(Ur), Ur, Mesh3D(*edges2))):
        got = fr.fr_dissipation_rate(c, V, TG.rho0)
        want = dissipation_rate(E, m, p, gas, TG.rho0)
        for g, w in zip(got, want):
            assert abs(g - w) <= 1e-12 * max(abs(w), 1e-30) + 1e-15


def test_unsupported_3d_options_rejected(fr):
    edges = S.uniform_mesh3d(2)
    for kw in (dict(precond=1), dict(riemann=1), dict(jv_precision=2)):
        with pytest.raises(fr.FrError):
            fr.Context3D(*edges, 3, _opts(fr, 0.01, **kw))
    with pytest.raises(fr.FrError):
        fr.Context3D(*edges, 5, _opts(fr, 0.01))
    with pytest.raises(fr.FrError):
        fr.Context3D(*edges, 4, _opts(fr, 0.01, precond=1, block_precision=1))
    ctx2 = fr.Context(*S.uniform_mesh(4), 2)
    with pytest.raises(fr.FrError):
        fr.fr_dissipation_rate(ctx2, ctx2.empty())


def test_taylor_green_64_cubed_p3_properties(fr):
    """The Taylor-Green workload at its full size (64^3 elements, p = 3,
    83.9 M DOFs) in the benchmark's configuration: the dissipation rate and
    kinetic energy of the initial field against their closed forms
    (<S:S> = 3/8, <rho |v|^2/2> = 1/8, eps3 = 0 by symmetry), discrete
    conservation of R, and a free stream kept to round-off."""
    import torch
    p, n = 3, 64
    edges = S.uniform_mesh3d(n)
    X, Y, Z = S.point_coords3d(*edges, p)
    U0 = TG.state(X, Y, Z)
    del X, Y, Z
    ctx = fr.Context3D(*edges, p, _opts(fr, TG.mu, m_max=4, gmres_m=4))
    U = _t(U0)
    del U0
    e1, e3, k = fr.fr_dissipation_rate(ctx, U, TG.rho0)
    # eps1 at 64^3 p = 3: the interpolation error of the velocity derivative
    # falls as h^4 (3.6e-4 at 8^3, so about 1e-7 here)
    assert abs(e1 / (2 * TG.mu * 0.375) - 1) < 1e-6
    assert abs(e3) < 1e-9 * 2 * TG.mu * 0.375
    assert abs(k / 0.125 - 1) < 1e-12
    R = ctx.empty()
    fr.fr_residual(ctx, U, R)
    b = Basis(p)
    w3 = torch.from_numpy(np.einsum("k,j,i->kji", b.w, b.w, b.w).reshape(-1)).cuda()
    h = 2 * np.pi / n
    tot = (R * w3).sum(dim=(0, 2)) * (h ** 3 / 8)
    scale = (R.abs() * w3).sum(dim=(0, 2)) * (h ** 3 / 8)
    assert bool((tot.abs() < 1e-11 * scale.clamp(min=1.0)).all())
    U.zero_()
    U[:, 0] = 1.0
    U[:, 1] = 0.5
    U[:, 4] = 80.0
    fr.fr_residual(ctx, U, R)
    assert float(R.abs().max()) < 1e-9     # flux terms ~ p 2/h = 32 x 20
