"""GPU path (C ABI through the binding) against the FP64 oracle on the same
seeded inputs.

Tolerances:
* R(U): 1e-12 relative L2 (two FP64 evaluations of the same formulas differ
  only by rounding order); free stream 1e-13 absolute.  On fine meshes the
  residual is a small difference of large flux-derivative terms (at 160^2 the
  vortex residual is ~1e-4 of its terms), so there the 1e-12 is measured
  against the magnitude of those terms, sJ (|D| |F| + |D| |G|), which is the
  scale the rounding error of any FP64 evaluation is proportional to.
* FD products: the difference quotient (R(U+eps z) - R0)/eps multiplies the
  O(u |R terms|) rounding difference between two correct evaluations of R by
  1/eps, with eps |z_i| ~ 1e-7 (1+||U||)/sqrt(N): about u * 1e4 / 1e-6
  ~ 1e-8 relative on these meshes.  TOL_FD = 1e-6 relative L2 sits above
  that and well below the O(eps) truncation error of the FD product itself
  (~1e-6 to 1e-4 relative), so a wrong eps, sign or shift still fails.
* Element blocks: forward differences with step 1e-7 (1+|q_j|), compared
  through their action z = M^-1 r, relative L2 1e-6 (same reasoning).
* End-of-run states with tol_lin = 1e-12: 1e-9 relative L2.
"""
import math

import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import ElementJacobi, Problem, element_blocks, fd_jv, gmres
from oracle.steppers import PtcOpts, SolverOpts
from oracle.steppers import step_bdf2 as o_bdf2
from oracle.steppers import step_esdirk as o_esdirk
from oracle.steppers import step_row as o_row
from oracle.tableaus import ESDIRK, ROW

pytestmark = pytest.mark.gpu

TOL_R = 1e-12
TOL_FD = 1e-6
TOL_RUN = 1e-9


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1904_04825_gb300 as mod
    return mod


def _case(kind, nx, ny, p, seed):
    if kind == "uniform":
        xe, ye = S.uniform_mesh(nx, ny=ny)
    else:
        xe, ye = S.stretched_mesh(nx, ny, seed=seed)
    X, Y = S.point_coords(xe, ye, p)
    return xe, ye, X, Y


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ R(U) --
@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("kind,nx,ny", [("uniform", 4, 4), ("stretched", 7, 5), ("stretched", 13, 11)])
def test_residual_matches_oracle(fr, p, kind, nx, ny):
    xe, ye, X, Y = _case(kind, nx, ny, p, seed=nx + p)
    U0 = S.smooth_random_state(X, Y, seed=100 + p, amp=0.1)
    ctx = fr.Context(xe, ye, p)
    U = _t(U0)
    R = ctx.empty()
    fr.fr_residual(ctx, U, R)
    Ro = Problem(Mesh(xe, ye), p).R(U0)
    Rg = R.cpu().numpy()
    assert _rel(Rg, Ro) < TOL_R
    assert np.max(np.abs(Rg - Ro)) < 1e-11 * np.max(np.abs(Ro))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_residual_free_stream_and_conservation(fr, p):
    xe, ye, X, Y = _case("stretched", 9, 6, p, seed=3)
    one = np.ones_like(X)
    ctx = fr.Context(xe, ye, p)
    R = ctx.empty()
    fr.fr_residual(ctx, _t(S.conserved(1.3 * one, 0.4 * one, -0.9 * one, 2.2 * one)), R)
    assert float(R.abs().max()) < 1e-13 * 10
    U0 = S.smooth_random_state(X, Y, seed=5, amp=0.1)
    fr.fr_residual(ctx, _t(U0), R)
    Rg = R.cpu().numpy()
    m = Mesh(xe, ye)
    from oracle.basis import Basis
    b = Basis(p)
    w2 = np.outer(b.w, b.w).reshape(-1)
    detJ = (0.25 * m.hx * m.hy).reshape(-1)
    tot = np.einsum("evp,p,e->v", Rg, w2, detJ)
    scale = np.einsum("evp,p,e->v", np.abs(Rg), w2, detJ)
    assert np.all(np.abs(tot) < 1e-13 * np.maximum(scale, 1.0))


def test_residual_vortex_full_size_c2(fr):
    """160 x 160, p = 3 (1.6 M DOFs) in the launch configuration the bench uses."""
    p = 3
    xe, ye = S.uniform_mesh(160)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.Vortex().state(X, Y)
    ctx = fr.Context(xe, ye, p)
    R = ctx.empty()
    fr.fr_residual(ctx, _t(U0), R)
    Ro = Problem(Mesh(xe, ye), p).R(U0)
    scale = _term_scale(U0, xe, ye, p)
    d = R.cpu().numpy() - Ro
    assert np.linalg.norm(d) < TOL_R * np.linalg.norm(scale)
    assert np.max(np.abs(d)) < TOL_R * np.max(scale)


def test_jv_vortex_full_size_c2(fr):
    """The FD operator at 160 x 160, p = 3 (the bench's size and launch
    configuration) against the oracle's product, all 1.6 M outputs."""
    p = 3
    xe, ye = S.uniform_mesh(160)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.Vortex().state(X, Y)
    z0 = S.random_vector(U0.shape, seed=160)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    ctx = fr.Context(xe, ye, p)
    y = ctx.empty()
    shift = 1.0 / (0.435866521508459 * 0.05)
    fr.fr_jv(ctx, _t(U0), _t(R0), _t(z0), shift, y)
    yo = fd_jv(prob, U0, R0, z0, shift)
    assert _rel(y.cpu().numpy(), yo) < TOL_FD


def _term_scale(U0, xe, ye, p):
    """sJ (|D| |F| + |D| |G|) per point: magnitude of the terms whose
    difference is R (oracle-side fluxes, test only)."""
    from oracle.basis import Basis
    from oracle.fr2d import as_grid, flux_x, flux_y, from_grid
    m = Mesh(xe, ye)
    b = Basis(p)
    Q = as_grid(U0, m, p)
    hx = m.hx[None, :, :, None, None]
    hy = m.hy[None, :, :, None, None]
    F = np.abs(0.5 * hy * flux_x(Q))
    G = np.abs(0.5 * hx * flux_y(Q))
    aD = np.abs(b.D)
    S = np.einsum("ik,...jk->...ji", aD, F) + np.einsum("jk,...ki->...ji", aD, G)
    return from_grid(S * 4.0 / (hx * hy), m, p)


# -------------------------------------------------------------------- Jv --
@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("shift", [0.0, 7.5])
def test_jv_matches_oracle(fr, p, shift):
    xe, ye, X, Y = _case("stretched", 6, 5, p, seed=p)
    U0 = S.smooth_random_state(X, Y, seed=7, amp=0.1)
    z0 = S.random_vector(U0.shape, 11)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    ctx = fr.Context(xe, ye, p)
    y = ctx.empty()
    fr.fr_jv(ctx, _t(U0), _t(R0), _t(z0), shift, y)
    yo = fd_jv(prob, U0, R0, z0, shift)
    assert _rel(y.cpu().numpy(), yo) < TOL_FD
    # zero direction gives exactly zero
    fr.fr_jv(ctx, _t(U0), _t(R0), _t(np.zeros_like(z0)), shift, y)
    assert float(y.abs().max()) == 0.0


def test_jv_paper_fixed_epsilon(fr):
    p = 3
    xe, ye, X, Y = _case("uniform", 5, 5, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    z0 = S.random_vector(U0.shape, 2) * 1e-2
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    ctx = fr.Context(xe, ye, p, fr.default_opts(eps_fixed=1e-8))
    y = ctx.empty()
    fr.fr_jv(ctx, _t(U0), _t(R0), _t(z0), 0.0, y)
    yo = fd_jv(prob, U0, R0, z0, 0.0, eps_fixed=1e-8)
    assert _rel(y.cpu().numpy(), yo) < 1e-5


# ------------------------------------------------------- element blocks --
@pytest.mark.parametrize("p", [2, 3, 4])
def test_element_jacobi_apply_matches_oracle(fr, p):
    xe, ye, X, Y = _case("stretched", 5, 4, p, seed=2 * p)
    U0 = S.smooth_random_state(X, Y, seed=17, amp=0.1)
    r0 = S.random_vector(U0.shape, 19)
    shift = 40.0
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p)
    U = _t(U0)
    fr.ejacobi_factor(ctx, U, None, shift)
    z = ctx.empty()
    fr.ejacobi_apply(ctx, _t(r0), z)
    zo = ElementJacobi(element_blocks(prob, U0, shift))(r0)
    assert _rel(z.cpu().numpy(), zo) < TOL_FD


def test_element_jacobi_full_size_sampled(fr):
    """160 x 160, p = 3: blocks of sampled elements (ragged sample incl. the
    first and last element) against the oracle's element-local FD."""
    p = 3
    xe, ye = S.uniform_mesh(160)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.Vortex().state(X, Y)
    shift = 1.0 / (0.25 * 0.05)
    ctx = fr.Context(xe, ye, p)
    fr.ejacobi_factor(ctx, _t(U0), None, shift)
    r0 = S.random_vector(U0.shape, 23)
    z = ctx.empty()
    fr.ejacobi_apply(ctx, _t(r0), z)
    zg = z.cpu().numpy()
    prob = Problem(Mesh(xe, ye), p)
    sample = np.unique(np.concatenate([[0, 159, 160 * 80 + 80, 25599],
                                       np.random.default_rng(0).integers(0, 25600, 60)]))
    M = element_blocks(prob, U0, shift, elements=sample)
    zo = np.linalg.solve(M, r0[sample].reshape(len(sample), -1, 1))[..., 0]
    assert _rel(zg[sample].reshape(len(sample), -1), zo) < TOL_FD


# ----------------------------------------------------------------- GMRES --
@pytest.mark.parametrize("precond", [1, 0])
def test_gmres_matches_oracle(fr, precond):
    p = 2
    xe, ye, X, Y = _case("uniform", 6, 6, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    b0 = S.random_vector(U0.shape, 31)
    shift = 1.0 / (0.43586652150845900 * 0.1)
    ctx = fr.Context(xe, ye, p, fr.default_opts(precond=precond))
    U = _t(U0)
    if precond:
        fr.ejacobi_factor(ctx, U, None, shift)
    x = ctx.empty().zero_()
    info = fr.gmres_solve(ctx, U, _t(R0), shift, _t(b0), x, m=30, rtol=1e-12, max_restarts=40)
    assert info.converged
    Minv = ElementJacobi(element_blocks(prob, U0, shift)) if precond else None
    A = lambda v: fd_jv(prob, U0, R0, v, shift)
    xo, io = gmres(A, b0, None, 30, 1e-12, 40, Minv)
    assert io.converged
    assert _rel(x.cpu().numpy(), xo) < 1e-8
    # iteration counts agree to within the last restart's slack
    assert abs(info.iters - io.iters) <= 2
    # The FD operator is linear only to O(eps): one FD product on x differs
    # from the Krylov combination of FD products on the basis.  The GPU
    # answer's one-product residual must match the oracle answer's.
    rg = np.linalg.norm(b0 - A(x.cpu().numpy()))
    ro = np.linalg.norm(b0 - A(xo))
    assert abs(rg - ro) <= 1e-3 * ro + 1e-9 * np.linalg.norm(b0)


def test_gmres_paper_restart_length_60(fr):
    """The paper's GMRES(60) (restart lengths up to 63 fit the workspace):
    the same answer and iteration count as the oracle's GMRES(60)."""
    p = 2
    xe, ye, X, Y = _case("stretched", 7, 6, p, seed=60)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    b0 = S.random_vector(U0.shape, 60)
    shift = 2.0
    ctx = fr.Context(xe, ye, p, fr.default_opts(m_max=60, gmres_m=60))
    U = _t(U0)
    fr.ejacobi_factor(ctx, U, None, shift)
    x = ctx.empty().zero_()
    info = fr.gmres_solve(ctx, U, _t(R0), shift, _t(b0), x, m=60, rtol=1e-11, max_restarts=20)
    assert info.converged and info.iters > 30
    A = lambda v: fd_jv(prob, U0, R0, v, shift)
    xo, io = gmres(A, b0, None, 60, 1e-11, 20, ElementJacobi(element_blocks(prob, U0, shift)))
    assert io.converged
    assert abs(info.iters - io.iters) <= 3
    assert _rel(x.cpu().numpy(), xo) < 1e-7


@pytest.mark.parametrize("eta", [0.0, 1.0 / 64.0, 1.0])
def test_gmres_orthogonalisation_variants_track_mgs(fr, eta):
    """One classical Gram-Schmidt pass (eta = 0), the selective second pass
    (default) and always two passes (eta = 1) all follow the oracle's
    modified Gram-Schmidt: same iterations, same answer."""
    p = 3
    xe, ye, X, Y = _case("uniform", 8, 8, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    b0 = R0.copy()
    shift = 1.0 / (0.43586652150845900 * 0.2)
    ctx = fr.Context(xe, ye, p, fr.default_opts(reorth_eta=eta))
    U = _t(U0)
    fr.ejacobi_factor(ctx, U, None, shift)
    x = ctx.empty().zero_()
    info = fr.gmres_solve(ctx, U, _t(R0), shift, _t(b0), x, m=30, rtol=1e-10, max_restarts=20)
    Minv = ElementJacobi(element_blocks(prob, U0, shift))
    xo, io = gmres(lambda v: fd_jv(prob, U0, R0, v, shift), b0, None, 30, 1e-10, 20, Minv)
    assert info.converged and io.converged
    assert abs(info.iters - io.iters) <= 1
    assert _rel(x.cpu().numpy(), xo) < 1e-7


def test_gmres_restarts_and_not_converged_status(fr):
    p = 2
    xe, ye, X, Y = _case("uniform", 4, 4, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    b0 = S.random_vector(U0.shape, 3)
    ctx = fr.Context(xe, ye, p, fr.default_opts(precond=0))
    x = ctx.empty().zero_()
    info = fr.gmres_solve(ctx, _t(U0), _t(R0), 2.0, _t(b0), x, m=3, rtol=1e-14, max_restarts=2)
    assert not info.converged and info.code == fr.FR_ERR_NOT_CONVERGED
    assert info.iters == 9 and info.restarts == 2
    xo, io = gmres(lambda v: fd_jv(prob, U0, R0, v, 2.0), b0, None, 3, 1e-14, 2, None)
    assert io.iters == 9
    assert abs(info.relres - io.relres) < 1e-6 * io.relres
    # zero right-hand side: x = 0, converged
    x.fill_(1.0)
    info = fr.gmres_solve(ctx, _t(U0), _t(R0), 2.0, _t(np.zeros_like(b0)), x, m=3, rtol=1e-8)
    assert info.converged and float(x.abs().max()) == 0.0


def test_gmres_nonzero_initial_guess(fr):
    p = 2
    xe, ye, X, Y = _case("uniform", 4, 4, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    R0 = prob.R(U0)
    b0 = S.random_vector(U0.shape, 4)
    shift = 30.0
    ctx = fr.Context(xe, ye, p, fr.default_opts(precond=0))
    U = _t(U0)
    x = ctx.empty().zero_()
    fr.gmres_solve(ctx, U, _t(R0), shift, _t(b0), x, m=30, rtol=1e-12)
    # restarting from a converged answer costs few iterations (the one-product
    # FD residual b - A x is ~1e-6 ||b|| here, not the Krylov 1e-12), and the
    # GPU and the oracle take the same number
    x2 = x.clone()
    info = fr.gmres_solve(ctx, U, _t(R0), shift, _t(b0), x2, m=30, rtol=1e-6)
    xo2, io2 = gmres(lambda v: fd_jv(prob, U0, R0, v, shift), b0, x.cpu().numpy(), 30, 1e-6, 20, None)
    assert info.converged and abs(info.iters - io2.iters) <= 1 and info.iters < 10
    # from a poor guess the GPU and the oracle take the same iterations
    g0 = 0.5 * x.cpu().numpy()
    x3 = _t(g0)
    info = fr.gmres_solve(ctx, U, _t(R0), shift, _t(b0), x3, m=30, rtol=1e-10)
    xo, io = gmres(lambda v: fd_jv(prob, U0, R0, v, shift), b0, g0, 30, 1e-10, 20, None)
    assert abs(info.iters - io.iters) <= 1
    assert _rel(x3.cpu().numpy(), xo) < 1e-8


# -------------------------------------------------------------- steppers --
TIGHT = SolverOpts(tol_lin=1e-12, m=30, max_restarts=40)


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_step_row_matches_oracle(fr, scheme):
    p = 2
    xe, ye, X, Y = _case("uniform", 6, 6, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-12, gmres_max_restarts=40))
    U = _t(U0)
    Uo = U0.copy()
    for _ in range(2):
        st = fr.step_row(ctx, scheme, 0.1, U)
        assert st.converged
        Uo, so = o_row(prob, ROW[scheme](), 0.1, Uo, TIGHT)
    assert _rel(U.cpu().numpy(), Uo) < TOL_RUN


def test_c1_end_of_run_matches_oracle(fr):
    """The plain-method workload: 20 x 20, p = 2, ROW2, 10 steps of 0.05,
    GMRES(30), element-Jacobi; tol_lin = 1e-12 so both sides stop alike."""
    p = 2
    xe, ye = S.uniform_mesh(20)
    X, Y = S.point_coords(xe, ye, p)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-12, gmres_max_restarts=40))
    U = _t(U0)
    Uo = U0.copy()
    for _ in range(10):
        fr.step_row(ctx, 2, 0.05, U)
        Uo, _ = o_row(prob, ROW[2](), 0.05, Uo, TIGHT)
    assert _rel(U.cpu().numpy(), Uo) < TOL_RUN


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_step_esdirk_matches_oracle(fr, scheme):
    p = 2
    xe, ye, X, Y = _case("uniform", 5, 5, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(gmres_max_restarts=40))
    po = fr.default_ptc_opts(tol_nl=1e-12, tol_lin=1e-3)
    U = _t(U0)
    st = fr.step_esdirk(ctx, scheme, 0.1, U, po)
    Uo, so = o_esdirk(prob, ESDIRK[scheme](), 0.1, U0, PtcOpts(tol_nl=1e-12, tol_lin=1e-3), TIGHT)
    assert st.converged and so.converged
    assert _rel(U.cpu().numpy(), Uo) < TOL_RUN


def test_step_bdf2_matches_oracle(fr):
    p = 2
    xe, ye, X, Y = _case("uniform", 5, 5, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(gmres_max_restarts=40))
    po = fr.default_ptc_opts(tol_nl=1e-12, tol_lin=1e-3)
    U = _t(U0)
    Up = ctx.empty()
    Uo, Upo = U0.copy(), None
    for k in range(3):
        fr.step_bdf2(ctx, 0.1, U, Up, k == 0, po)
        Uo, Upo, _ = o_bdf2(prob, 0.1, Uo, Upo, k == 0, PtcOpts(tol_nl=1e-12, tol_lin=1e-3), TIGHT)
    assert _rel(U.cpu().numpy(), Uo) < TOL_RUN
    assert _rel(Up.cpu().numpy(), Upo) < TOL_RUN


def test_ptc_rejection_path_on_gpu(fr):
    """A one-iteration GMRES without preconditioner cannot cut the residual
    by a decade: pseudo steps are rejected until the stall limit."""
    p = 2
    xe, ye, X, Y = _case("uniform", 4, 4, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    ctx = fr.Context(xe, ye, p, fr.default_opts(precond=0, gmres_m=1, gmres_max_restarts=0))
    po = fr.default_ptc_opts(tol_nl=1e-8, tol_lin=1e-1, max_rejections=3, max_iters=5)
    U = _t(U0)
    st = fr.step_esdirk(ctx, 2, 0.5, U, po, allow=(fr.FR_ERR_PTC_STALLED, fr.FR_ERR_NOT_CONVERGED))
    assert st.rejections > 0 and not st.converged
    assert np.array_equal(U.cpu().numpy(), U0)  # a stalled step leaves U unchanged


def test_nonfinite_input_reported(fr):
    p = 2
    xe, ye, X, Y = _case("uniform", 4, 4, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    U0[3, 1, 2] = np.nan
    ctx = fr.Context(xe, ye, p)
    U = _t(U0)
    with pytest.raises(fr.FrError) as ei:
        fr.step_row(ctx, 2, 0.05, U)
    assert ei.value.code == fr.FR_ERR_NONFINITE


def test_step_esdirk_refresh_every_iterate_matches_oracle(fr):
    """precond_refresh = 1 (blocks formed again at every pseudo iterate)
    against the oracle's refresh = "iterate"."""
    p = 2
    xe, ye, X, Y = _case("uniform", 5, 5, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(gmres_max_restarts=40, precond_refresh=1))
    po = fr.default_ptc_opts(tol_nl=1e-12, tol_lin=1e-3)
    U = _t(U0)
    st = fr.step_esdirk(ctx, 3, 0.1, U, po)
    Uo, so = o_esdirk(prob, ESDIRK[3](), 0.1, U0,
                      PtcOpts(tol_nl=1e-12, tol_lin=1e-3, refresh="iterate"), TIGHT)
    assert st.converged and so.converged
    assert _rel(U.cpu().numpy(), Uo) < TOL_RUN


@pytest.mark.parametrize("p", [2, 3, 4])
def test_step_ssprk3_matches_oracle(fr, p):
    """Explicit SSPRK3 steps on a jittered mesh: only the rounding of three
    residual evaluations per step differs, 1e-12 after five steps."""
    from oracle.steppers import step_ssprk3 as o_ssprk3
    xe, ye, X, Y = _case("stretched", 9, 7, p, seed=p)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p)
    U = _t(U0)
    Uo = U0.copy()
    dt = 0.2 * 10.0 / 9 / (3 * math.sqrt(2) * (p + 1))  # CFL 0.2 on the mean cell
    for _ in range(5):
        st = fr.step_ssprk3(ctx, dt, U)
        assert st.residual_evals == 3
        Uo = o_ssprk3(prob, dt, Uo)
    assert _rel(U.cpu().numpy(), Uo) < 1e-12


# ------------------------------------------------------- Roe common flux --
@pytest.mark.parametrize("p", [2, 3, 4])
def test_roe_residual_jv_blocks_match_oracle(fr, p):
    """riemann = 1 (the paper's Roe flux): R(U), the FD operator (FP64 and
    with FP32 linear parts) and the element blocks against the oracle with
    the Roe flux, at the tolerances of the Rusanov tests."""
    from oracle.jfnk import fd_jv
    xe, ye, X, Y = _case("stretched", 11, 9, p, seed=20 + p)
    U0 = S.smooth_random_state(X, Y, seed=40 + p, amp=0.1)
    z0 = S.random_vector(U0.shape, seed=41 + p)
    prob = Problem(Mesh(xe, ye), p, riemann="roe")
    Ro = prob.R(U0)
    ctx = fr.Context(xe, ye, p, fr.default_opts(riemann=1))
    U, z = _t(U0), _t(z0)
    R = ctx.empty()
    fr.fr_residual(ctx, U, R)
    assert _rel(R.cpu().numpy(), Ro) < TOL_R
    # and it differs from the Rusanov residual
    assert _rel(Problem(Mesh(xe, ye), p).R(U0), Ro) > 1e-6
    y = ctx.empty()
    fr.fr_jv(ctx, U, _t(Ro), z, 5.0, y)
    yo = fd_jv(prob, U0, Ro, z0, 5.0)
    assert _rel(y.cpu().numpy(), yo) < TOL_FD
    mix = fr.Context(xe, ye, p, fr.default_opts(riemann=1, jv_precision=1))
    fr.fr_jv(mix, U, _t(Ro), z, 5.0, y)
    assert _rel(y.cpu().numpy(), yo) < 1e-5
    # element blocks through their action z = M^-1 r
    shift = 40.0
    fr.ejacobi_factor(ctx, U, None, shift)
    r0 = S.random_vector(U0.shape, seed=43 + p)
    zg = ctx.empty()
    fr.ejacobi_apply(ctx, _t(r0), zg)
    zo = ElementJacobi(element_blocks(prob, U0, shift))(r0)
    assert _rel(zg.cpu().numpy(), zo) < TOL_FD


def test_roe_step_row_matches_oracle(fr):
    p = 2
    xe, ye, X, Y = _case("uniform", 6, 6, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p, riemann="roe")
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-12, gmres_max_restarts=40, riemann=1))
    U = _t(U0)
    Uo = U0.copy()
    for _ in range(2):
        assert fr.step_row(ctx, 3, 0.1, U).converged
        Uo, _ = o_row(prob, ROW[3](), 0.1, Uo, TIGHT)
    assert _rel(U.cpu().numpy(), Uo) < TOL_RUN


def test_roe_rejected_for_navier_stokes(fr):
    xe, ye = np.linspace(0.0, 2.0, 5), S.channel_y_edges(4)
    with pytest.raises(fr.FrError):
        fr.Context(xe, ye, 2, fr.default_opts(riemann=1, mu=0.01, wall_temperature=1.0), wall_y=True)


# ------------------------------------------------- degrees 5 and 6 (Euler) --
@pytest.mark.parametrize("p", [5, 6])
def test_high_degree_residual_jv_blocks_match_oracle(fr, p):
    """p = 5, 6 (the paper's P6 vortex runs): R(U) and A z at the usual
    tolerances; the element-Jacobi action with FP64 blocks at p = 5 (1e-6)
    and FP32 blocks at p = 6 (196 x 196 FP64 blocks do not fit in shared
    memory; FP32 Gauss-Jordan: 1e-4, as for the other reduced-precision
    tests)."""
    xe, ye, X, Y = _case("stretched", 7, 5, p, seed=50 + p)
    U0 = S.smooth_random_state(X, Y, seed=60 + p, amp=0.1)
    z0 = S.random_vector(U0.shape, seed=61 + p)
    prob = Problem(Mesh(xe, ye), p, riemann="roe")
    R0 = prob.R(U0)
    prec = 0 if p == 5 else 1
    ctx = fr.Context(xe, ye, p, fr.default_opts(riemann=1, block_precision=prec))
    U = _t(U0)
    R = ctx.empty()
    fr.fr_residual(ctx, U, R)
    assert _rel(R.cpu().numpy(), R0) < TOL_R
    y = ctx.empty()
    fr.fr_jv(ctx, U, _t(R0), _t(z0), 4.0, y)
    assert _rel(y.cpu().numpy(), fd_jv(prob, U0, R0, z0, 4.0)) < TOL_FD
    shift = 40.0
    fr.ejacobi_factor(ctx, U, None, shift)
    r0 = S.random_vector(U0.shape, seed=62 + p)
    zg = ctx.empty()
    fr.ejacobi_apply(ctx, _t(r0), zg)
    zo = ElementJacobi(element_blocks(prob, U0, shift))(r0)
    assert _rel(zg.cpu().numpy(), zo) < (TOL_FD if p == 5 else 1e-4)


@pytest.mark.parametrize("p,prec,tol", [(5, 0, TOL_RUN), (6, 1, 3e-8)])
def test_high_degree_step_matches_oracle(fr, p, prec, tol):
    """Two ROW3 steps at p = 5 (FP64 blocks, the usual 1e-9) and p = 6 (FP32
    blocks).  The oracle solves with FP64 blocks; each FD product carries its
    own eps, so the stage solves converge to slightly different points of the
    FD operator's O(eps) nonlinearity along the two preconditioners' Krylov
    paths; at p = 6 the derivative entries ((p+1)^2 = 49) make that spread
    about ten times the p <= 4 one, hence 3e-8 there."""
    xe, ye, X, Y = _case("uniform", 4, 4, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p, riemann="roe")
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-12, gmres_max_restarts=40, riemann=1,
                                                block_precision=prec))
    U = _t(U0)
    Uo = U0.copy()
    for _ in range(2):
        assert fr.step_row(ctx, 3, 0.2, U).converged
        Uo, _ = o_row(prob, ROW[3](), 0.2, Uo, TIGHT)
    assert _rel(U.cpu().numpy(), Uo) < tol


def test_degree_6_fp64_blocks_rejected(fr):
    xe, ye, X, Y = _case("uniform", 4, 4, 6, seed=0)
    with pytest.raises(fr.FrError):
        fr.Context(xe, ye, 6, fr.default_opts(block_precision=0))


def test_step_esdirk_frozen_preconditioner_matches_oracle(fr):
    """precond_refresh = 2 (each stage's first blocks kept, no re-inversion)
    against the oracle's refresh = "frozen"."""
    p = 2
    xe, ye, X, Y = _case("uniform", 5, 5, p, seed=0)
    U0 = S.Vortex().state(X, Y)
    prob = Problem(Mesh(xe, ye), p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(gmres_max_restarts=40, precond_refresh=2))
    po = fr.default_ptc_opts(tol_nl=1e-12, tol_lin=1e-3)
    U = _t(U0)
    st = fr.step_esdirk(ctx, 3, 0.1, U, po)
    Uo, so = o_esdirk(prob, ESDIRK[3](), 0.1, U0,
                      PtcOpts(tol_nl=1e-12, tol_lin=1e-3, refresh="frozen"), TIGHT)
    assert st.converged and so.converged
    assert _rel(U.cpu().numpy(), Uo) < TOL_RUN
