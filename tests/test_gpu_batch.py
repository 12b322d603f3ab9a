"""Batched instances and launch configurations on the GPU.

A batch advances independent instances (own mesh and degree) with one
CUDA-graph launch per GMRES restart cycle for all of them.  Each instance
must take the same iterations as a single-instance ROW step and reach the
same state: the cycle kernels are the single-instance kernels, the
reductions use the same grid, so the states agree to round-off (checked at
1e-12 relative L2; in practice they are identical).  One instance is also
checked against the oracle directly, at the end-of-run tolerance of the
parity tests (1e-9 with tol_lin = 1e-12).

Launch configurations change only the speed: the two residual tile shapes
compute every face and volume term with the same arithmetic (identical
results); another vector-kernel grid changes the summation order of the
reductions (relative 1e-12 on one GMRES solve at tol 1e-12).
"""
import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import Problem
from oracle.steppers import SolverOpts
from oracle.steppers import step_row as o_row
from oracle.tableaus import ROW

pytestmark = pytest.mark.gpu

TIGHT = SolverOpts(tol_lin=1e-12, m=30, max_restarts=40)
# instances of uneven size and degree (nx, ny, p, stretched?)
CASES = [(8, 8, 2, False), (12, 10, 3, True), (6, 6, 4, False), (16, 16, 3, False), (5, 9, 2, True)]


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1904_04825_gb300 as mod
    return mod


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _instances():
    out = []
    for k, (nx, ny, p, st) in enumerate(CASES):
        if st:
            xe, ye = S.stretched_mesh(nx, ny, seed=k)
        else:
            xe, ye = S.uniform_mesh(nx, ny=ny)
        X, Y = S.point_coords(xe, ye, p)
        box = (xe[0], xe[-1], ye[0], ye[-1])
        v = S.Vortex(x0=0.5 * (box[0] + box[1]) + 0.3 * k / len(CASES), y0=0.5 * (box[2] + box[3]))
        out.append((xe, ye, p, v.state(X, Y)))
    return out


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_batch_matches_single_instance_steps(fr, scheme):
    inst = _instances()
    opts = fr.default_opts(tol_lin=1e-10, gmres_max_restarts=40)
    B = fr.Batch([(xe, ye) for xe, ye, _, _ in inst], [p for _, _, p, _ in inst], opts)
    Ub = [_t(U0) for *_, U0 in inst]
    singles = [fr.Context(xe, ye, p, opts) for xe, ye, p, _ in inst]
    Us = [_t(U0) for *_, U0 in inst]
    launches = fr.fr_kernel_launches()
    for _ in range(3):  # the first step captures the cycle graphs, the others replay them
        stb = B.step_row(scheme, 0.1, Ub)
        for ctx, U, sb in zip(singles, Us, stb):
            ss = fr.step_row(ctx, scheme, 0.1, U)
            assert sb.converged and ss.converged
            assert sb.gmres_iters == ss.gmres_iters
            assert sb.gmres_calls == ss.gmres_calls == ROW[scheme]().stages
            assert sb.residual_evals == ss.residual_evals
    for U, V in zip(Ub, Us):
        assert _rel(U.cpu().numpy(), V.cpu().numpy()) < 1e-12
    assert fr.fr_kernel_launches() > launches


def test_batch_member_matches_oracle(fr):
    inst = _instances()
    opts = fr.default_opts(tol_lin=1e-12, gmres_max_restarts=40)
    B = fr.Batch([(xe, ye) for xe, ye, _, _ in inst], [p for _, _, p, _ in inst], opts)
    Ub = [_t(U0) for *_, U0 in inst]
    k = 1  # the stretched p = 3 instance
    xe, ye, p, U0 = inst[k]
    prob = Problem(Mesh(xe, ye), p)
    Uo = U0.copy()
    for _ in range(2):
        B.step_row(3, 0.1, Ub)
        Uo, _ = o_row(prob, ROW[3](), 0.1, Uo, TIGHT)
    assert _rel(Ub[k].cpu().numpy(), Uo) < 1e-9


def test_batch_recaptures_when_states_move(fr):
    """New state buffers (another U pointer) and another dt must not replay a
    stale graph: the result equals single-instance steps again."""
    inst = _instances()[:3]
    opts = fr.default_opts(tol_lin=1e-10, gmres_max_restarts=40)
    B = fr.Batch([(xe, ye) for xe, ye, _, _ in inst], [p for _, _, p, _ in inst], opts)
    singles = [fr.Context(xe, ye, p, opts) for xe, ye, p, _ in inst]
    for dt in (0.1, 0.05):
        Ub = [_t(U0) for *_, U0 in inst]  # fresh buffers each round
        Us = [_t(U0) for *_, U0 in inst]
        B.step_row(3, dt, Ub)
        for ctx, U in zip(singles, Us):
            fr.step_row(ctx, 3, dt, U)
        for U, V in zip(Ub, Us):
            assert _rel(U.cpu().numpy(), V.cpu().numpy()) < 1e-12


def test_batch_errors(fr):
    inst = _instances()[:2]
    with pytest.raises(fr.FrError):
        fr.Batch([(xe, ye) for xe, ye, _, _ in inst], [p for _, _, p, _ in inst], fr.default_opts(guess=1))
    B = fr.Batch([(xe, ye) for xe, ye, _, _ in inst], [p for _, _, p, _ in inst])
    Ub = [_t(U0) for *_, U0 in inst]
    with pytest.raises(fr.FrError):
        B.step_row(7, 0.1, Ub)
    with pytest.raises(fr.FrError):
        B.step_row(3, -1.0, Ub)
    with pytest.raises(ValueError):
        B.step_row(3, 0.1, Ub[:1])
    # states untouched by the rejected calls
    for U, (*_, U0) in zip(Ub, inst):
        assert np.array_equal(U.cpu().numpy(), U0)


def test_tile_variants_give_identical_residuals(fr):
    for p in (2, 3, 4):
        xe, ye = S.stretched_mesh(23, 17, seed=p)
        X, Y = S.point_coords(xe, ye, p)
        U = _t(S.smooth_random_state(X, Y, seed=p, amp=0.1))
        ctx = fr.Context(xe, ye, p)
        out = []
        for tv in (0, 1):
            fr.set_launch_config(ctx, 456, tv)
            assert fr.get_launch_config(ctx) == (456, tv)
            R = ctx.empty()
            fr.fr_residual(ctx, U, R)
            out.append(R.cpu().numpy())
        assert np.array_equal(out[0], out[1])


def test_vector_grid_changes_only_rounding(fr):
    p = 3
    xe, ye = S.uniform_mesh(24)
    X, Y = S.point_coords(xe, ye, p)
    U = _t(S.Vortex().state(X, Y))
    ctx = fr.Context(xe, ye, p)
    R0 = ctx.empty()
    fr.fr_residual(ctx, U, R0)
    shift = 1.0 / 0.05
    xs = []
    for vb in (152, 456, 1216, 4096):
        fr.set_launch_config(ctx, vb, 0)
        fr.ejacobi_factor(ctx, U, R0, shift)
        x = ctx.empty().zero_()
        info = fr.gmres_solve(ctx, U, R0, shift, R0, x, m=30, rtol=1e-12, max_restarts=40)
        assert info.converged
        xs.append(x.cpu().numpy())
    for x in xs[1:]:
        assert _rel(x, xs[0]) < 1e-10
    with pytest.raises(fr.FrError):
        fr.set_launch_config(ctx, 0, 0)
    with pytest.raises(fr.FrError):
        fr.set_launch_config(ctx, 456, 2)


def test_autotune_picks_a_candidate(fr):
    p = 3
    xe, ye = S.uniform_mesh(32)
    X, Y = S.point_coords(xe, ye, p)
    U = _t(S.Vortex().state(X, Y))
    ctx = fr.Context(xe, ye, p, fr.default_opts(gmres_m=10))
    vb, tv, best, dflt = fr.autotune(ctx, U, 20.0, reps=1)
    assert vb in (152, 304, 456, 608, 912, 1216) and tv in (0, 1)
    assert 0.0 < best <= dflt
    # the context still solves correctly after tuning
    R0 = ctx.empty()
    fr.fr_residual(ctx, U, R0)
    st = fr.step_row(ctx, 3, 0.05, U)
    assert st.converged


@pytest.mark.parametrize("scheme", [2, 4])
def test_batch_esdirk_matches_single_instance_steps(fr, scheme):
    inst = _instances()
    opts = fr.default_opts(gmres_max_restarts=40)
    ptc = fr.default_ptc_opts(tol_nl=1e-8, tol_lin=1e-2)
    B = fr.Batch([(xe, ye) for xe, ye, _, _ in inst], [p for _, _, p, _ in inst], opts)
    Ub = [_t(U0) for *_, U0 in inst]
    singles = [fr.Context(xe, ye, p, opts) for xe, ye, p, _ in inst]
    Us = [_t(U0) for *_, U0 in inst]
    for threads in (0, 2):
        stb = B.step_esdirk(scheme, 0.1, Ub, ptc, threads=threads)
        for ctx, U, sb in zip(singles, Us, stb):
            ss = fr.step_esdirk(ctx, scheme, 0.1, U, ptc)
            assert sb.converged and ss.converged
            assert (sb.gmres_iters, sb.ptc_iters, sb.rejections) == (ss.gmres_iters, ss.ptc_iters, ss.rejections)
    for U, V in zip(Ub, Us):
        assert np.array_equal(U.cpu().numpy(), V.cpu().numpy())


def test_batch_bdf2_matches_single_instance_steps(fr):
    import torch
    inst = _instances()[:3]
    opts = fr.default_opts(gmres_max_restarts=40)
    ptc = fr.default_ptc_opts(tol_nl=1e-8, tol_lin=1e-2)
    B = fr.Batch([(xe, ye) for xe, ye, _, _ in inst], [p for _, _, p, _ in inst], opts)
    Ub = [_t(U0) for *_, U0 in inst]
    Pb = [torch.empty_like(U) for U in Ub]
    singles = [fr.Context(xe, ye, p, opts) for xe, ye, p, _ in inst]
    Us = [_t(U0) for *_, U0 in inst]
    Ps = [torch.empty_like(U) for U in Us]
    for step in range(2):
        B.step_bdf2(0.1, Ub, Pb, step == 0, ptc)
        for ctx, U, P in zip(singles, Us, Ps):
            fr.step_bdf2(ctx, 0.1, U, P, step == 0, ptc)
    for U, V in zip(Ub + Pb, Us + Ps):
        assert np.array_equal(U.cpu().numpy(), V.cpu().numpy())


def test_seeded_batch_instances_run(fr):
    """A few members of the seeded uneven batch (random centres, strengths
    and flow angles) on their own meshes: a batched ROW4 step with BF16
    blocks converges and keeps every state finite and positive."""
    import synthetic as S2
    inst = [i for i in S2.batch_instances(64, seed=0) if i.n <= 48][:6]
    opts = fr.default_opts(tol_lin=1e-6, block_precision=2)
    B = fr.Batch([i.mesh() for i in inst], [i.p for i in inst], opts)
    Ub = [_t(i.state()) for i in inst]
    st = B.step_row(4, 0.05, Ub)
    for s, U in zip(st, Ub):
        u = U.cpu().numpy()
        assert s.converged and np.isfinite(u).all() and u[:, 0].min() > 0.0


def test_batched_arnoldi_launches_equal_per_instance_cycles(fr):
    """The batched Arnoldi launches (one grid per kernel over all instances)
    reproduce the per-instance cycle kernels bit for bit (each instance keeps
    its own CTA partition, so every reduction sums in the same order), with
    far fewer kernel nodes per cycle graph."""
    inst = _instances()
    opts = fr.default_opts(tol_lin=1e-10, gmres_max_restarts=40)
    meshes = [(xe, ye) for xe, ye, _, _ in inst]
    degs = [p for _, _, p, _ in inst]
    res, nodes = {}, {}
    for on in (True, False):
        B = fr.Batch(meshes, degs, opts)
        B.set_batched(on)
        Us = [_t(U0) for *_, U0 in inst]
        its = []
        for _ in range(2):
            its.append([s.gmres_iters for s in B.step_row(4, 0.1, Us)])
        res[on] = ([U.cpu().numpy() for U in Us], its)
        nodes[on] = B.cycle_kernels()
        B.close()
    assert res[True][1] == res[False][1]
    for a, b in zip(res[True][0], res[False][0]):
        assert np.array_equal(a, b)
    m = opts.gmres_m
    # per Arnoldi iteration: 7 kernels per instance, against 7 batched
    # launches per degree present (apply, FD operator, two Gram-Schmidt
    # passes of two kernels, Givens), plus the per-instance cycle set-up and end
    assert nodes[False] >= 7 * m * len(inst)
    assert nodes[True] <= 7 * len(set(degs)) * m + 20 * len(inst)
