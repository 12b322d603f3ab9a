"""Learned initial guess: the MLP kernels against the oracle MLP, and the
guess inside ROW stage solves.

Tolerances: the training path runs FP32 GEMMs (u_32 = 6e-8, K <= 300 terms),
so forward outputs and gradients match the FP64 oracle to 1e-5 relative; the
BF16 inference path rounds inputs and weights to 8 bits, so it matches the
oracle evaluated on BF16-rounded inputs and weights to 1e-3 relative (FP32
accumulation) and the FP64 network to 3e-2."""
import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import Problem
from oracle.mlp import Adam, backward, forward, init_params
from oracle.steppers import SolverOpts
from oracle.steppers import step_row as o_row
from oracle.tableaus import ROW

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    import paper_1904_04825_gb300 as mod
    return mod


def _f32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


SIZES = [108, 256, 256, 36]


def _setup(fr, M=300, seed=0):
    rng = np.random.default_rng(seed)
    params = init_params(SIZES, seed=seed + 1)
    params = [(W.astype(np.float32).astype(np.float64), (0.1 * rng.standard_normal(b.shape)).astype(np.float32).astype(np.float64))
              for W, b in params]
    X = rng.standard_normal((M, SIZES[0])).astype(np.float32).astype(np.float64)
    T = rng.standard_normal((M, SIZES[-1])).astype(np.float32).astype(np.float64)
    m = fr.MLP(SIZES[0], 256, SIZES[-1], max_batch=M)
    m.set_params(fr.flat_params(params))
    return m, params, X, T


def test_fp32_forward_and_gradients_match_oracle(fr):
    import torch
    m, params, X, T = _setup(fr)
    Y = torch.empty((X.shape[0], SIZES[-1]), dtype=torch.float32, device="cuda")
    m.forward(_f32(X), Y)
    yo, _, _ = forward(params, X)
    assert np.linalg.norm(Y.cpu().numpy() - yo) / np.linalg.norm(yo) < 1e-5
    loss = m.backward(_f32(X), _f32(T))
    assert abs(loss - 0.5 * np.mean((yo - T) ** 2)) < 1e-5 * loss
    g = fr.unflat_params(m.get_grads().astype(np.float64), SIZES)
    go = backward(params, X, T)
    for (gW, gb), (oW, ob) in zip(g, go):
        assert np.linalg.norm(gW - oW) / np.linalg.norm(oW) < 1e-5
        assert np.linalg.norm(gb - ob) / np.linalg.norm(ob) < 1e-5


def test_adam_steps_match_oracle(fr):
    m, params, X, T = _setup(fr, M=200, seed=3)
    opt = Adam(params, lr=1e-3)
    import torch
    Y = torch.empty((X.shape[0], SIZES[-1]), dtype=torch.float32, device="cuda")
    for _ in range(3):
        m.forward(_f32(X), Y)
        m.backward(_f32(X), _f32(T))
        m.adam(1e-3)
        params = opt.step(params, backward(params, X, T))
    got = fr.unflat_params(m.get_params().astype(np.float64), SIZES)
    for (W, b), (Wo, bo) in zip(got, params):
        assert np.max(np.abs(W - Wo)) < 1e-5
        assert np.max(np.abs(b - bo)) < 1e-5


def test_bf16_tensor_core_inference(fr):
    import torch
    m, params, X, T = _setup(fr, M=333, seed=5)
    Y = torch.empty((X.shape[0], SIZES[-1]), dtype=torch.float32, device="cuda")
    m.forward(_f32(X), Y, bf16=True)
    yg = Y.cpu().numpy()
    # oracle with BF16-rounded operands at every layer input (FP32 accumulation on the GPU)
    h = _bf16_round(X)
    for li, (W, b) in enumerate(params):
        z = h @ _bf16_round(W).T + b
        h = _bf16_round(np.maximum(z, 0.0)) if li < 2 else z
    assert np.linalg.norm(yg - h) / np.linalg.norm(h) < 1e-3
    yo, _, _ = forward(params, X)
    assert np.linalg.norm(yg - yo) / np.linalg.norm(yo) < 3e-2


def _bf16_forward(params, X):
    h = _bf16_round(X)
    for li, (W, b) in enumerate(params):
        z = h @ _bf16_round(W).T + b
        h = _bf16_round(np.maximum(z, 0.0)) if li < 2 else z
    return h


@pytest.mark.parametrize("sizes,M", [
    ([20, 64, 64, 7], 5),          # one partial tile everywhere (K 20 -> 24, N 7 -> 16)
    ([300, 256, 256, 100], 1000),  # the p = 4 network shape, ragged last row tile
    ([36, 300, 300, 17], 257),     # hidden width above one 256-column tile
    ([108, 256, 256, 36], 128),    # exactly one row tile
])
def test_tensor_core_gemm_shapes(fr, sizes, M):
    """The tcgen05 GEMMs on ragged shapes: rows, columns and K slices that
    do not fill a tile are zero-filled, so every output matches the oracle
    network on BF16-rounded operands (FP32 accumulation) to 1e-3."""
    import torch
    rng = np.random.default_rng(len(sizes) + M)
    params = [(W.astype(np.float32).astype(np.float64), (0.1 * rng.standard_normal(b.shape)).astype(np.float32).astype(np.float64))
              for W, b in init_params(sizes, seed=M)]
    X = rng.standard_normal((M, sizes[0])).astype(np.float32).astype(np.float64)
    m = fr.MLP(sizes[0], sizes[1], sizes[-1], max_batch=M)
    m.set_params(fr.flat_params(params))
    Y = torch.full((M, sizes[-1]), float("nan"), dtype=torch.float32, device="cuda")
    m.forward(_f32(X), Y, bf16=True)
    yg = Y.cpu().numpy()
    assert np.isfinite(yg).all()
    h = _bf16_forward(params, X)
    assert np.linalg.norm(yg - h) / np.linalg.norm(h) < 1e-3
    assert np.max(np.abs(yg - h)) < 1e-2 * np.max(np.abs(h))


def test_tensor_core_gemm_full_size_sampled(fr):
    """The largest inference (73,728 elements of a 384 x 192 p = 4 mesh,
    300-256-256-100): 512 sampled rows against the oracle."""
    import torch
    sizes, M = [300, 256, 256, 100], 384 * 192
    rng = np.random.default_rng(3)
    params = [(W.astype(np.float32).astype(np.float64), (0.1 * rng.standard_normal(b.shape)).astype(np.float32).astype(np.float64))
              for W, b in init_params(sizes, seed=3)]
    X = rng.standard_normal((M, sizes[0])).astype(np.float32)
    m = fr.MLP(300, 256, 100, max_batch=M)
    m.set_params(fr.flat_params(params))
    Y = torch.empty((M, 100), dtype=torch.float32, device="cuda")
    m.forward(_f32(X), Y, bf16=True)
    rows = np.sort(rng.choice(M, 512, replace=False))
    yg = Y.cpu().numpy()[rows]
    h = _bf16_forward(params, X[rows].astype(np.float64))
    assert np.linalg.norm(yg - h) / np.linalg.norm(h) < 1e-3


def test_learned_guess_in_row_stages(fr):
    """Train on stage solves captured from plain ROW2 steps (zero guess) of
    20 x 20, p = 2 vortices; then run a held-out vortex with the zero guess,
    the previous-step guess and the learned guess at tol_lin = 1e-8.  GMRES
    tests every guess (same absolute target tol * ||b||), so the states
    agree at the tolerance level; the guesses cut iterations.  At
    tol_lin = 1e-12 the learned-guess run matches the oracle to 1e-9."""
    import torch
    p = 2
    xe, ye = S.uniform_mesh(20)
    X0, Y0 = S.point_coords(xe, ye, p)
    nb = 36
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-8, gmres_max_restarts=60))
    maxs = 60000
    Xc = torch.empty((maxs, 3 * nb), dtype=torch.float32, device="cuda")
    Tc = torch.empty((maxs, nb), dtype=torch.float32, device="cuda")
    fr.fr_set_stage_capture(ctx, Xc, Tc, maxs, 1)
    rng = np.random.default_rng(11)
    for seed in range(4):
        v = S.Vortex(x0=float(rng.uniform(-2, 2)), y0=float(rng.uniform(-2, 2)), alpha=float(rng.uniform(3, 6)))
        U = torch.from_numpy(v.state(X0, Y0)).cuda()
        fr.fr_reset_history(ctx)
        for _ in range(4):
            fr.step_row(ctx, 2, 0.05, U)
    n = fr.fr_stage_capture_count(ctx)
    assert n == 4 * 4 * 3 * 400          # vortices x steps x stages x elements
    fr.fr_set_stage_capture(ctx, None, None, 0, 1)
    m = fr.MLP(3 * nb, 256, nb, max_batch=4096)
    m.set_params(fr.flat_params(init_params([3 * nb, 256, 256, nb], seed=7)))
    Yb = torch.empty((4096, nb), dtype=torch.float32, device="cuda")
    losses = []
    for it in range(600):
        idx = torch.from_numpy(rng.integers(0, n, 4096)).cuda()
        xb, tb = Xc[idx].contiguous(), Tc[idx].contiguous()
        m.forward(xb, Yb)
        losses.append(m.backward(xb, tb))
        m.adam(1e-3 if it < 400 else 3e-4)
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:5])

    v = S.Vortex(x0=1.3, y0=-0.7, alpha=4.7)
    U0 = v.state(X0, Y0)
    iters, finals = {}, {}
    c = None
    for mode in (0, 1, 2):
        c = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-8, gmres_max_restarts=60, guess=mode))
        if mode == 2:
            fr.fr_attach_guess_model(c, m)
        U = torch.from_numpy(U0).cuda()
        total = 0
        for k in range(4):
            st = fr.step_row(c, 2, 0.05, U)
            assert st.converged
            total += st.gmres_iters if k > 0 else 0   # first step has no history
        iters[mode] = total
        finals[mode] = U.cpu().numpy()
        if mode < 2:
            c.close()
    tried, used = fr.fr_guess_stats(c)
    print("GMRES iterations over steps 2-4 (zero / previous-step / learned):", iters,
          "learned guess kept in", used, "of", tried, "stage solves")
    assert iters[1] < iters[0]
    assert iters[2] < iters[0]
    assert iters[2] <= iters[1] + 3
    for mode in (1, 2):
        assert np.linalg.norm(finals[mode] - finals[0]) / np.linalg.norm(finals[0]) < 1e-7

    c = fr.Context(xe, ye, p, fr.default_opts(tol_lin=1e-12, gmres_max_restarts=60, guess=2))
    fr.fr_attach_guess_model(c, m)
    U = torch.from_numpy(U0).cuda()
    Uo = U0.copy()
    prob = Problem(Mesh(xe, ye), p)
    for _ in range(2):
        fr.step_row(c, 2, 0.05, U)
        Uo, _ = o_row(prob, ROW[2](), 0.05, Uo, SolverOpts(tol_lin=1e-12, m=30, max_restarts=60))
    assert np.linalg.norm(U.cpu().numpy() - Uo) / np.linalg.norm(Uo) < 1e-9


def test_learned_guess_at_the_channel_workload(fr):
    """The learned guess on its own workload's mesh: the wall-clustered viscous
    channel, 384 x 192 quadrilaterals at p = 4 (7.4 M DOFs, 100 x 100 FP64
    element blocks), ROW3 steps of dt = 1e-3 with GMRES(30) to tol 1e-8.
    A sample of the experiment: training stage solves captured from seeds
    1..4 (the second step of each, after one step of history), 400 Adam
    steps, evaluation on held-out seeds 10001 and 10002 against the zero and
    previous-step guesses.  Checks what the method guarantees: every stage
    solve reaches the same absolute target; the kept learned guess is never
    worse than the previous-step guess by more than a few iterations (the
    safeguard keeps it only when its residual is lower); the end states agree
    at the tolerance level."""
    import torch
    ch = S.Channel()
    nx, ny, p, dt = 384, 192, 4, 1e-3
    xe = np.linspace(0.0, ch.lx, nx + 1)
    ye = S.channel_y_edges(ny, first=1e-3, ratio=1.15)
    X, Y = S.point_coords(xe, ye, p)
    nb = 100

    def opts(mode):
        return fr.default_opts(tol_lin=1e-8, gmres_max_restarts=60, mu=ch.mu, prandtl=ch.prandtl,
                               body_force_x=ch.body_force, wall_temperature=ch.temperature, guess=mode)
    ctx = {m: fr.Context(xe, ye, p, opts(m), wall_y=True) for m in (0, 1, 2)}
    stride = 61
    per_seed = 4 * ((nx * ny + stride - 1) // stride)
    Xc = torch.empty((4 * per_seed, 3 * nb), dtype=torch.float32, device="cuda")
    Tc = torch.empty((4 * per_seed, nb), dtype=torch.float32, device="cuda")
    n = 0
    for s in range(1, 5):
        U = torch.from_numpy(ch.state(X, Y, seed=s)).cuda()
        fr.fr_reset_history(ctx[1])
        assert fr.step_row(ctx[1], 3, dt, U).converged
        fr.fr_set_stage_capture(ctx[1], Xc[n:], Tc[n:], per_seed, stride)
        assert fr.step_row(ctx[1], 3, dt, U).converged
        n += fr.fr_stage_capture_count(ctx[1])
        fr.fr_set_stage_capture(ctx[1], None, None, 0, 1)
    assert 0 < n <= 4 * per_seed
    rng = np.random.default_rng(5)
    model = fr.MLP(3 * nb, 256, nb, max_batch=nx * ny)
    model.set_params(fr.flat_params(init_params([3 * nb, 256, 256, nb], seed=9)))
    Yb = torch.empty((4096, nb), dtype=torch.float32, device="cuda")
    losses = []
    for it in range(400):
        idx = torch.from_numpy(rng.integers(0, n, 4096)).cuda()
        xb, tb = Xc[idx].contiguous(), Tc[idx].contiguous()
        model.forward(xb, Yb)
        losses.append(model.backward(xb, tb))
        model.adam(1e-3)
    assert np.isfinite(losses[-1])
    del Xc, Tc
    fr.fr_attach_guess_model(ctx[2], model)
    iters = {0: [], 1: [], 2: []}
    finals = {}
    for s in (10001, 10002):
        for m in (0, 1, 2):
            U = torch.from_numpy(ch.state(X, Y, seed=s)).cuda()
            fr.fr_reset_history(ctx[m])
            assert fr.step_row(ctx[m], 3, dt, U).converged
            st = fr.step_row(ctx[m], 3, dt, U)
            assert st.converged
            iters[m].append(st.gmres_iters)
            finals[(s, m)] = U.cpu().numpy()
    tried, used = fr.fr_guess_stats(ctx[2])
    print("second-step GMRES iterations (zero / previous-step / learned):", iters,
          "learned guess kept in", used, "of", tried, "stage solves; loss", losses[0], "->", losses[-1])
    for a, b in zip(iters[2], iters[1]):
        assert a <= b + 3
    for s in (10001, 10002):
        ref = finals[(s, 0)]
        for m in (1, 2):
            assert np.linalg.norm(finals[(s, m)] - ref) / np.linalg.norm(ref) < 1e-6
    for c in ctx.values():
        c.close()
