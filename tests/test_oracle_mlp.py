"""Pins of the oracle MLP (oracle/mlp.py)."""
import numpy as np

from oracle.mlp import Adam, backward, forward, init_params, loss, stage_features


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    params = init_params([12, 9, 7, 5], seed=1)
    X = rng.standard_normal((6, 12))
    Y = rng.standard_normal((6, 5))
    grads = backward(params, X, Y)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g, name in ((W, grads[li][0], "W"), (b, grads[li][1], "b")):
            idx = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(5)]
            for ij in idx:
                orig = arr[ij]
                arr[ij] = orig + h
                lp = loss(params, X, Y)
                arr[ij] = orig - h
                lm = loss(params, X, Y)
                arr[ij] = orig
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[ij]) < 1e-7 * max(1.0, abs(fd)), (li, name, ij, fd, g[ij])


def test_adam_first_step_is_signed_learning_rate():
    params = init_params([4, 3], seed=2)
    grads = [(np.full((3, 4), 0.3), np.array([-2.0, 5.0, 1e-3]))]
    opt = Adam(params, lr=0.01)
    new = opt.step(params, grads)
    assert np.allclose(new[0][0] - params[0][0], -0.01, atol=1e-8)
    assert np.allclose(new[0][1] - params[0][1], [0.01, -0.01, -0.01], atol=1e-6)


def test_learns_a_linear_map():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 6)) * 0.5
    X = rng.standard_normal((512, 6))
    Y = X @ A.T
    params = init_params([6, 32, 32, 3], seed=4)
    opt = Adam(params, lr=3e-3)
    l0 = loss(params, X, Y)
    for _ in range(600):
        params = opt.step(params, backward(params, X, Y))
    assert loss(params, X, Y) < 0.02 * l0


def test_stage_features_scale_invariant():
    rng = np.random.default_rng(5)
    b = rng.standard_normal((3, 4, 9))
    Y = rng.standard_normal((3, 4, 9))
    U = rng.standard_normal((3, 4, 9)) + 2
    X1, s1 = stage_features(b, Y, U)
    X2, s2 = stage_features(10 * b, 10 * Y, U)
    assert np.allclose(X1, X2) and np.isclose(s2, 10 * s1)
    assert X1.shape == (3, 3 * 36)
