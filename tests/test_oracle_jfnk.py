"""Pins of the oracle JFNK pieces (oracle/jfnk.py)."""
import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import (ElementJacobi, Problem, brute_jacobian, element_blocks,
                         element_jacobians, fd_epsilon, fd_jv, gmres)


@pytest.fixture(scope="module")
def tiny():
    p = 2
    xe, ye = S.stretched_mesh(2, 2, seed=4)
    prob = Problem(Mesh(xe, ye), p)
    X, Y = S.point_coords(xe, ye, p)
    U = S.smooth_random_state(X, Y, seed=9, amp=0.1)
    J = brute_jacobian(prob, U)
    return prob, U, J


def test_fd_jv_matches_brute_force_jacobian(tiny):
    prob, U, J = tiny
    R0 = prob.R(U)
    for seed, shift in [(1, 0.0), (2, 3.5)]:
        z = S.random_vector(U.shape, seed)
        y = fd_jv(prob, U, R0, z, shift)
        exact = shift * z - (J @ z.reshape(-1)).reshape(U.shape)
        assert np.linalg.norm(y - exact) / np.linalg.norm(exact) < 2e-6


def test_fd_jv_paper_fixed_epsilon(tiny):
    prob, U, J = tiny
    R0 = prob.R(U)
    z = S.random_vector(U.shape, 5) * 1e-2
    y = fd_jv(prob, U, R0, z, 0.0, eps_fixed=1e-8)
    exact = -(J @ z.reshape(-1)).reshape(U.shape)
    assert np.linalg.norm(y - exact) / np.linalg.norm(exact) < 1e-5


def test_fd_jv_zero_and_linearity(tiny):
    prob, U, _ = tiny
    R0 = prob.R(U)
    assert np.all(fd_jv(prob, U, R0, np.zeros_like(U), 2.0) == 0.0)
    z = S.random_vector(U.shape, 3)
    y1 = fd_jv(prob, U, R0, z, 0.0)
    y2 = fd_jv(prob, U, R0, 2.0 * z, 0.0)
    assert np.linalg.norm(y2 - 2 * y1) / np.linalg.norm(y1) < 1e-6
    # epsilon rule 1e-7 (1 + ||U||) / ||z||
    assert fd_epsilon(U, z) == pytest.approx(1e-7 * (1 + np.sqrt(np.sum(U * U))) / np.sqrt(np.sum(z * z)))


def test_element_blocks_match_brute_force_diagonal_blocks(tiny):
    prob, U, J = tiny
    nb = prob.nb
    Je = element_jacobians(prob, U)
    scale = np.max(np.abs(J))
    for e in range(prob.mesh.ne):
        diag = J[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb]
        assert np.max(np.abs(Je[e] - diag)) < 1e-5 * scale
    # off-diagonal blocks are not part of the preconditioner but must exist
    assert np.max(np.abs(J[:nb, nb:2 * nb])) > 1e-3 * scale
    M = element_blocks(prob, U, 4.0)
    assert np.allclose(M[0], 4.0 * np.eye(nb) - Je[0])


def test_element_jacobi_apply_inverts_blocks(tiny):
    prob, U, _ = tiny
    M = element_blocks(prob, U, 10.0)
    r = S.random_vector(U.shape, 8)
    z = ElementJacobi(M)(r)
    back = np.einsum("eij,ej->ei", M, z.reshape(prob.mesh.ne, -1)).reshape(U.shape)
    assert np.max(np.abs(back - r)) < 1e-12 * np.max(np.abs(r))


def _nonsym(n, seed, shift=6.0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n)) / np.sqrt(n) + shift * np.eye(n) * 0.3


@pytest.mark.parametrize("n", [10, 40, 120])
def test_gmres_exact_when_m_at_least_n(n):
    A = _nonsym(n, n)
    b = np.random.default_rng(n + 1).standard_normal(n)
    x, info = gmres(lambda v: A @ v, b, m=n, rtol=1e-14, max_restarts=0)
    xd = np.linalg.solve(A, b)
    assert np.max(np.abs(x - xd)) < 1e-11 * np.max(np.abs(xd))
    assert info.iters <= n


def test_gmres_restarted_monotone_and_reaches_tolerance():
    n = 150
    A = _nonsym(n, 3)
    b = np.random.default_rng(4).standard_normal(n)
    x, info = gmres(lambda v: A @ v, b, m=8, rtol=1e-10, max_restarts=500)
    assert info.converged
    h = np.array(info.history)
    assert np.all(np.diff(h) <= 1e-12)
    assert np.linalg.norm(b - A @ x) <= 1.01e-10 * np.linalg.norm(b)
    assert info.restarts > 0


def test_gmres_right_preconditioned_block_jacobi():
    rng = np.random.default_rng(7)
    nblk, bs = 12, 6
    n = nblk * bs
    A = 0.05 * rng.standard_normal((n, n))
    blocks = rng.standard_normal((nblk, bs, bs)) + 4 * np.eye(bs)
    for e in range(nblk):
        A[e * bs:(e + 1) * bs, e * bs:(e + 1) * bs] += blocks[e]
    b = rng.standard_normal(n)
    Minv = lambda r: np.linalg.solve(blocks, r.reshape(nblk, bs, 1))[..., 0].reshape(-1)
    x1, i1 = gmres(lambda v: A @ v, b, m=40, rtol=1e-12, max_restarts=10)
    x2, i2 = gmres(lambda v: A @ v, b, m=40, rtol=1e-12, max_restarts=10, apply_Minv=Minv)
    xd = np.linalg.solve(A, b)
    assert np.allclose(x1, xd, atol=1e-10) and np.allclose(x2, xd, atol=1e-10)
    assert i2.iters < i1.iters


def test_gmres_zero_rhs_and_initial_guess():
    A = _nonsym(20, 5)
    x, info = gmres(lambda v: A @ v, np.zeros(20), m=5)
    assert info.converged and np.all(x == 0)
    b = np.random.default_rng(2).standard_normal(20)
    xd = np.linalg.solve(A, b)
    x, info = gmres(lambda v: A @ v, b, x0=xd, m=5, rtol=1e-10)
    assert info.iters == 0 and info.converged


def test_gmres_stops_at_max_restarts():
    A = _nonsym(100, 9, shift=0.5)
    b = np.ones(100)
    x, info = gmres(lambda v: A @ v, b, m=3, rtol=1e-14, max_restarts=2)
    assert not info.converged
    assert info.iters == 9 and info.restarts == 2
