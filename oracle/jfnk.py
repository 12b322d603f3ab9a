"""Jacobian-free linear algebra of Sec. 4.5.

* ``fd_jv``: the finite-difference Jacobian-vector product
  (dR/dq) z ~ (R(q + eps z) - R(q)) / eps, applied as the operator
  A z = shift * z - (dR/dq) z of Eq. linear with D = shift * I.
  eps = 1e-7 (1 + ||q||_2) / ||z||_2 by default (global Euclidean norms over
  all DOFs); the paper's fixed eps = 1e-8 is available via ``eps_fixed``.
  A zero z gives A z = 0.
* ``brute_jacobian``: the full dR/dq column by column by central differences
  (test fixture for tiny meshes).
* ``element_blocks``: the element-Jacobi preconditioner (the diagonal blocks of
  the Jacobian, Sec. 4.5).  The paper does not say how the blocks are formed;
  here J_ee = dR_e/dq_e with every neighbour trace frozen, by forward
  differences with eps_j = 1e-7 (1 + |q_j|), and M_e = shift * I - J_ee.
  Rows and columns are ordered like the element's slice of the state
  (variable-major, then point).
* ``gmres``: restarted GMRES(m) with right preconditioning, modified
  Gram-Schmidt Arnoldi, Givens rotations on the Hessenberg matrix.  The
  relative tolerance is against ||b|| (the first residual of a zero initial
  guess, Sec. 5.1), and the stopping test uses the Givens residual estimate.

Pins (tests/test_oracle_jfnk.py): Jv against brute-force J v on a 2x2 mesh;
blocks against the brute-force Jacobian's diagonal blocks; GMRES against a
dense solve on small nonsymmetric systems, with exactness at m >= N and a
monotone restarted residual.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .basis import Basis
from .fr2d import Mesh, as_grid, from_grid, local_residual, neighbour_traces, residual


class Problem:
    """A mesh, a degree and the 1D basis: what R(q) needs.  With ``viscous``
    (an ``ns2d.Viscous``) R is the Navier-Stokes BR2 residual."""

    def __init__(self, mesh: Mesh, p: int, gamma: float = 1.4, viscous=None, riemann: str = "rusanov"):
        if viscous is not None and riemann != "rusanov":
            raise ValueError("the Navier-Stokes residual uses the Rusanov flux")
        self.riemann = riemann
        self.mesh = mesh
        self.p = p
        self.np = (p + 1) ** 2
        self.nb = 4 * self.np
        self.basis = Basis(p)
        self.gamma = gamma
        self.viscous = viscous
        self.n_residuals = 0

    @property
    def ndof(self):
        return self.mesh.ne * self.nb

    def R(self, U):
        self.n_residuals += 1
        if self.viscous is not None:
            from .ns2d import ns_residual
            return ns_residual(U, self.mesh, self.p, self.viscous, self.basis)
        return residual(U, self.mesh, self.p, self.basis, self.gamma, self.riemann)


def fd_epsilon(U, z, eps_rel=1e-7, eps_fixed=None):
    zn = np.linalg.norm(z)
    if zn == 0.0:
        return 0.0
    if eps_fixed is not None:
        return eps_fixed
    return eps_rel * (1.0 + np.linalg.norm(U)) / zn


def fd_jv(prob: Problem, U, R0, z, shift=0.0, eps_rel=1e-7, eps_fixed=None):
    """A z = shift z - (R(U + eps z) - R0)/eps."""
    eps = fd_epsilon(U, z, eps_rel, eps_fixed)
    if eps == 0.0:
        return np.zeros_like(z)
    return shift * z - (prob.R(U + eps * z) - R0) / eps


def brute_jacobian(prob: Problem, U):
    """dR/dq (N x N) by central differences, step 1e-6 max(1, |U_j|)."""
    u = np.asarray(U, dtype=np.float64).reshape(-1)
    n = u.size
    J = np.zeros((n, n))
    for j in range(n):
        h = 1e-6 * max(1.0, abs(u[j]))
        up = u.copy(); up[j] += h
        um = u.copy(); um[j] -= h
        J[:, j] = (prob.R(up.reshape(U.shape)) - prob.R(um.reshape(U.shape))).reshape(-1) / (2 * h)
    return J


def element_jacobians(prob: Problem, U, elements=None, eps_rel=1e-7):
    """J_ee = dR_e/dq_e with the neighbour traces frozen (forward FD).

    Returns (len(elements), nb, nb); row/column index = var*Np + point."""
    mesh, p, b = prob.mesh, prob.p, prob.basis
    n = p + 1
    Q = as_grid(U, mesh, p)                          # (4, ny, nx, n, n)
    nW, nE, nS, nN = neighbour_traces(Q, b)          # (4, ny, nx, n)
    if elements is None:
        elements = np.arange(mesh.ne)
    elements = np.asarray(elements)
    iy, ix = np.divmod(elements, mesh.nx)
    Qe = Q[:, iy, ix]                                # (4, E, n, n)
    args = [t[:, iy, ix] for t in (nW, nE, nS, nN)]
    hx = mesh.hx[iy, ix]
    hy = mesh.hy[iy, ix]
    R0 = local_residual(Qe, hx, hy, *args, b, prob.gamma, prob.riemann).reshape(4, len(elements), n * n)
    q0 = Qe.reshape(4, len(elements), n * n)
    nb = 4 * n * n
    J = np.zeros((len(elements), nb, nb))
    for col in range(nb):
        v, pt = divmod(col, n * n)
        eps = eps_rel * (1.0 + np.abs(q0[v, :, pt]))          # (E,)
        Qp = q0.copy()
        Qp[v, :, pt] += eps
        Rp = local_residual(Qp.reshape(4, len(elements), n, n), hx, hy, *args, b,
                            prob.gamma, prob.riemann).reshape(4, len(elements), n * n)
        J[:, :, col] = ((Rp - R0) / eps[None, :, None]).transpose(1, 0, 2).reshape(len(elements), nb)
    return J


def diagonal_blocks(prob: Problem, U, elements=None, eps_rel=1e-7):
    """J_ee for the Euler or the Navier-Stokes residual of ``prob`` (a
    problem with its own ``element_jacobians``, such as the 3D one, forms them)."""
    if hasattr(prob, "element_jacobians"):
        return prob.element_jacobians(U, elements, eps_rel)
    if prob.viscous is not None:
        from .ns2d import ns_element_jacobians
        return ns_element_jacobians(U, prob.mesh, prob.p, prob.viscous, elements, eps_rel, prob.basis)
    return element_jacobians(prob, U, elements, eps_rel)


def element_blocks(prob: Problem, U, shift, elements=None, eps_rel=1e-7):
    """M_e = shift * I - J_ee for each requested element."""
    J = diagonal_blocks(prob, U, elements, eps_rel)
    return shift * np.eye(J.shape[1])[None] - J


class ElementJacobi:
    """z_e = M_e^{-1} r_e, each block solved by a dense LU solve."""

    def __init__(self, blocks):
        self.blocks = blocks

    def __call__(self, r):
        ne, nb = self.blocks.shape[0], self.blocks.shape[1]
        rr = np.asarray(r).reshape(ne, nb)
        return np.linalg.solve(self.blocks, rr[..., None])[..., 0].reshape(np.shape(r))


@dataclass
class GmresInfo:
    iters: int = 0
    restarts: int = 0
    relres: float = 0.0
    converged: bool = False
    history: list = field(default_factory=list)


def gmres(apply_A, b, x0=None, m=30, rtol=1e-8, max_restarts=20, apply_Minv=None):
    """Restarted right-preconditioned GMRES(m) with MGS and Givens rotations.

    Runs at most ``max_restarts + 1`` cycles of at most ``m`` iterations.
    Stops when the Givens estimate of ||b - A x|| is <= rtol * ||b||."""
    shape = np.shape(b)
    bv = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(bv) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
    Minv = (lambda v: v) if apply_Minv is None else (lambda v: np.asarray(apply_Minv(v.reshape(shape))).reshape(-1))
    A = lambda v: np.asarray(apply_A(v.reshape(shape))).reshape(-1)
    info = GmresInfo()
    bnorm = np.linalg.norm(bv)
    if bnorm == 0.0:
        info.converged = True
        return np.zeros(shape), info
    target = rtol * bnorm
    for cycle in range(max_restarts + 1):
        r = bv - A(x) if np.any(x) else bv.copy()
        beta = np.linalg.norm(r)
        info.relres = beta / bnorm
        if beta <= target:
            info.converged = True
            break
        if cycle > 0:
            info.restarts += 1
        V = np.zeros((m + 1, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = A(Minv(V[j]))
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                     # earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            info.iters += 1
            info.history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= target or den == 0.0:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):             # back substitution
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + Minv(V[:k].T @ y)
        info.relres = abs(g[k]) / bnorm
        if abs(g[k]) <= target:
            info.converged = True
            break
    return x.reshape(shape), info
