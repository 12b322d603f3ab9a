"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module only *places* problem data: mesh edge coordinates, physical
coordinates of sample points, the isentropic-vortex initial state of Sec. 5.1
(Eq. VP_Solution), smooth random states and random vectors.  It holds none of
the flux-reconstruction, Krylov or time-integration arithmetic, and it imports
neither the oracle nor the CUDA package.

Point layout used everywhere: state arrays have shape ``(Ne, 4, Np)`` with
``Np = (p+1)**2``; point ``i + (p+1)*j`` is the i-th node along x and the j-th
node along y; element ``ix + Nx*iy``.  Variables are the conserved
``(rho, rho*u, rho*v, E)`` of Sec. 2 in two dimensions.

The node positions used to *place* a field come from NumPy's Gauss-Legendre
routine; they only decide where the smooth input field is sampled.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 1.4


def uniform_edges(n: int, lo: float, hi: float) -> np.ndarray:
    """``n+1`` equally spaced element edges on ``[lo, hi]``."""
    return np.linspace(lo, hi, n + 1, dtype=np.float64)


def channel_y_edges(ny: int, first: float = 1e-3, ratio: float = 1.15,
                    height: float = 1.0) -> np.ndarray:
    """Wall-clustered edges on ``[0, height]``.

    Cells grow geometrically by ``ratio`` from ``first`` at each wall until
    they reach the uniform size that fills the rest of each half, which is
    kept from then on (the capped reading of the stretched channel mesh).
    """
    if ny % 2:
        raise ValueError("ny must be even")
    half = ny // 2
    half_h = 0.5 * height
    # find the number of geometric cells g such that the remaining uniform
    # cells are at least as large as the last geometric cell
    best = None
    for g in range(0, half + 1):
        geo = [first * ratio ** k for k in range(g)]
        rest = half - g
        if rest == 0:
            if abs(sum(geo) - half_h) / half_h < 1e-9:
                best = (g, geo, 0.0)
            continue
        u = (half_h - sum(geo)) / rest
        if u <= 0:
            break
        if not geo or u >= geo[-1] * ratio * 0.999999:
            best = (g, geo, u)
        else:
            break
    if best is None:
        raise ValueError("cannot build the stretched half-channel")
    g, geo, u = best
    sizes = geo + [u] * (half - g)
    lower = np.concatenate([[0.0], np.cumsum(sizes)])
    lower[-1] = half_h
    upper = height - lower[::-1]
    return np.concatenate([lower, upper[1:]])


def sample_nodes(p: int) -> np.ndarray:
    """Gauss-Legendre nodes on [-1, 1] used to place sample points."""
    x, _ = np.polynomial.legendre.leggauss(p + 1)
    return x


def point_coords(x_edges: np.ndarray, y_edges: np.ndarray, p: int):
    """Physical coordinates ``X, Y`` of shape ``(Ne, Np)`` in the point layout."""
    s = sample_nodes(p)
    nx, ny = len(x_edges) - 1, len(y_edges) - 1
    xa, hx = x_edges[:-1], np.diff(x_edges)
    ya, hy = y_edges[:-1], np.diff(y_edges)
    # (ny, nx, p+1 [j], p+1 [i])
    X = xa[None, :, None, None] + 0.5 * (s[None, None, None, :] + 1.0) * hx[None, :, None, None]
    Y = ya[:, None, None, None] + 0.5 * (s[None, None, :, None] + 1.0) * hy[:, None, None, None]
    X = np.broadcast_to(X, (ny, nx, p + 1, p + 1)).reshape(nx * ny, (p + 1) ** 2)
    Y = np.broadcast_to(Y, (ny, nx, p + 1, p + 1)).reshape(nx * ny, (p + 1) ** 2)
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def conserved(rho, u, v, pr, gamma: float = GAMMA) -> np.ndarray:
    """Stack primitive fields into conserved ``(Ne, 4, Np)``."""
    E = pr / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, E], axis=1))


@dataclass(frozen=True)
class Vortex:
    """Isentropic vortex of Sec. 5.1 (Eq. VP_Solution).

    Free stream density 1, speed ``sqrt(2)`` along angle ``theta`` (45 degrees
    gives u = v = 1), Mach number ``mach`` on that speed, gas constant R = 1,
    strength ``alpha`` and ``phi``.  ``r`` is read as the Euclidean distance to
    the centre, so the exponent is ``phi * (1 - r**2)``.
    """
    alpha: float = 5.0
    phi: float = 0.5
    mach: float = 0.5
    theta: float = math.pi / 4
    x0: float = 0.0
    y0: float = 0.0
    gamma: float = GAMMA

    @property
    def speed(self) -> float:
        return math.sqrt(2.0)

    @property
    def uinf(self) -> float:
        return self.speed * math.cos(self.theta)

    @property
    def vinf(self) -> float:
        return self.speed * math.sin(self.theta)

    @property
    def pinf(self) -> float:
        return self.speed ** 2 / (self.gamma * self.mach ** 2)

    def state(self, X, Y, t: float = 0.0, box=(-5.0, 5.0, -5.0, 5.0)) -> np.ndarray:
        """Conserved state at time ``t``: the vortex advected with the free
        stream, centre taken at its nearest periodic image."""
        g = self.gamma
        lx, ly = box[1] - box[0], box[3] - box[2]
        xc = self.x0 + self.uinf * t
        yc = self.y0 + self.vinf * t
        dx = X - xc
        dy = Y - yc
        dx = dx - lx * np.round(dx / lx)
        dy = dy - ly * np.round(dy / ly)
        r2 = dx * dx + dy * dy
        ex = np.exp(self.phi * (1.0 - r2))
        du = -self.alpha / (2 * math.pi) * dy * ex
        dv = self.alpha / (2 * math.pi) * dx * ex
        dT = -self.alpha ** 2 * (g - 1.0) / (16 * self.phi * g * math.pi ** 2) * ex * ex
        Tinf = self.pinf  # rho_inf = 1, R = 1
        T = Tinf + dT
        rho = (T / Tinf) ** (1.0 / (g - 1.0))
        pr = rho * T
        return conserved(rho, self.uinf + du, self.vinf + dv, pr, g)


def density_wave_state(X, Y, t: float = 0.0, amp: float = 0.2, u: float = 1.0, v: float = 1.0,
                       pr: float = 1.0, box=(-5.0, 5.0, -5.0, 5.0), gamma: float = GAMMA):
    """Smooth density wave advected at constant (u, v, p): exact solution of
    the Euler equations is pure translation."""
    lx = box[1] - box[0]
    ly = box[3] - box[2]
    kx, ky = 2 * math.pi / lx, 2 * math.pi / ly
    rho = 1.0 + amp * np.sin(kx * (X - u * t) + ky * (Y - v * t))
    return conserved(rho, np.full_like(X, u), np.full_like(X, v), np.full_like(X, pr), gamma)


def smooth_random_state(X, Y, seed: int, amp: float = 0.05, modes: int = 3,
                        box=(-5.0, 5.0, -5.0, 5.0), base=(1.0, 0.7, -0.4, 2.0),
                        gamma: float = GAMMA) -> np.ndarray:
    """Free stream ``base = (rho, u, v, p)`` plus random periodic Fourier
    modes of relative amplitude ``amp`` in every primitive field."""
    rng = np.random.default_rng(seed)
    lx = box[1] - box[0]
    ly = box[3] - box[2]
    fields = []
    for b in base:
        f = np.full_like(X, b)
        for _ in range(modes):
            kx, ky = rng.integers(-3, 4, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1) * amp * max(abs(b), 1.0)
            f = f + a * np.sin(2 * math.pi * (kx * X / lx + ky * Y / ly) + ph)
        fields.append(f)
    rho, u, v, pr = fields
    return conserved(rho, u, v, pr, gamma)


def random_vector(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Standard-normal array of the given shape (fp64)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)


def uniform_mesh(n: int, box=(-5.0, 5.0, -5.0, 5.0), ny: int | None = None):
    ny = n if ny is None else ny
    return uniform_edges(n, box[0], box[1]), uniform_edges(ny, box[2], box[3])


def stretched_mesh(nx: int, ny: int, seed: int = 0, amp: float = 0.3,
                   box=(-5.0, 5.0, -5.0, 5.0)):
    """Tensor-product mesh with randomly jittered (non-uniform) edges."""
    rng = np.random.default_rng(seed)
    def jitter(n, lo, hi):
        e = np.linspace(lo, hi, n + 1)
        h = (hi - lo) / n
        e[1:-1] += rng.uniform(-amp, amp, n - 1) * h
        return e
    return jitter(nx, box[0], box[1]), jitter(ny, box[2], box[3])


@dataclass(frozen=True)
class Channel:
    """Plane channel between walls y = 0 and y = 1, periodic in x over
    [0, lx]: laminar Poiseuille profile u = 4 uc y (1 - y), uniform density
    and temperature (Mach ``mach`` on uc, gas constant 1), plus a seeded
    divergence-free perturbation from a stream function
    psi = y^2 (1-y)^2 sum_m a_m sin(kx_m x + phi_m) cos(ky_m y + theta_m)
    (u' = dpsi/dy, v' = -dpsi/dx vanish at the walls), scaled so that
    max |u'| = amp * uc over the sample points."""
    lx: float = 2.0
    uc: float = 1.0
    mach: float = 0.2
    reynolds: float = 1000.0     # rho uc lx / mu
    prandtl: float = 0.72
    gamma: float = GAMMA

    @property
    def temperature(self) -> float:
        return (self.uc / self.mach) ** 2 / self.gamma

    @property
    def mu(self) -> float:
        return self.uc * self.lx / self.reynolds

    @property
    def body_force(self) -> float:
        """Force per unit mass that balances the Poiseuille wall shear."""
        return 8.0 * self.mu * self.uc

    def state(self, X, Y, seed: int, amp: float = 1e-2, modes: int = 4) -> np.ndarray:
        rng = np.random.default_rng(seed)
        w = Y * Y * (1 - Y) ** 2
        dw = 2 * Y * (1 - Y) * (1 - 2 * Y)
        up = np.zeros_like(X)
        vp = np.zeros_like(X)
        for _ in range(modes):
            kx = 2 * math.pi * rng.integers(1, 4) / self.lx
            ky = math.pi * rng.integers(0, 3)
            a = rng.uniform(-1, 1)
            ph, th = rng.uniform(0, 2 * math.pi, 2)
            sx, cx = np.sin(kx * X + ph), np.cos(kx * X + ph)
            cy, sy = np.cos(ky * Y + th), np.sin(ky * Y + th)
            up += a * sx * (dw * cy - w * ky * sy)
            vp += -a * w * kx * cx * cy
        scale = amp * self.uc / max(np.max(np.abs(up)), 1e-300)
        u = 4 * self.uc * Y * (1 - Y) + scale * up
        v = scale * vp
        T = self.temperature
        return conserved(np.ones_like(X), u, v, T * np.ones_like(X), self.gamma)


@dataclass
class Instance:
    """One member of a batch of independent vortex problems."""
    n: int          # n x n uniform quads of [-5,5]^2
    p: int          # polynomial degree
    vortex: Vortex

    def mesh(self):
        return uniform_mesh(self.n)

    def state(self) -> np.ndarray:
        xe, ye = self.mesh()
        X, Y = point_coords(xe, ye, self.p)
        return self.vortex.state(X, Y)


BATCH_MESHES = (32, 48, 64, 96, 128)
BATCH_DEGREES = (2, 3, 4)


def batch_instances(count: int = 64, seed: int = 0, meshes=BATCH_MESHES, degrees=BATCH_DEGREES):
    """Independent vortex instances of uneven size and degree.

    One PCG64 stream (``seed``); per instance, in this order: centre
    (x0, y0) ~ U([-2.5, 2.5]^2), strength alpha ~ U[3, 6], flow angle
    theta ~ U[0, 2 pi), mesh n uniform over ``meshes``, degree p uniform
    over ``degrees``.  Mach 0.5 on the free-stream speed sqrt(2), phi = 1/2.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        x0, y0 = rng.uniform(-2.5, 2.5, 2)
        alpha = rng.uniform(3.0, 6.0)
        theta = rng.uniform(0.0, 2.0 * math.pi)
        n = int(meshes[rng.integers(len(meshes))])
        p = int(degrees[rng.integers(len(degrees))])
        out.append(Instance(n, p, Vortex(alpha=float(alpha), theta=float(theta), x0=float(x0), y0=float(y0))))
    return out


# ------------------------------------------------------------------ 3D ------
# State arrays of the 3D path have shape ``(Ne, 5, Np)`` with ``Np = (p+1)**3``;
# point ``i + n*j + n*n*k`` (i along x, j along y, k along z, n = p+1);
# element ``ix + Nx*(iy + Ny*iz)``; variables (rho, rho u, rho v, rho w, E).

def point_coords3d(x_edges, y_edges, z_edges, p: int):
    """Physical coordinates ``X, Y, Z`` of shape ``(Ne, Np)`` (3D layout)."""
    s = sample_nodes(p)
    n = p + 1
    nx, ny, nz = len(x_edges) - 1, len(y_edges) - 1, len(z_edges) - 1
    def place(edges):
        a, h = np.asarray(edges[:-1]), np.diff(edges)
        return a[:, None] + 0.5 * (s[None, :] + 1.0) * h[:, None]      # (n_el, n)
    px, py, pz = place(x_edges), place(y_edges), place(z_edges)
    shape = (nz, ny, nx, n, n, n)                                      # [iz, iy, ix, k, j, i]
    X = np.broadcast_to(px[None, None, :, None, None, :], shape)
    Y = np.broadcast_to(py[None, :, None, None, :, None], shape)
    Z = np.broadcast_to(pz[:, None, None, :, None, None], shape)
    ne = nx * ny * nz
    return tuple(np.ascontiguousarray(A.reshape(ne, n ** 3)) for A in (X, Y, Z))


def conserved3d(rho, u, v, w, pr, gamma: float = GAMMA) -> np.ndarray:
    """Stack primitive fields into conserved ``(Ne, 5, Np)``."""
    E = pr / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, E], axis=1))


def uniform_mesh3d(n: int, lo: float = -math.pi, hi: float = math.pi):
    e = uniform_edges(n, lo, hi)
    return e, e.copy(), e.copy()


def stretched_mesh3d(nx: int, ny: int, nz: int, seed: int = 0, amp: float = 0.3,
                     lo: float = -math.pi, hi: float = math.pi):
    """Tensor-product hexahedral mesh with randomly jittered edges."""
    rng = np.random.default_rng(seed)
    out = []
    for n in (nx, ny, nz):
        e = np.linspace(lo, hi, n + 1)
        e[1:-1] += rng.uniform(-amp, amp, n - 1) * (hi - lo) / n
        out.append(e)
    return tuple(out)


def smooth_random_state3d(X, Y, Z, seed: int, amp: float = 0.05, modes: int = 3,
                          lo: float = -math.pi, hi: float = math.pi,
                          base=(1.0, 0.7, -0.4, 0.3, 2.0), gamma: float = GAMMA) -> np.ndarray:
    """Free stream ``base = (rho, u, v, w, p)`` plus random periodic Fourier
    modes of relative amplitude ``amp`` in every primitive field."""
    rng = np.random.default_rng(seed)
    L = hi - lo
    fields = []
    for b in base:
        f = np.full_like(X, b)
        for _ in range(modes):
            k = rng.integers(-2, 3, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1) * amp * max(abs(b), 1.0)
            f = f + a * np.sin(2 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) / L + ph)
        fields.append(f)
    return conserved3d(*fields, gamma=gamma)


@dataclass(frozen=True)
class TaylorGreen:
    """Initial field of the Taylor-Green vortex (Sec. 5): on [-pi L, pi L]^3,
    u = V0 sin(x/L) cos(y/L) cos(z/L), v = -V0 cos(x/L) sin(y/L) cos(z/L),
    w = 0, p = p0 + rho0 V0^2/16 (cos(2x/L) + cos(2y/L)) (cos(2z/L) + 2),
    Ma = V0 / c0 = 0.1 with c0 the sound speed at (rho0, p0), Re = rho0 V0 L / mu
    = 1600, Pr = 0.71.  The paper does not give the initial density; the
    temperature is taken uniform, T0 = p0 / (rho0 R), so rho = rho0 p / p0."""
    rho0: float = 1.0
    v0: float = 1.0
    length: float = 1.0
    mach: float = 0.1
    reynolds: float = 1600.0
    prandtl: float = 0.71
    gamma: float = GAMMA

    @property
    def p0(self) -> float:
        return self.rho0 * self.v0 ** 2 / (self.gamma * self.mach ** 2)

    @property
    def mu(self) -> float:
        return self.rho0 * self.v0 * self.length / self.reynolds

    @property
    def t_c(self) -> float:
        return self.length / self.v0

    def state(self, X, Y, Z) -> np.ndarray:
        L, V0 = self.length, self.v0
        u = V0 * np.sin(X / L) * np.cos(Y / L) * np.cos(Z / L)
        v = -V0 * np.cos(X / L) * np.sin(Y / L) * np.cos(Z / L)
        w = np.zeros_like(X)
        pr = self.p0 + self.rho0 * V0 ** 2 / 16.0 * (np.cos(2 * X / L) + np.cos(2 * Y / L)) * (np.cos(2 * Z / L) + 2.0)
        rho = self.rho0 * pr / self.p0
        return conserved3d(rho, u, v, w, pr, self.gamma)
