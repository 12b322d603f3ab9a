"""The vortex error kernel (exact solution of Eq. VP_Solution and the error
norm of Sec. 5.1) through the C ABI against the oracle's restatement.

Tolerance: each E(s)^2 is a sum of positive terms w |J| d^2; the two sides
evaluate the exact state with different exp/pow implementations (relative
differences of a few ulp) and sum in different orders, so E agrees to
~1e-13 relative wherever d is not itself at the rounding level.  1e-11 is
used; on an exact state (d at the rounding level) the check is absolute.
"""
import math

import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh
from oracle.vortex import VortexCase, exact_state, vortex_errors

pytestmark = pytest.mark.gpu

TOL_E = 1e-11


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1904_04825_gb300 as mod
    return mod


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _perturbed(U, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    V = U.copy()
    V[:, 0] *= 1.0 + amp * rng.standard_normal(V[:, 0].shape)
    V[:, 1:3] += amp * rng.standard_normal(V[:, 1:3].shape)
    V[:, 3] *= 1.0 + amp * rng.standard_normal(V[:, 3].shape)
    return V


@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_vortex_error_matches_oracle_jittered_mesh(fr, p):
    box = (-10.0, 10.0, -10.0, 10.0)
    xe, ye = S.stretched_mesh(11, 9, seed=p, box=box)
    m = Mesh(xe, ye)
    case = VortexCase(box=box)
    t = 0.7
    U = _perturbed(exact_state(case, m, p, t), seed=10 + p)
    ctx = fr.Context(xe, ye, p, fr.default_opts(precond=0))
    got = fr.fr_vortex_error(ctx, _t(U), t)
    want = vortex_errors(U, case, m, p, t)
    for k in ("rho", "u", "v", "p"):
        assert abs(got[k] - want[k]) <= TOL_E * want[k], (k, got[k], want[k])
    ctx.close()


def test_vortex_error_other_parameters_and_periodic_image(fr):
    """Another strength, width, Mach number, free stream and centre on the
    [-5,5]^2 box, at a time when the centre has left the box (nearest image)."""
    box = (-5.0, 5.0, -5.0, 5.0)
    xe, ye = S.stretched_mesh(12, 10, seed=5, box=box)
    m = Mesh(xe, ye)
    th = 2.2
    case = VortexCase(alpha=3.7, phi=0.8, mach=0.4, u_inf=math.sqrt(2) * math.cos(th),
                      v_inf=math.sqrt(2) * math.sin(th), x0=1.3, y0=-0.4, box=box)
    t = 6.3
    U = _perturbed(exact_state(case, m, 3, t), seed=3)
    ctx = fr.Context(xe, ye, 3, fr.default_opts(precond=0))
    vx = fr.default_vortex(alpha=case.alpha, phi=case.phi, mach=case.mach, u_inf=case.u_inf,
                           v_inf=case.v_inf, x0=case.x0, y0=case.y0)
    got = fr.fr_vortex_error(ctx, _t(U), t, vx)
    want = vortex_errors(U, case, m, 3, t)
    for k in ("rho", "u", "v", "p"):
        assert abs(got[k] - want[k]) <= TOL_E * want[k], (k, got[k], want[k])
    # the exact state itself: zero up to the rounding of the two exact evaluations
    got0 = fr.fr_vortex_error(ctx, _t(exact_state(case, m, 3, t)), t, vx)
    assert max(got0.values()) < 1e-13
    ctx.close()


def test_vortex_error_full_size_160_p3(fr):
    """The 160 x 160 p = 3 vortex of the benchmark after a seeded perturbation."""
    box = (-5.0, 5.0, -5.0, 5.0)
    xe, ye = S.uniform_mesh(160)
    m = Mesh(xe, ye)
    case = VortexCase(box=box)
    U = _perturbed(S.Vortex().state(*S.point_coords(xe, ye, 3), t=2.5), seed=1, amp=1e-5)
    ctx = fr.Context(xe, ye, 3, fr.default_opts(precond=0))
    got = fr.fr_vortex_error(ctx, _t(U), 2.5)
    want = vortex_errors(U, case, m, 3, 2.5)
    for k in ("rho", "u", "v", "p"):
        assert abs(got[k] - want[k]) <= TOL_E * want[k], (k, got[k], want[k])
    ctx.close()


def test_vortex_error_rejects_viscous_context(fr):
    xe, ye = S.uniform_mesh(4)
    ctx = fr.Context(xe, ye, 2, fr.default_opts(mu=1e-3, precond=0))
    import torch
    U = torch.zeros(ctx.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(fr.FrError) as e:
        fr.fr_vortex_error(ctx, U, 0.0)
    assert e.value.code == fr.FR_ERR_UNSUPPORTED
    ctx.close()
