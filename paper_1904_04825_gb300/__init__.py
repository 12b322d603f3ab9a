"""Python binding of libfrjfnk (GB300 Jacobian-free Newton-Krylov for 2D FR/CPR).

Argument marshalling only: every step of the computation runs in the CUDA
library built from ``csrc/`` (see ``include/frjfnk.h`` for the C ABI).  The
functions keep the C names and take PyTorch CUDA float64 tensors laid out as
``(Ne, 4, Np)`` (any contiguous shape with ``ndof`` elements); PyTorch only
provides device memory and the current stream.

Importing this package loads ``lib/libfrjfnk.so`` and fails loudly when it
has not been built (``python -c "import __graft_entry__ as g; g.build()"``):
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libfrjfnk.so")

FR_OK = 0
FR_ERR_INVALID_ARG = 1
FR_ERR_CUDA = 2
FR_ERR_NONFINITE = 3
FR_ERR_NOT_CONVERGED = 4
FR_ERR_PTC_STALLED = 5
FR_ERR_TIMEOUT = 6
FR_ERR_UNSUPPORTED = 7

# kernel families of the measurement hooks
KF_NAMES = ["residual", "jv", "factor", "apply", "dots", "update", "solupdate", "other", "invert"]
FR_KF_COUNT = len(KF_NAMES)
ERROR_NAMES = {0: "FR_OK", 1: "FR_ERR_INVALID_ARG", 2: "FR_ERR_CUDA", 3: "FR_ERR_NONFINITE",
               4: "FR_ERR_NOT_CONVERGED", 5: "FR_ERR_PTC_STALLED", 6: "FR_ERR_TIMEOUT",
               7: "FR_ERR_UNSUPPORTED"}


class FrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class fr_mesh_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x_edges", ctypes.POINTER(ctypes.c_double)),
                ("y_edges", ctypes.POINTER(ctypes.c_double)),
                ("wall_y", ctypes.c_int)]


class fr_mesh3d_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x_edges", ctypes.POINTER(ctypes.c_double)),
                ("y_edges", ctypes.POINTER(ctypes.c_double)),
                ("z_edges", ctypes.POINTER(ctypes.c_double))]


class fr_opts(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("m_max", ctypes.c_int),
                ("eps_rel", ctypes.c_double), ("eps_fixed", ctypes.c_double),
                ("block_eps_rel", ctypes.c_double), ("precond", ctypes.c_int),
                ("gmres_m", ctypes.c_int), ("gmres_max_restarts", ctypes.c_int),
                ("tol_lin", ctypes.c_double), ("reorth_eta", ctypes.c_double),
                ("mu", ctypes.c_double), ("prandtl", ctypes.c_double),
                ("body_force_x", ctypes.c_double), ("wall_temperature", ctypes.c_double),
                ("block_precision", ctypes.c_int), ("precond_refresh", ctypes.c_int),
                ("guess", ctypes.c_int), ("jv_precision", ctypes.c_int), ("riemann", ctypes.c_int),
                ("block_columns", ctypes.c_int)]


class fr_ptc_opts(ctypes.Structure):
    _fields_ = [("tol_nl", ctypes.c_double), ("tol_lin", ctypes.c_double),
                ("dtau_init", ctypes.c_double), ("dtau_max", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("max_rejections", ctypes.c_int),
                ("reject_above", ctypes.c_double)]


class fr_vortex(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("phi", ctypes.c_double), ("mach", ctypes.c_double),
                ("rho_inf", ctypes.c_double), ("u_inf", ctypes.c_double), ("v_inf", ctypes.c_double),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double)]


class fr_gmres_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("relres", ctypes.c_double)]


class fr_step_stats(ctypes.Structure):
    _fields_ = [("gmres_iters", ctypes.c_int), ("gmres_calls", ctypes.c_int),
                ("ptc_iters", ctypes.c_int), ("rejections", ctypes.c_int),
                ("residual_evals", ctypes.c_int), ("converged", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I, V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    sig = {
        "fr_default_opts": (None, [ctypes.POINTER(fr_opts)]),
        "fr_default_ptc_opts": (None, [ctypes.POINTER(fr_ptc_opts)]),
        "fr_ctx_create": (I, [ctypes.POINTER(fr_mesh_desc), I, ctypes.POINTER(fr_opts),
                              ctypes.POINTER(ctypes.c_void_p)]),
        "fr_ctx_create_3d": (I, [ctypes.POINTER(fr_mesh3d_desc), I, ctypes.POINTER(fr_opts),
                                 ctypes.POINTER(ctypes.c_void_p)]),
        "fr_dissipation_rate": (I, [P, P, D, ctypes.POINTER(ctypes.c_double), V]),
        "fr_default_vortex": (None, [ctypes.POINTER(fr_vortex)]),
        "fr_vortex_error": (I, [P, P, ctypes.POINTER(fr_vortex), D, ctypes.POINTER(ctypes.c_double), V]),
        "fr_ctx_destroy": (I, [P]),
        "fr_last_error": (ctypes.c_char_p, [P]),
        "fr_ndof": (ctypes.c_longlong, [P]),
        "fr_residual": (I, [P, P, P, V]),
        "fr_jv": (I, [P, P, P, P, D, P, V]),
        "ejacobi_factor": (I, [P, P, P, D, V]),
        "ejacobi_apply": (I, [P, P, P, V]),
        "gmres_solve": (I, [P, P, P, D, P, P, I, D, I, ctypes.POINTER(fr_gmres_info), V]),
        "step_row": (I, [P, I, D, P, ctypes.POINTER(fr_step_stats), V]),
        "step_esdirk": (I, [P, I, D, P, ctypes.POINTER(fr_ptc_opts),
                            ctypes.POINTER(fr_step_stats), V]),
        "step_bdf2": (I, [P, D, P, P, I, ctypes.POINTER(fr_ptc_opts),
                          ctypes.POINTER(fr_step_stats), V]),
        "step_ssprk3": (I, [P, D, P, ctypes.POINTER(fr_step_stats), V]),
        "fr_kernel_launches": (ctypes.c_longlong, []),
        "fr_set_wait_test": (I, [P, ctypes.c_uint, I]),
        "fr_set_block_chunk": (I, [P, ctypes.c_longlong]),
        "fr_jv_noalloc": (I, [ctypes.POINTER(fr_mesh_desc), I, ctypes.POINTER(fr_opts), P, P, P, D, P, V]),
        "fr_mlp_create": (I, [I, I, I, I, ctypes.POINTER(ctypes.c_void_p)]),
        "fr_mlp_destroy": (I, [P]),
        "fr_mlp_last_error": (ctypes.c_char_p, [P]),
        "fr_mlp_num_params": (ctypes.c_longlong, [P]),
        "fr_mlp_set_params": (I, [P, P, V]),
        "fr_mlp_get_params": (I, [P, P, V]),
        "fr_mlp_get_grads": (I, [P, P, V]),
        "fr_mlp_forward": (I, [P, P, I, P, I, V]),
        "fr_mlp_backward": (I, [P, P, P, I, ctypes.POINTER(ctypes.c_double), V]),
        "fr_mlp_adam": (I, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, V]),
        "fr_attach_guess_model": (I, [P, P]),
        "fr_set_stage_capture": (I, [P, P, P, ctypes.c_longlong, I]),
        "fr_stage_capture_count": (ctypes.c_longlong, [P]),
        "fr_stage_features": (I, [P, P, P, P, P, V]),
        "fr_reset_history": (I, [P]),
        "fr_guess_stats": (I, [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "fr_batch_create": (I, [I, ctypes.POINTER(fr_mesh_desc), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(fr_opts), ctypes.POINTER(ctypes.c_void_p)]),
        "fr_batch_destroy": (I, [P]),
        "fr_batch_last_error": (ctypes.c_char_p, [P]),
        "fr_batch_member": (P, [P, I]),
        "fr_batch_set_batched": (I, [P, I]),
        "fr_batch_cycle_kernels": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
        "fr_batch_step_row": (I, [P, I, D, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(fr_step_stats), V]),
        "fr_batch_step_esdirk": (I, [P, I, D, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(fr_ptc_opts), I,
                                     ctypes.POINTER(fr_step_stats), V]),
        "fr_batch_step_bdf2": (I, [P, D, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), I,
                                   ctypes.POINTER(fr_ptc_opts), I, ctypes.POINTER(fr_step_stats), V]),
        "fr_set_launch_config": (I, [P, I, I]),
        "fr_get_launch_config": (I, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "fr_autotune": (I, [P, P, D, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), V]),
        "fr_profile_begin": (I, [P, ctypes.c_uint]),
        "fr_profile_end": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def default_opts(**kw) -> fr_opts:
    o = fr_opts()
    lib.fr_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def default_ptc_opts(**kw) -> fr_ptc_opts:
    o = fr_ptc_opts()
    lib.fr_default_ptc_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _sized(t, n: int, name: str = "tensor"):
    """_ptr after checking that t holds exactly n elements: the library takes
    the length from the mesh and trusts the pointer, so a shorter tensor would
    be read or written past its end."""
    if t is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return _ptr(t)


def _vec(ctx, t, name: str = "vector"):
    """Pointer to a state-shaped float64 CUDA tensor of exactly ctx.ndof elements."""
    return _sized(t, ctx.ndof, name)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """Owns an ``fr_ctx`` (mesh, degree, options, device workspace)."""

    def __init__(self, x_edges, y_edges, p: int, opts: fr_opts | None = None, wall_y: bool = False):
        xe = np.ascontiguousarray(x_edges, dtype=np.float64)
        ye = np.ascontiguousarray(y_edges, dtype=np.float64)
        desc = fr_mesh_desc(len(xe) - 1, len(ye) - 1,
                            xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            ye.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(bool(wall_y)))
        self.opts = opts if opts is not None else default_opts()
        h = ctypes.c_void_p()
        rc = lib.fr_ctx_create(ctypes.byref(desc), p, ctypes.byref(self.opts), ctypes.byref(h))
        if rc != FR_OK:
            raise FrError(rc, "fr_ctx_create failed")
        self.handle = h
        self.p = p
        self.nx, self.ny = len(xe) - 1, len(ye) - 1
        self.ne = self.nx * self.ny
        self.np = (p + 1) ** 2
        self.ndof = int(lib.fr_ndof(h))
        self.shape = (self.ne, 4, self.np)

    @classmethod
    def _view(cls, handle, nx, ny, p, opts):
        """A non-owning Context over a context that a Batch owns."""
        c = cls.__new__(cls)
        c.handle, c.p, c.nx, c.ny, c.opts = handle, p, nx, ny, opts
        c.ne, c.np = nx * ny, (p + 1) ** 2
        c.ndof = int(lib.fr_ndof(handle))
        c.shape = (c.ne, 4, c.np)
        c._owner = False
        return c

    def close(self):
        if getattr(self, "handle", None) and getattr(self, "_owner", True):
            lib.fr_ctx_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc, allow=()):
        if rc != FR_OK and rc not in allow:
            raise FrError(rc, lib.fr_last_error(self.handle).decode())
        return rc

    def empty(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")


class Context3D(Context):
    """Owns a 3D ``fr_ctx``: periodic hexahedra, state ``(Ne, 5, (p+1)**3)``."""

    def __init__(self, x_edges, y_edges, z_edges, p: int, opts: fr_opts | None = None):
        es = [np.ascontiguousarray(e, dtype=np.float64) for e in (x_edges, y_edges, z_edges)]
        dp = [e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for e in es]
        desc = fr_mesh3d_desc(len(es[0]) - 1, len(es[1]) - 1, len(es[2]) - 1, *dp)
        self.opts = opts if opts is not None else default_opts()
        h = ctypes.c_void_p()
        rc = lib.fr_ctx_create_3d(ctypes.byref(desc), p, ctypes.byref(self.opts), ctypes.byref(h))
        if rc != FR_OK:
            raise FrError(rc, "fr_ctx_create_3d failed")
        self.handle = h
        self.p = p
        self.nx, self.ny, self.nz = (len(e) - 1 for e in es)
        self.ne = self.nx * self.ny * self.nz
        self.np = (p + 1) ** 3
        self.ndof = int(lib.fr_ndof(h))
        self.shape = (self.ne, 5, self.np)


def fr_dissipation_rate(ctx: Context3D, U, rho0: float = 1.0, stream=None):
    """(eps1, eps3, kinetic energy) of the Taylor-Green study for the 3D state U."""
    out = (ctypes.c_double * 3)()
    ctx.check(lib.fr_dissipation_rate(ctx.handle, _vec(ctx, U, "U"), rho0, out, _stream(stream)))
    return out[0], out[1], out[2]


def default_vortex(**kw) -> fr_vortex:
    v = fr_vortex()
    lib.fr_default_vortex(ctypes.byref(v))
    for k, val in kw.items():
        setattr(v, k, val)
    return v


def fr_vortex_error(ctx: Context, U, t: float, vortex: fr_vortex | None = None, stream=None):
    """E(rho), E(u), E(v), E(p) of the state U against the exact isentropic vortex at time t."""
    v = vortex if vortex is not None else default_vortex()
    out = (ctypes.c_double * 4)()
    ctx.check(lib.fr_vortex_error(ctx.handle, _vec(ctx, U), ctypes.byref(v), float(t), out, _stream(stream)))
    return {"rho": out[0], "u": out[1], "v": out[2], "p": out[3]}


def fr_residual(ctx: Context, U, R, stream=None):
    return ctx.check(lib.fr_residual(ctx.handle, _vec(ctx, U, "U"), _vec(ctx, R, "R"), _stream(stream)))


def fr_jv(ctx: Context, U, R0, z, shift, y, stream=None):
    return ctx.check(lib.fr_jv(ctx.handle, _vec(ctx, U, "U"), _vec(ctx, R0, "R0"), _vec(ctx, z, "z"), float(shift),
                               _vec(ctx, y, "y"),
                               _stream(stream)))


def ejacobi_factor(ctx: Context, U, R0, shift, stream=None):
    return ctx.check(lib.ejacobi_factor(ctx.handle, _vec(ctx, U, "U"), _vec(ctx, R0, "R0"), float(shift), _stream(stream)))


def ejacobi_apply(ctx: Context, r, z, stream=None):
    return ctx.check(lib.ejacobi_apply(ctx.handle, _vec(ctx, r, "r"), _vec(ctx, z, "z"), _stream(stream)))


@dataclass
class GmresInfo:
    iters: int
    restarts: int
    converged: bool
    relres: float
    code: int


def gmres_solve(ctx: Context, U, R0, shift, b, x, m=30, rtol=1e-8, max_restarts=20, stream=None,
                allow_not_converged=True) -> GmresInfo:
    info = fr_gmres_info()
    rc = lib.gmres_solve(ctx.handle, _vec(ctx, U, "U"), _vec(ctx, R0, "R0"), float(shift), _vec(ctx, b, "b"),
                         _vec(ctx, x, "x"), int(m),
                         float(rtol), int(max_restarts), ctypes.byref(info), _stream(stream))
    ctx.check(rc, allow=(FR_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return GmresInfo(info.iters, info.restarts, bool(info.converged), info.relres, rc)


@dataclass
class StepStats:
    gmres_iters: int
    gmres_calls: int
    ptc_iters: int
    rejections: int
    residual_evals: int
    converged: bool
    code: int


def _stats(st, rc):
    return StepStats(st.gmres_iters, st.gmres_calls, st.ptc_iters, st.rejections,
                     st.residual_evals, bool(st.converged), rc)


def step_row(ctx: Context, scheme: int, dt: float, U, stream=None, allow=(FR_ERR_NOT_CONVERGED,)):
    st = fr_step_stats()
    rc = lib.step_row(ctx.handle, int(scheme), float(dt), _vec(ctx, U, "U"), ctypes.byref(st), _stream(stream))
    ctx.check(rc, allow=allow)
    return _stats(st, rc)


def step_esdirk(ctx: Context, scheme: int, dt: float, U, ptc: fr_ptc_opts | None = None, stream=None,
                allow=(FR_ERR_NOT_CONVERGED,)):
    st = fr_step_stats()
    rc = lib.step_esdirk(ctx.handle, int(scheme), float(dt), _vec(ctx, U, "U"),
                         ctypes.byref(ptc) if ptc is not None else None, ctypes.byref(st),
                         _stream(stream))
    ctx.check(rc, allow=allow)
    return _stats(st, rc)


def step_bdf2(ctx: Context, dt: float, U, U_prev, first_step: bool, ptc: fr_ptc_opts | None = None,
              stream=None, allow=(FR_ERR_NOT_CONVERGED,)):
    st = fr_step_stats()
    rc = lib.step_bdf2(ctx.handle, float(dt), _vec(ctx, U, "U"), _vec(ctx, U_prev, "U_prev"), int(bool(first_step)),
                       ctypes.byref(ptc) if ptc is not None else None, ctypes.byref(st),
                       _stream(stream))
    ctx.check(rc, allow=allow)
    return _stats(st, rc)


def step_ssprk3(ctx: Context, dt: float, U, stream=None):
    st = fr_step_stats()
    rc = lib.step_ssprk3(ctx.handle, float(dt), _vec(ctx, U, "U"), ctypes.byref(st), _stream(stream))
    ctx.check(rc)
    return _stats(st, rc)


def fr_set_wait_test(ctx: Context, polls: int = 0, skip_first_copy: bool = False):
    """Test hook for the element-Jacobi apply's bounded waits (see the C header)."""
    return ctx.check(lib.fr_set_wait_test(ctx.handle, int(polls), int(bool(skip_first_copy))))


def fr_set_block_chunk(ctx: Context, n: int):
    """Elements whose FD element blocks are staged and inverted at a time (see the C header)."""
    return ctx.check(lib.fr_set_block_chunk(ctx.handle, int(n)))


def fr_kernel_launches() -> int:
    """Kernels this library has launched in this process."""
    return int(lib.fr_kernel_launches())


def fr_profile_begin(ctx: Context, families=None):
    """Time every launch of the given kernel families (names of KF_NAMES)."""
    names = KF_NAMES if families is None else families
    mask = 0
    for n in names:
        mask |= 1 << KF_NAMES.index(n)
    return ctx.check(lib.fr_profile_begin(ctx.handle, mask))


def fr_profile_end(ctx: Context):
    """{family: dict(ms, launches, bytes, flops)} for the timed families:
    summed kernel time, launches that did work, algorithmic bytes and flops."""
    ms = (ctypes.c_double * FR_KF_COUNT)()
    n = (ctypes.c_longlong * FR_KF_COUNT)()
    by = (ctypes.c_double * FR_KF_COUNT)()
    fl = (ctypes.c_double * FR_KF_COUNT)()
    ctx.check(lib.fr_profile_end(ctx.handle, ms, n, by, fl))
    return {KF_NAMES[i]: {"ms": ms[i], "launches": n[i], "bytes": by[i], "flops": fl[i]}
            for i in range(FR_KF_COUNT) if n[i] > 0 or ms[i] > 0}


def fr_jv_noalloc(x_edges, y_edges, p: int, U, R0, z, shift, y, opts: fr_opts | None = None, stream=None):
    """fr_jv without a context and without device allocation (see the C
    header: fixed static working memory, meshes up to 4096 x 4096, calls must
    not overlap on the GPU)."""
    xe = np.ascontiguousarray(x_edges, dtype=np.float64)
    ye = np.ascontiguousarray(y_edges, dtype=np.float64)
    desc = fr_mesh_desc(len(xe) - 1, len(ye) - 1,
                        xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        ye.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    n = (len(xe) - 1) * (len(ye) - 1) * 4 * (int(p) + 1) ** 2
    rc = lib.fr_jv_noalloc(ctypes.byref(desc), int(p), ctypes.byref(opts) if opts is not None else None,
                           _sized(U, n, "U"), _sized(R0, n, "R0"), _sized(z, n, "z"), float(shift),
                           _sized(y, n, "y"), _stream(stream))
    if rc != FR_OK:
        raise FrError(rc, lib.fr_last_error(None).decode())
    return rc


def _fsized(t, n: int, name: str = "tensor"):
    """_fptr after checking that t holds exactly n elements."""
    if t is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return _fptr(t)


def _fptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class MLP:
    """Per-element MLP of the learned initial guess (see the C header)."""

    def __init__(self, n_in: int, n_hidden: int, n_out: int, max_batch: int):
        h = ctypes.c_void_p()
        rc = lib.fr_mlp_create(n_in, n_hidden, n_out, max_batch, ctypes.byref(h))
        if rc != FR_OK:
            raise FrError(rc, "fr_mlp_create failed")
        self.handle = h
        self.sizes = (n_in, n_hidden, n_hidden, n_out)
        self.nparam = int(lib.fr_mlp_num_params(h))

    def close(self):
        if getattr(self, "handle", None):
            lib.fr_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc != FR_OK:
            raise FrError(rc, lib.fr_mlp_last_error(self.handle).decode())
        return rc

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparam
        return self.check(lib.fr_mlp_set_params(self.handle, a.ctypes.data_as(ctypes.c_void_p), _stream(None)))

    def get_params(self):
        a = np.empty(self.nparam, dtype=np.float32)
        self.check(lib.fr_mlp_get_params(self.handle, a.ctypes.data_as(ctypes.c_void_p), _stream(None)))
        return a

    def get_grads(self):
        a = np.empty(self.nparam, dtype=np.float32)
        self.check(lib.fr_mlp_get_grads(self.handle, a.ctypes.data_as(ctypes.c_void_p), _stream(None)))
        return a

    def forward(self, X, Y, bf16=False):
        M = int(X.shape[0])
        return self.check(lib.fr_mlp_forward(self.handle, _fsized(X, M * self.sizes[0], "X"), M,
                                             _fsized(Y, M * self.sizes[3], "Y"), int(bool(bf16)), _stream(None)))

    def backward(self, X, T):
        loss = ctypes.c_double()
        M = int(X.shape[0])
        self.check(lib.fr_mlp_backward(self.handle, _fsized(X, M * self.sizes[0], "X"),
                                       _fsized(T, M * self.sizes[3], "T"), M, ctypes.byref(loss), _stream(None)))
        return loss.value

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        return self.check(lib.fr_mlp_adam(self.handle, lr, beta1, beta2, eps, _stream(None)))


def flat_params(params):
    """Oracle (W, b) list -> the flat [W1 b1 W2 b2 W3 b3] layout."""
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params])


def unflat_params(flat, sizes):
    out, o = [], 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        W = flat[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = flat[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def fr_attach_guess_model(ctx: Context, model):
    return ctx.check(lib.fr_attach_guess_model(ctx.handle, model.handle if model is not None else None))


def fr_set_stage_capture(ctx: Context, X, T, max_samples, elem_stride):
    nb = 4 * ctx.np
    if X is not None and X.numel() < int(max_samples) * 3 * nb:
        raise ValueError(f"X holds {X.numel()} floats, fewer than max_samples * 3 nb = {int(max_samples) * 3 * nb}")
    if T is not None and T.numel() < int(max_samples) * nb:
        raise ValueError(f"T holds {T.numel()} floats, fewer than max_samples * nb = {int(max_samples) * nb}")
    return ctx.check(lib.fr_set_stage_capture(ctx.handle, _fptr(X) if X is not None else None,
                                              _fptr(T) if T is not None else None, int(max_samples),
                                              int(elem_stride)))


def fr_stage_capture_count(ctx: Context) -> int:
    return int(lib.fr_stage_capture_count(ctx.handle))


def fr_stage_features(ctx: Context, b, bl, yl, X, stream=None):
    return ctx.check(lib.fr_stage_features(ctx.handle, _vec(ctx, b, "b"), _vec(ctx, bl, "bl"), _vec(ctx, yl, "yl"),
                                              _fsized(X, ctx.ne * 12 * ctx.np, "X"), _stream(stream)))


def fr_reset_history(ctx: Context):
    return ctx.check(lib.fr_reset_history(ctx.handle))


def fr_guess_stats(ctx: Context):
    t, u = ctx_ll(), ctx_ll()
    ctx.check(lib.fr_guess_stats(ctx.handle, ctypes.byref(t), ctypes.byref(u)))
    return int(t.value), int(u.value)


def ctx_ll():
    return ctypes.c_longlong()


def set_launch_config(ctx: Context, vec_blocks: int, tile_variant: int):
    ctx.check(lib.fr_set_launch_config(ctx.handle, int(vec_blocks), int(tile_variant)))


def get_launch_config(ctx: Context):
    vb, tv = ctypes.c_int(), ctypes.c_int()
    ctx.check(lib.fr_get_launch_config(ctx.handle, ctypes.byref(vb), ctypes.byref(tv)))
    return int(vb.value), int(tv.value)


def autotune(ctx: Context, U, shift: float, reps: int = 2, stream=None):
    """Pick the fastest launch configuration for GMRES cycles at U; returns
    (vec_blocks, tile_variant, ms per cycle chosen, ms per cycle on entry)."""
    best, dflt = ctypes.c_double(), ctypes.c_double()
    ctx.check(lib.fr_autotune(ctx.handle, _vec(ctx, U, "U"), float(shift), int(reps), ctypes.byref(best),
                              ctypes.byref(dflt), _stream(stream)))
    vb, tv = get_launch_config(ctx)
    return vb, tv, best.value, dflt.value


class Batch:
    """Independent instances (own mesh and degree, shared options) stepped
    together; the stage GMRES cycles of all of them run as one CUDA graph."""

    def __init__(self, meshes, degrees, opts: fr_opts | None = None):
        if len(meshes) != len(degrees) or not meshes:
            raise ValueError("one degree per mesh, at least one instance")
        self.opts = opts if opts is not None else default_opts()
        self._edges = []
        descs = (fr_mesh_desc * len(meshes))()
        for k, (xe, ye) in enumerate(meshes):
            xe = np.ascontiguousarray(xe, dtype=np.float64)
            ye = np.ascontiguousarray(ye, dtype=np.float64)
            self._edges.append((xe, ye))
            descs[k] = fr_mesh_desc(len(xe) - 1, len(ye) - 1,
                                    xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    ye.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
        degs = (ctypes.c_int * len(degrees))(*[int(d) for d in degrees])
        h = ctypes.c_void_p()
        rc = lib.fr_batch_create(len(meshes), descs, degs, ctypes.byref(self.opts), ctypes.byref(h))
        if rc != FR_OK:
            raise FrError(rc, "fr_batch_create failed")
        self.handle = h
        self.members = [Context._view(lib.fr_batch_member(h, k), len(xe) - 1, len(ye) - 1, int(d), self.opts)
                        for k, ((xe, ye), d) in enumerate(zip(self._edges, degrees))]

    def __len__(self):
        return len(self.members)

    def close(self):
        if getattr(self, "handle", None):
            for m in self.members:
                m.handle = None
            lib.fr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _states(self, Us):
        if len(Us) != len(self.members):
            raise ValueError("one state per instance")
        for U, m in zip(Us, self.members):
            if U.numel() != m.ndof:
                raise ValueError("state shape does not match its instance")
        return (ctypes.c_void_p * len(Us))(*[_ptr(U).value for U in Us])

    def _finish(self, rc, st, allow):
        if rc != FR_OK and rc not in allow:
            raise FrError(rc, lib.fr_batch_last_error(self.handle).decode())
        return [_stats(st[k], rc) for k in range(len(self.members))]

    def set_batched(self, on: bool):
        """Batched Arnoldi launches over all instances (True, the default) or
        per-instance cycle kernels (False)."""
        rc = lib.fr_batch_set_batched(self.handle, int(bool(on)))
        if rc != FR_OK:
            raise FrError(rc, lib.fr_batch_last_error(self.handle).decode())

    def cycle_kernels(self) -> int:
        """Kernel nodes of the largest captured GMRES-cycle graph."""
        n = ctypes.c_longlong()
        lib.fr_batch_cycle_kernels(self.handle, ctypes.byref(n))
        return int(n.value)

    def step_row(self, scheme: int, dt: float, Us, stream=None, allow=(FR_ERR_NOT_CONVERGED,)):
        ptrs = self._states(Us)
        st = (fr_step_stats * len(Us))()
        rc = lib.fr_batch_step_row(self.handle, int(scheme), float(dt), ptrs, st, _stream(stream))
        return self._finish(rc, st, allow)

    def step_esdirk(self, scheme: int, dt: float, Us, ptc: fr_ptc_opts | None = None, threads: int = 0,
                    stream=None, allow=(FR_ERR_NOT_CONVERGED,)):
        ptrs = self._states(Us)
        st = (fr_step_stats * len(Us))()
        rc = lib.fr_batch_step_esdirk(self.handle, int(scheme), float(dt), ptrs,
                                      ctypes.byref(ptc) if ptc is not None else None, int(threads), st,
                                      _stream(stream))
        return self._finish(rc, st, allow)

    def step_bdf2(self, dt: float, Us, Uprevs, first_step: bool, ptc: fr_ptc_opts | None = None,
                  threads: int = 0, stream=None, allow=(FR_ERR_NOT_CONVERGED,)):
        ptrs = self._states(Us)
        prev = self._states(Uprevs)
        st = (fr_step_stats * len(Us))()
        rc = lib.fr_batch_step_bdf2(self.handle, float(dt), ptrs, prev, int(bool(first_step)),
                                    ctypes.byref(ptc) if ptc is not None else None, int(threads), st,
                                    _stream(stream))
        return self._finish(rc, st, allow)
