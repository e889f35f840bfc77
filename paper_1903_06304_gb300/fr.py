"""Thin ctypes binding of the C-ABI library ``libfr.so`` (declared in ``include/fr.h``).

Argument marshalling only: every step of the path runs in the library's CUDA kernels.
Device arrays are torch CUDA tensors (float64, contiguous, layout [4][Ne][n][n] for
solution vectors); the stream is torch's current CUDA stream unless one is given.
The module raises if the library is missing or fails to load: there is no fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfr.so")

FR_OK = 0
ERRORS = {-1: "FR_ERR_ARG", -2: "FR_ERR_CUDA", -3: "FR_ERR_NONFINITE",
          -4: "FR_ERR_NOT_CONVERGED", -5: "FR_ERR_TIMEOUT"}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
MAX_NEWTON = 64
BDF2 = (1.5, -2.0, 0.5)
BDF1 = (1.0, -1.0, 0.0)


class FrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int),
                ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double),
                ("mach", ctypes.c_double), ("re", ctypes.c_double),
                ("kappa", ctypes.c_double), ("eps_floor", ctypes.c_double),
                ("prec_dtype", ctypes.c_int),
                ("restart", ctypes.c_int), ("maxit_lin", ctypes.c_int),
                ("maxit_newton", ctypes.c_int), ("lag", ctypes.c_int),
                ("tol_res", ctypes.c_double), ("tol_pseudo", ctypes.c_double),
                ("dtau0", ctypes.c_double), ("dtau_min", ctypes.c_double),
                ("dtau_max", ctypes.c_double), ("r_ser", ctypes.c_double),
                ("dtau_unsteady", ctypes.c_double), ("gmres_side", ctypes.c_int),
                ("ser_unsteady", ctypes.c_int), ("dtau0_unsteady", ctypes.c_double),
                ("line_search", ctypes.c_int), ("jvp_mode", ctypes.c_int),
                ("graphs", ctypes.c_int), ("apply_accum", ctypes.c_int), ("tiles", ctypes.c_int),
                ("block_mode", ctypes.c_int), ("orthog", ctypes.c_int),
                ("krylov_arith", ctypes.c_int), ("precond", ctypes.c_int),
                ("mg_sweeps", ctypes.c_int), ("mg_omega", ctypes.c_double),
                ("mg_prec", ctypes.c_int), ("factor_tc", ctypes.c_int),
                ("apply_bulk", ctypes.c_int), ("wait_spins", ctypes.c_longlong),
                ("arnoldi_fused", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("newton_iterations", ctypes.c_int),
                ("converged", ctypes.c_int),
                ("line_search_halvings", ctypes.c_int),
                ("gmres_iterations", ctypes.c_int * MAX_NEWTON),
                ("res_history", ctypes.c_double * (MAX_NEWTON + 1)),
                ("dtau_history", ctypes.c_double * (MAX_NEWTON + 1)),
                ("block_builds", ctypes.c_int)]

    def summary(self) -> dict:
        n = self.newton_iterations
        return {"newton_iterations": n, "converged": bool(self.converged),
                "gmres_iterations": list(self.gmres_iterations[:n]),
                "res_history": list(self.res_history[: n + 1]),
                "dtau_history": list(self.dtau_history[: n + 1]),
                "block_builds": self.block_builds,
                "line_search_halvings": self.line_search_halvings}


_lib = None

_D = ctypes.c_double
_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "fr_default_config": (None, [ctypes.POINTER(_Config)]),
    "fr_create": (_I, [ctypes.POINTER(_Config), ctypes.POINTER(_P)]),
    "fr_destroy": (None, [_P]),
    "fr_set_mesh": (_I, [_P, _I, _I, _I, _I]),
    "fr_set_mesh_bounded": (_I, [_P, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_double)]),
    "fr_wall_force": (_I, [_P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "fr_update_mesh": (_I, [_P, _P, _P, _P]),
    "fr_residual": (_I, [_P, _P, _P, _P]),
    "fr_bdf_rhs": (_I, [_P, _P, _P, _P, _D, _D, _D, _D, _P, _P]),
    "fr_conservative": (_I, [_P, _P, _P, _P]),
    "fr_jvp": (_I, [_P, _P, _P, _D, _D, _P, _P]),
    "fr_precond_build": (_I, [_P, _P, _D, _D, _P]),
    "fr_precond_blocks": (_I, [_P, _P, _P]),
    "fr_precond_apply": (_I, [_P, _P, _P, _P]),
    "fr_gmres": (_I, [_P, _P, _P, _D, _D, _P, ctypes.POINTER(_I), _P]),
    "fr_bdf2_step": (_I, [_P, _P, _P, _P, _D, _D, _D, _D, ctypes.POINTER(Stats), _P]),
    "fr_ptc_solve": (_I, [_P, _P, ctypes.POINTER(Stats), _P]),
    "fr_residual_norms": (_I, [_P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
    "fr_num_dof": (ctypes.c_size_t, [_P]),
    "fr_block_size": (_I, [_P]),
    "fr_kernel_launches": (ctypes.c_longlong, [_P]),
    "fr_last_error": (ctypes.c_char_p, [_P]),
    "fr_version": (ctypes.c_char_p, []),
    "fr_profile": (_I, [_P, _I]),
    "fr_profile_read": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                             ctypes.POINTER(_D), _I]),
    "fr_profile_name": (ctypes.c_char_p, [_I]),
    "fr_residual_noalloc": (_I, [ctypes.POINTER(_Config), _I, _I, _P, _P, _P, _P, _P]),
    "fr_linearize": (_I, [_P, _P, _D, _D, _P]),
    "fr_apply_linear": (_I, [_P, _P, _P, _I, _P]),
    "fr_vjp": (_I, [_P, _P, _P, _D, _D, _P, _P]),
    "fr_tiles": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "fr_param_vjp": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(_D), _P, _P, _P]),
    "fr_param_jvp": (_I, [_P, _P, _P, _P, _P, _P, _P, _D, ctypes.POINTER(_D), ctypes.POINTER(_D),
                          ctypes.POINTER(_D), _P]),
    "fr_adjoint_solve": (_I, [_P, _P, _P, _D, _D, _P, ctypes.POINTER(_I), _P]),
    "fr_precond_apply_transposed": (_I, [_P, _P, _P, _P]),
    "fr_wall_force_vjp": (_I, [_P, _P, _D, _D, _D, _D, _P, _P]),
    "fr_conservative_vjp": (_I, [_P, _P, _P, _D, _D, _P, _P]),
    "fr_conservative_dmach": (_I, [_P, _P, _P, ctypes.POINTER(_D), _P]),
    "fr_inject_barrier_offset": (_I, [_P, ctypes.c_longlong]),
    "fr_batch_create": (_I, [ctypes.POINTER(_Config), _P, _I, ctypes.POINTER(_P)]),
    "fr_batch_destroy": (None, [_P]),
    "fr_batch_case_info": (_I, [_P, _I, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "fr_batch_num_dof": (ctypes.c_size_t, [_P]),
    "fr_batch_num_elements": (ctypes.c_size_t, [_P]),
    "fr_batch_num_groups": (_I, [_P]),
    "fr_batch_update_mesh": (_I, [_P, _P, _P, _P]),
    "fr_batch_residual": (_I, [_P, _P, _P, _P]),
    "fr_batch_conservative": (_I, [_P, _P, _P, _P]),
    "fr_batch_bdf2_step": (_I, [_P, _P, _P, _P, ctypes.POINTER(_D), _P, _P]),
    "fr_batch_ptc_solve": (_I, [_P, _P, _P, _P]),
    "fr_batch_profile": (_I, [_P, _I]),
    "fr_batch_profile_read": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                                   ctypes.POINTER(_D), _I]),
    "fr_batch_kernel_launches": (ctypes.c_longlong, [_P]),
    "fr_batch_last_error": (ctypes.c_char_p, [_P]),
}
PROF_KINDS = 17


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (building it first if it is absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    _build.build()
    if not os.path.exists(path):
        raise FrError(-1, f"{path} missing: the CUDA library was not built")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


@dataclasses.dataclass
class Config:
    p: int = 3
    mach: float = 0.05
    re: float = 0.0
    kappa: float = 1.0
    gamma: float = 1.4
    prandtl: float = 0.72
    eps_floor: float = 1e-8
    prec: str = "fp64"
    restart: int = 30
    maxit_lin: int = 100
    maxit_newton: int = 20
    lag: int = 2
    tol_res: float = 1e-6
    tol_pseudo: float = 1e-8
    dtau0: float = 0.01
    dtau_min: float = 0.01
    dtau_max: float = 1e20
    r_ser: float = 2.0
    dtau_unsteady: float = 1e20
    gmres_side: str = "left"
    ser_unsteady: int = 0
    dtau0_unsteady: float = 0.01
    line_search: int = 0
    jvp_mode: str = "linearized"
    graphs: int = 1
    apply_accum: str = "df64"
    tiles: int = 1
    block_mode: str = "linearized"
    orthog: str = "cgs2"
    krylov_arith: str = "fp64"
    precond: str = "block"
    mg_sweeps: int = 2
    mg_omega: float = 0.7
    mg_prec: str = "fp32"
    factor: str = "simt"
    apply_bulk: int = 0
    wait_spins: int = 0
    arnoldi_fused: int = 0

    def to_c(self) -> _Config:
        c = _Config()
        load().fr_default_config(ctypes.byref(c))
        for f in dataclasses.fields(self):
            if f.name == "prec":
                c.prec_dtype = PREC[self.prec]
            elif f.name == "gmres_side":
                c.gmres_side = {"left": 0, "right": 1}[self.gmres_side]
            elif f.name == "jvp_mode":
                c.jvp_mode = {"dual": 0, "linearized": 1}[self.jvp_mode]
            elif f.name == "orthog":
                c.orthog = {"cgs2": 0, "cgs": 1}[self.orthog]
            elif f.name == "krylov_arith":
                c.krylov_arith = {"fp64": 0, "df64": 1}[self.krylov_arith]
            elif f.name == "block_mode":
                c.block_mode = {"linearized": 0, "dual": 1}[self.block_mode]
            elif f.name == "apply_accum":
                c.apply_accum = {"fp32": 0, "df64": 1}[self.apply_accum]
            elif f.name == "factor":
                c.factor_tc = {"simt": 0, "tc_bf16": 1, "tc_bf16x3": 2}[self.factor]
            elif f.name == "mg_prec":
                c.mg_prec = PREC[self.mg_prec]
            elif f.name == "precond":
                c.precond = {"block": 0, "twolevel": 1}[self.precond]
            else:
                setattr(c, f.name, getattr(self, f.name))
        return c


class _Case(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("mach", ctypes.c_double), ("re", ctypes.c_double), ("kappa", ctypes.c_double)]


@dataclasses.dataclass
class Case:
    """One case of a batch: degree, periodic box size and gas (fr_case)."""
    p: int
    nx: int
    ny: int
    mach: float
    re: float
    kappa: float = 1.0


class Batch:
    """Independent cases advanced together (fr_batch_*): state vectors concatenate the
    cases' single-case layouts at the offsets of ``case_slice``."""

    def __init__(self, cfg: Config, cases):
        self.lib = load()
        self.cfg = cfg
        self.cases = list(cases)
        self._cc = cfg.to_c()
        arr = (_Case * len(self.cases))(*[_Case(c.p, c.nx, c.ny, c.mach, c.re, c.kappa)
                                          for c in self.cases])
        h = ctypes.c_void_p()
        rc = self.lib.fr_batch_create(ctypes.byref(self._cc), ctypes.cast(arr, _P), len(self.cases),
                                      ctypes.byref(h))
        if rc != FR_OK:
            raise FrError(rc, "fr_batch_create failed")
        self.b = h
        self.ndof = int(self.lib.fr_batch_num_dof(self.b))
        self.ne = int(self.lib.fr_batch_num_elements(self.b))
        self.num_groups = int(self.lib.fr_batch_num_groups(self.b))
        self.dof_off, self.case_ndof, self.elem_off, self.case_ne = [], [], [], []
        for k in range(len(self.cases)):
            v = [ctypes.c_size_t() for _ in range(4)]
            self._check(self.lib.fr_batch_case_info(self.b, k, *[ctypes.byref(x) for x in v]))
            self.dof_off.append(v[0].value)
            self.case_ndof.append(v[1].value)
            self.elem_off.append(v[2].value)
            self.case_ne.append(v[3].value)

    def _check(self, rc):
        if rc != FR_OK:
            msg = self.lib.fr_batch_last_error(self.b)
            raise FrError(rc, (msg or b"").decode())

    def close(self):
        if getattr(self, "b", None):
            self.lib.fr_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def case_slice(self, k) -> slice:
        return slice(self.dof_off[k], self.dof_off[k] + self.case_ndof[k])

    def elem_slice(self, k) -> slice:
        return slice(self.elem_off[k], self.elem_off[k] + self.case_ne[k])

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.fr_batch_kernel_launches(self.b))

    def update_mesh(self, corners, vel, stream=None):
        self._check(self.lib.fr_batch_update_mesh(self.b, _ptr(corners), _ptr(vel), _stream(stream)))

    def residual(self, q, out, stream=None):
        self._check(self.lib.fr_batch_residual(self.b, _ptr(q), _ptr(out), _stream(stream)))
        return out

    def conservative(self, q, out, stream=None):
        self._check(self.lib.fr_batch_conservative(self.b, _ptr(q), _ptr(out), _stream(stream)))
        return out

    def bdf2_step(self, q, qc_n, qc_nm1, coef, stream=None, allow_unconverged=False,
                  allow_nonfinite=False):
        """coef: per case (a0, a1, a2, dt).  Returns the per-case Stats list; the call's
        status code is kept in ``last_rc`` (FR_ERR_NOT_CONVERGED and FR_ERR_NONFINITE are
        returned instead of raised when allowed: the other cases still advanced)."""
        nc = len(self.cases)
        flat = (ctypes.c_double * (4 * nc))(*[float(x) for row in coef for x in row])
        st = (Stats * nc)()
        pnm1 = _ptr(qc_nm1) if qc_nm1 is not None else None
        rc = self.lib.fr_batch_bdf2_step(self.b, _ptr(q), _ptr(qc_n), pnm1, flat,
                                         ctypes.cast(st, _P), _stream(stream))
        self.last_rc = rc
        if not ((allow_unconverged and rc == -4) or (allow_nonfinite and rc == -3)):
            self._check(rc)
        return list(st)

    def ptc_solve(self, q, stream=None, allow_unconverged=False):
        nc = len(self.cases)
        st = (Stats * nc)()
        rc = self.lib.fr_batch_ptc_solve(self.b, _ptr(q), ctypes.cast(st, _P), _stream(stream))
        if not (allow_unconverged and rc == -4):
            self._check(rc)
        return list(st)

    def profile(self, enable: bool):
        self._check(self.lib.fr_batch_profile(self.b, 1 if enable else 0))

    def profile_read(self, reset: bool = True) -> dict:
        ms = (ctypes.c_double * PROF_KINDS)()
        cnt = (ctypes.c_longlong * PROF_KINDS)()
        tot = (ctypes.c_longlong * PROF_KINDS)()
        fl = (ctypes.c_double * PROF_KINDS)()
        by = (ctypes.c_double * PROF_KINDS)()
        self._check(self.lib.fr_batch_profile_read(self.b, ms, cnt, tot, fl, by, 1 if reset else 0))
        return {self.lib.fr_profile_name(k).decode():
                dict(ms=ms[k], launches=cnt[k], all_launches=tot[k], flops=fl[k], bytes=by[k])
                for k in range(PROF_KINDS)}


BC = {"wall": 1, "farfield": 2}


class Solver:
    """One library context: a mesh of nx-by-ny bilinear quads at degree p, periodic in
    both directions, or with ``bc=(below row 0, above row ny-1)`` (each "wall" or
    "farfield", far-field state ``q_inf`` = (p, u, v, T)) periodic in xi only."""

    def __init__(self, cfg: Config, nx: int, ny: int, bc=None, q_inf=None):
        self.lib = load()
        self.cfg = cfg
        self._cc = cfg.to_c()
        h = ctypes.c_void_p()
        self._check(self.lib.fr_create(ctypes.byref(self._cc), ctypes.byref(h)), None)
        self.ctx = h
        self.nx, self.ny = nx, ny
        if bc is None:
            self._check(self.lib.fr_set_mesh(self.ctx, nx, ny, 1, 1))
        else:
            qi = None if q_inf is None else (ctypes.c_double * 4)(*[float(x) for x in q_inf])
            self._check(self.lib.fr_set_mesh_bounded(self.ctx, nx, ny, BC[bc[0]], BC[bc[1]], qi))
        self.n = cfg.p + 1
        self.ne = nx * ny
        self.ndof = int(self.lib.fr_num_dof(self.ctx))
        self.block_size = int(self.lib.fr_block_size(self.ctx))

    def _check(self, rc, ctx="self"):
        if rc != FR_OK:
            msg = self.lib.fr_last_error(self.ctx if ctx == "self" else None)
            raise FrError(rc, (msg or b"").decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (4, self.ne, self.n, self.n)

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.fr_kernel_launches(self.ctx))

    @property
    def tiles(self) -> dict:
        """Tile shape K (elements per CTA = K x floor(128 / n^2)) of each point kernel."""
        k = (ctypes.c_int * 5)()
        self._check(self.lib.fr_tiles(self.ctx, k))
        return dict(zip(("trace", "elem", "trace_jvp", "elem_jvp", "linear_elem"), list(k)))

    # -- calls of include/fr.h
    def update_mesh(self, corners, vel, stream=None):
        self._check(self.lib.fr_update_mesh(self.ctx, _ptr(corners), _ptr(vel), _stream(stream)))

    def residual(self, q, out, stream=None):
        self._check(self.lib.fr_residual(self.ctx, _ptr(q), _ptr(out), _stream(stream)))
        return out

    def wall_force(self, q, stream=None):
        """(F_x, F_y) of the fluid on the wall faces of a bounded mesh (per unit span)."""
        f = (ctypes.c_double * 2)()
        self._check(self.lib.fr_wall_force(self.ctx, _ptr(q), f, _stream(stream)))
        return float(f[0]), float(f[1])

    def bdf_rhs(self, q, qc_n, qc_nm1, coeffs, dt, out, stream=None):
        a0, a1, a2 = coeffs
        pnm1 = _ptr(qc_nm1) if qc_nm1 is not None else None
        self._check(self.lib.fr_bdf_rhs(self.ctx, _ptr(q), _ptr(qc_n), pnm1, a0, a1, a2, dt,
                                         _ptr(out), _stream(stream)))
        return out

    def conservative(self, q, out, stream=None):
        self._check(self.lib.fr_conservative(self.ctx, _ptr(q), _ptr(out), _stream(stream)))
        return out

    def jvp(self, q, v, out, inv_dtau=0.0, a0_dt=0.0, stream=None):
        self._check(self.lib.fr_jvp(self.ctx, _ptr(q), _ptr(v), inv_dtau, a0_dt, _ptr(out),
                                    _stream(stream)))
        return out

    def linearize(self, q, inv_dtau=0.0, a0_dt=0.0, stream=None):
        self._check(self.lib.fr_linearize(self.ctx, _ptr(q), inv_dtau, a0_dt, _stream(stream)))

    def apply_linear(self, v, out, transpose=False, stream=None):
        self._check(self.lib.fr_apply_linear(self.ctx, _ptr(v), _ptr(out), 1 if transpose else 0,
                                             _stream(stream)))
        return out

    def vjp(self, q, w, out, inv_dtau=0.0, a0_dt=0.0, stream=None):
        self._check(self.lib.fr_vjp(self.ctx, _ptr(q), _ptr(w), inv_dtau, a0_dt, _ptr(out),
                                    _stream(stream)))
        return out

    def param_vjp(self, q, w, corners, vel, dcorners=None, dvel=None, mach=True, stream=None):
        """w . dR/dM_inf (returned; None if mach is False), and w . dR/d(corners),
        w . dR/d(corner velocities) into dcorners / dvel ([Ne, 4, 2] tensors) if given."""
        dm = ctypes.c_double(0.0)
        self._check(self.lib.fr_param_vjp(
            self.ctx, _ptr(q), _ptr(w), _ptr(corners), _ptr(vel),
            ctypes.byref(dm) if mach else None,
            _ptr(dcorners) if dcorners is not None else None,
            _ptr(dvel) if dvel is not None else None, _stream(stream)))
        return dm.value if mach else None

    def param_jvp(self, q, corners, vel, dcorners=None, dvel=None, dmach=0.0, dqinf=None, w=None,
                  force=False, stream=None):
        """Directional derivative at fixed q along (dcorners, dvel, dmach, dqinf): returns
        (w . R' or None, (F_x', F_y') or None)."""
        wd = ctypes.c_double(0.0)
        f = (ctypes.c_double * 2)()
        dq = (ctypes.c_double * 4)(*dqinf) if dqinf is not None else None
        self._check(self.lib.fr_param_jvp(
            self.ctx, _ptr(q), _ptr(w) if w is not None else None, _ptr(corners), _ptr(vel),
            _ptr(dcorners) if dcorners is not None else None,
            _ptr(dvel) if dvel is not None else None, float(dmach), dq,
            ctypes.byref(wd) if w is not None else None, f if force else None, _stream(stream)))
        return (wd.value if w is not None else None), ((float(f[0]), float(f[1])) if force else None)

    def adjoint_solve(self, q, g, lam, inv_dtau=0.0, a0_dt=0.0, stream=None) -> int:
        """A^T lam = g at q (transposed GMRES with the transposed element blocks)."""
        its = ctypes.c_int(0)
        self._check(self.lib.fr_adjoint_solve(self.ctx, _ptr(q), _ptr(g), inv_dtau, a0_dt,
                                              _ptr(lam), ctypes.byref(its), _stream(stream)))
        return its.value

    def precond_apply_transposed(self, r, out, stream=None):
        """out = M^-T r with the preconditioner of the last build."""
        self._check(self.lib.fr_precond_apply_transposed(self.ctx, _ptr(r), _ptr(out), _stream(stream)))
        return out

    def wall_force_vjp(self, q, wx, wy, out, alpha=1.0, beta=0.0, stream=None):
        """out = beta out + alpha d(wx F_x + wy F_y)/dq."""
        self._check(self.lib.fr_wall_force_vjp(self.ctx, _ptr(q), float(wx), float(wy), float(alpha),
                                               float(beta), _ptr(out), _stream(stream)))
        return out

    def conservative_vjp(self, q, w, out, alpha=1.0, beta=0.0, stream=None):
        """out = beta out + alpha (dq^c/dq)^T w."""
        self._check(self.lib.fr_conservative_vjp(self.ctx, _ptr(q), _ptr(w), float(alpha),
                                                 float(beta), _ptr(out), _stream(stream)))
        return out

    def conservative_dmach(self, q, w, stream=None) -> float:
        """sum of w . dq^c/dM at fixed q."""
        d = ctypes.c_double(0.0)
        self._check(self.lib.fr_conservative_dmach(self.ctx, _ptr(q), _ptr(w), ctypes.byref(d),
                                                   _stream(stream)))
        return d.value

    def inject_barrier_offset(self, n: int):
        """Test hook: n extra arrivals on the fused Arnoldi step's barrier counters."""
        self._check(self.lib.fr_inject_barrier_offset(self.ctx, n))

    def precond_build(self, q, inv_dtau=0.0, a0_dt=0.0, stream=None):
        self._check(self.lib.fr_precond_build(self.ctx, _ptr(q), inv_dtau, a0_dt, _stream(stream)))

    def precond_blocks(self, out, stream=None):
        self._check(self.lib.fr_precond_blocks(self.ctx, _ptr(out), _stream(stream)))
        return out

    def precond_apply(self, r, out, stream=None):
        self._check(self.lib.fr_precond_apply(self.ctx, _ptr(r), _ptr(out), _stream(stream)))
        return out

    def gmres(self, q, b, x, inv_dtau=0.0, a0_dt=0.0, stream=None) -> int:
        its = ctypes.c_int(0)
        self._check(self.lib.fr_gmres(self.ctx, _ptr(q), _ptr(b), inv_dtau, a0_dt, _ptr(x),
                                      ctypes.byref(its), _stream(stream)))
        return its.value

    def bdf2_step(self, q, qc_n, qc_nm1, dt, coeffs=BDF2, stream=None, allow_unconverged=False):
        st = Stats()
        a0, a1, a2 = coeffs
        pnm1 = _ptr(qc_nm1) if qc_nm1 is not None else None
        rc = self.lib.fr_bdf2_step(self.ctx, _ptr(q), _ptr(qc_n), pnm1, a0, a1, a2, dt,
                                   ctypes.byref(st), _stream(stream))
        if not (allow_unconverged and rc == -4):
            self._check(rc)
        return st

    def ptc_solve(self, q, stream=None, allow_unconverged=False):
        st = Stats()
        rc = self.lib.fr_ptc_solve(self.ctx, _ptr(q), ctypes.byref(st), _stream(stream))
        if not (allow_unconverged and rc == -4):
            self._check(rc)
        return st

    def profile(self, enable: bool):
        self._check(self.lib.fr_profile(self.ctx, 1 if enable else 0))

    def profile_read(self, reset: bool = True) -> dict:
        """{kernel class: dict(ms, launches, all_launches, flops, bytes)} since the last reset:
        device milliseconds and timed launches (while profiling is on), launches since
        creation, algorithmic flops and DRAM bytes issued."""
        ms = (ctypes.c_double * PROF_KINDS)()
        cnt = (ctypes.c_longlong * PROF_KINDS)()
        tot = (ctypes.c_longlong * PROF_KINDS)()
        fl = (ctypes.c_double * PROF_KINDS)()
        by = (ctypes.c_double * PROF_KINDS)()
        self._check(self.lib.fr_profile_read(self.ctx, ms, cnt, tot, fl, by, 1 if reset else 0))
        return {self.lib.fr_profile_name(k).decode():
                dict(ms=ms[k], launches=cnt[k], all_launches=tot[k], flops=fl[k], bytes=by[k])
                for k in range(PROF_KINDS)}

    def residual_norms(self, r, stream=None):
        m, a = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.fr_residual_norms(self.ctx, _ptr(r), ctypes.byref(m), ctypes.byref(a),
                                               _stream(stream)))
        return m.value, a.value


def residual_function():
    """A torch.autograd.Function computing R(q^p) with a Solver.

    ``Residual.apply(q, solver)``: backward is the library's reverse-mode product
    (fr_vjp), dR/dq^T g = -(A^T g) at inv_dtau = a0_dt = 0.
    ``Residual.apply(q, solver, corners, vel, mach)``: the mesh is first set from
    ``corners``, ``vel`` ([Ne, 4, 2] tensors) and the gradients also flow to them and to
    ``mach`` (a 0-d tensor equal to the solver's Mach number) through fr_param_vjp."""
    import torch

    class Residual(torch.autograd.Function):
        @staticmethod
        def forward(ctx, q, solver, corners=None, vel=None, mach=None):
            if corners is not None:
                solver.update_mesh(corners.contiguous(), vel.contiguous())
            if mach is not None and abs(float(mach) - solver.cfg.mach) > 1e-15 * solver.cfg.mach:
                raise ValueError("mach must equal the solver's Mach number")
            out = torch.empty_like(q)
            solver.residual(q.contiguous(), out)
            ctx.save_for_backward(q, corners, vel)
            ctx.solver = solver
            ctx.has_mach = mach is not None
            return out

        @staticmethod
        def backward(ctx, grad):
            q, corners, vel = ctx.saved_tensors
            g = grad.contiguous()
            out = torch.empty_like(q)
            ctx.solver.vjp(q.contiguous(), g, out, 0.0, 0.0)
            gc = gv = gm = None
            if corners is not None:
                need_c, need_v = ctx.needs_input_grad[2], ctx.needs_input_grad[3]
                gc = torch.empty_like(corners) if need_c else None
                gv = torch.empty_like(vel) if need_v else None
                want_m = ctx.has_mach and ctx.needs_input_grad[4]
                if need_c or need_v or want_m:
                    dm = ctx.solver.param_vjp(q.contiguous(), g, corners.contiguous(),
                                              vel.contiguous(), gc, gv, mach=want_m)
                    if want_m:
                        gm = torch.tensor(dm, dtype=q.dtype, device=q.device)
            return -out, None, gc, gv, gm

    return Residual
