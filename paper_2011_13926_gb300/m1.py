"""Thin ctypes binding of libm1.so (include/m1.h): argument marshalling only.

Every step of the M1 path runs in the CUDA library; this module converts
numpy arrays / torch tensors to (pointer, m1_mem) pairs, fills the C structs
and turns status codes into exceptions. There is no CPU fallback: importing a
missing or stale library raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libm1.so")

M1_OK, M1_ERR_ARG, M1_ERR_CUDA, M1_ERR_NOMEM, M1_ERR_NOT_CONVERGED, M1_ERR_NONFINITE, M1_ERR_TIMEOUT, \
    M1_ERR_STATE = range(8)
STATUS_NAMES = ["M1_OK", "M1_ERR_ARG", "M1_ERR_CUDA", "M1_ERR_NOMEM", "M1_ERR_NOT_CONVERGED",
                "M1_ERR_NONFINITE", "M1_ERR_TIMEOUT", "M1_ERR_STATE"]
BC = {"outflow": 0, "periodic": 1, "reflect": 2, "dirichlet": 3}
MEM_HOST, MEM_DEVICE = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
PRECOND_NONE, PRECOND_BJ, PRECOND_LEARNED, PRECOND_MG, PRECOND_LINE = 0, 1, 2, 3, 4
FP64_AUTO, FP64_NATIVE, FP64_DOUBLE_WORD = 0, 1, 2
KRYLOV_GMRES, KRYLOV_BICGSTAB = 0, 1

EXPORTED = ["m1_default_opts", "m1_init_grid", "m1_destroy", "m1_set_opacity", "m1_set_state", "m1_get_state",
            "m1_get_solution", "m1_set_boundary", "m1_set_emission", "m1_set_source", "m1_explicit_step",
            "m1_implicit_step", "m1_residual", "m1_jv", "m1_diag_blocks", "m1_gmres_solve", "m1_stats",
            "m1_profile", "m1_last_error", "m1_residual_noalloc", "m1_nn_num_params", "m1_nn_create",
            "m1_nn_destroy", "m1_nn_set_params", "m1_nn_get_params", "m1_nn_forward", "m1_nn_loss_grad",
            "m1_nn_train", "m1_nn_last_error", "m1_nn_make_pair", "m1_set_preconditioner", "m1_set_velocity",
            "m1_advect", "m1_batch_create", "m1_batch_destroy", "m1_batch_set_problem", "m1_batch_tune",
            "m1_batch_implicit_step", "m1_batch_get_solution", "m1_batch_num_classes", "m1_batch_last_error",
            "m1_batch_set_class", "m1_set_learned_form"]
LEARNED_ADDITIVE, LEARNED_TWO_STAGE, LEARNED_TWO_STAGE_ALL = 0, 1, 2


class GridDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", (C.c_int * 2) * 3), ("c", C.c_double), ("a_r", C.c_double),
                ("gas_coupling", C.c_int), ("well_balanced", C.c_int), ("ap_correction", C.c_int),
                ("fixed_eigs", C.c_int), ("lambda_floor", C.c_double), ("wb_boundary", C.c_int),
                ("implicit_eigs", C.c_int)]


class SolverOpts(C.Structure):
    _fields_ = [("newton_rtol", C.c_double), ("newton_max", C.c_int), ("restart", C.c_int),
                ("gmres_max", C.c_int), ("gmres_rtol", C.c_double), ("precision", C.c_int),
                ("precond", C.c_int), ("line_search", C.c_int), ("advance", C.c_int),
                ("refine_max", C.c_int), ("krylov", C.c_int), ("pc_rebuild", C.c_int),
                ("realizability", C.c_int), ("check_every", C.c_int), ("forcing", C.c_int)]


M1_HIST = 64
KERNEL_CLASSES = ["residual", "jv64", "jv32", "pc_build", "pc_apply", "ortho", "vector", "explicit"]


class StepInfo(C.Structure):
    _fields_ = [("converged", C.c_int), ("newton_iters", C.c_int), ("gmres_iters", C.c_int),
                ("refinements", C.c_int), ("res0", C.c_double), ("res", C.c_double),
                ("realizability_violations", C.c_longlong), ("time_ms", C.c_double),
                ("res_hist", C.c_double * M1_HIST), ("gmres_hist", C.c_int * M1_HIST),
                ("theta_hist", C.c_double * M1_HIST), ("fallback_cells", C.c_longlong),
                ("fallback_rounds", C.c_int), ("fp64_double_word", C.c_int), ("fp64_floor", C.c_double)]

    def as_dict(self, history: bool = False):
        out = {k: getattr(self, k) for k, _ in self._fields_[:8]}
        out["fallback_cells"] = self.fallback_cells
        out["fallback_rounds"] = self.fallback_rounds
        out["fp64_double_word"] = self.fp64_double_word
        out["fp64_floor"] = self.fp64_floor
        if history:
            k = min(self.newton_iters, M1_HIST)
            out["res_hist"] = list(self.res_hist[:k])
            out["gmres_hist"] = list(self.gmres_hist[:k])
            out["theta_hist"] = list(self.theta_hist[:k])
        return out


class SolveInfo(C.Structure):
    _fields_ = [("converged", C.c_int), ("iters", C.c_int), ("res0", C.c_double), ("res", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("newton_iters", C.c_longlong), ("gmres_iters", C.c_longlong), ("jv_calls", C.c_longlong),
                ("residual_calls", C.c_longlong), ("precond_builds", C.c_longlong),
                ("explicit_steps", C.c_longlong), ("implicit_steps", C.c_longlong),
                ("kernel_launches", C.c_longlong), ("bytes_per_jv", C.c_double),
                ("bytes_per_residual", C.c_double), ("bytes_per_jv32", C.c_double),
                ("kernel_ms", C.c_double * 8), ("kernel_count", C.c_longlong * 8), ("ortho_bytes", C.c_double),
                ("bytes_per_mg_cycle", C.c_double)]

    def as_dict(self):
        out = {k: getattr(self, k) for k, _ in self._fields_[:11]}
        out["ortho_bytes"] = self.ortho_bytes
        out["bytes_per_mg_cycle"] = self.bytes_per_mg_cycle
        out["kernel_ms"] = dict(zip(KERNEL_CLASSES, list(self.kernel_ms)))
        out["kernel_count"] = dict(zip(KERNEL_CLASSES, list(self.kernel_count)))
        return out


NOALLOC_MAX_CELLS = 65536


class BatchProblemInfo(C.Structure):
    _fields_ = [("converged", C.c_int), ("newton_iters", C.c_int), ("gmres_iters", C.c_int),
                ("res0", C.c_double), ("res", C.c_double)]


class TrainOpts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("lr", C.c_double), ("lr_decay", C.c_double), ("seed", C.c_ulonglong)]


class TrainInfo(C.Structure):
    _fields_ = [("steps", C.c_int), ("first_loss", C.c_double), ("final_loss", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DeviceFields(C.Structure):
    """m1_device_fields: device pointers of one grid's inputs."""
    _fields_ = [("Un", C.c_void_p), ("sigma_a", C.c_void_p), ("sigma_f", C.c_void_p), ("B", C.c_void_p),
                ("S", C.c_void_p), ("rho_cv", C.c_void_p), ("bE", (C.c_void_p * 2) * 3),
                ("bF", (C.c_void_p * 2) * 3), ("bmask", (C.c_void_p * 2) * 3)]


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libm1.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2011_13926_gb300.build.build()")
    lib = C.CDLL(path)
    P, D, I, V = C.c_void_p, C.c_double, C.c_int, None
    sig = {
        "m1_default_opts": (V, [C.POINTER(SolverOpts)]),
        "m1_init_grid": (I, [C.POINTER(GridDesc), P, C.POINTER(P)]),
        "m1_destroy": (I, [P]),
        "m1_set_opacity": (I, [P, P, P, I]),
        "m1_set_state": (I, [P, P, P, P, P, I]),
        "m1_get_state": (I, [P, P, P, P, I]),
        "m1_get_solution": (I, [P, P, I]),
        "m1_set_boundary": (I, [P, I, I, P, P, P, I]),
        "m1_set_emission": (I, [P, P, I]),
        "m1_set_source": (I, [P, P, I]),
        "m1_explicit_step": (I, [P, D]),
        "m1_implicit_step": (I, [P, D, C.POINTER(SolverOpts), C.POINTER(StepInfo)]),
        "m1_residual": (I, [P, D, P, P, I]),
        "m1_get_fallback": (I, [P, P, I]),
        "m1_jv": (I, [P, D, P, P, P, I, I]),
        "m1_diag_blocks": (I, [P, D, P, P, I]),
        "m1_mg_apply": (I, [P, D, P, P, P, I]),
        "m1_mg_blocks": (I, [P, I, C.POINTER(I), P, I]),
        "m1_gmres_solve": (I, [P, D, P, P, P, C.POINTER(SolverOpts), C.POINTER(SolveInfo), I]),
        "m1_stats": (I, [P, C.POINTER(Stats)]),
        "m1_profile": (I, [P, I]),
        "m1_set_fp64_arithmetic": (I, [P, I]),
        "m1_get_fp64_arithmetic": (I, [P, C.POINTER(I), C.POINTER(C.c_longlong)]),
        "m1_last_error": (C.c_char_p, [P]),
        "m1_residual_noalloc": (I, [C.POINTER(GridDesc), D, C.POINTER(DeviceFields), P, P, P, P]),
        "m1_nn_num_params": (C.c_size_t, []),
        "m1_nn_create": (I, [I, I, I, P, C.POINTER(P)]),
        "m1_nn_destroy": (I, [P]),
        "m1_nn_set_params": (I, [P, P, I]),
        "m1_nn_get_params": (I, [P, P, I]),
        "m1_nn_forward": (I, [P, P, P, I, I]),
        "m1_nn_loss_grad": (I, [P, P, P, C.POINTER(D), P, I]),
        "m1_nn_train": (I, [P, P, P, I, C.POINTER(TrainOpts), C.POINTER(TrainInfo), I]),
        "m1_nn_last_error": (C.c_char_p, [P]),
        "m1_nn_set_tensor_cores": (I, [P, I]),
        "m1_nn_make_pair": (I, [P, D, P, P, P, P, I]),
        "m1_set_preconditioner": (I, [P, P]),
        "m1_set_learned_form": (I, [P, I]),
        "m1_set_velocity": (I, [P, P, P, P, I]),
        "m1_batch_create": (I, [I, P, P, C.POINTER(P)]),
        "m1_batch_destroy": (I, [P]),
        "m1_batch_set_problem": (I, [P, I, P, P, P, P, P, I]),
        "m1_batch_tune": (I, [P, P, C.POINTER(SolverOpts), P]),
        "m1_batch_implicit_step": (I, [P, P, C.POINTER(SolverOpts), P, C.POINTER(D)]),
        "m1_batch_get_solution": (I, [P, I, P, I]),
        "m1_batch_num_classes": (I, [P]),
        "m1_batch_set_class": (I, [P, I, I]),
        "m1_batch_last_error": (C.c_char_p, [P]),
        "m1_advect": (I, [P, D]),
        "m1_velocity_sources": (I, [P, D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class M1Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def default_opts(**kw) -> SolverOpts:
    o = SolverOpts()
    load().m1_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _ptr(x, dtype=np.float64, allow_none=True):
    """(pointer, mem, keepalive) of a numpy array or torch tensor."""
    if x is None:
        if not allow_none:
            raise ValueError("array required")
        return None, MEM_HOST, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.float64: torch.float64, np.float32: torch.float32, np.uint8: torch.uint8}[dtype]
            if x.dtype != want:
                raise TypeError(f"expected {want}, got {x.dtype}")
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if x.is_cuda:
                return x.data_ptr(), MEM_DEVICE, x
            a = x.numpy()
            return a.ctypes.data, MEM_HOST, a
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, MEM_HOST, a


def _check_mem(*mems):
    ms = {m for m in mems if m is not None}
    if len(ms) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ms.pop() if ms else MEM_HOST


class Context:
    """One grid on the current CUDA device (m1_ctx)."""

    def __init__(self, desc: GridDesc, stream: Optional[int] = None):
        self.lib = load()
        self.desc = desc
        h = C.c_void_p()
        st = self.lib.m1_init_grid(C.byref(desc), C.c_void_p(stream or 0), C.byref(h))
        if st != M1_OK:
            raise M1Error(st, "m1_init_grid failed")
        self.h = h
        self.dim = desc.dim
        self.N = desc.n[0] * desc.n[1] * desc.n[2]
        self.nu = 1 + desc.dim + (1 if desc.gas_coupling else 0)
        self.shape2d = (desc.n[1], desc.n[0])

    def close(self):
        """m1_destroy: free the context's device memory."""
        if getattr(self, "h", None):
            self.lib.m1_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        st = getattr(self.lib, name)(self.h, *args)
        if st != M1_OK:
            raise M1Error(st, self.lib.m1_last_error(self.h).decode())
        return st

    def _call_status(self, name, *args):
        return getattr(self.lib, name)(self.h, *args)

    def last_error(self) -> str:
        """m1_last_error: the message of the last failed call."""
        return self.lib.m1_last_error(self.h).decode()

    # ---------------------------------------------------------------- inputs
    def set_opacity(self, sigma_a, sigma_f=None):
        """m1_set_opacity: sigma_a (exchange) and sigma_f (flux, alpha; None: sigma_a), N values each."""
        pa, ma, ka = _ptr(sigma_a)
        pf, mf, kf = _ptr(sigma_f)
        self._call("m1_set_opacity", pa, pf, _check_mem(ma, mf if pf else None))

    def set_state(self, E, F, T=None, rho_cv=None):
        """m1_set_state: the time-n state E (N), F (dim x N), and with gas coupling T and rho c_v (N each)."""
        pe, me, ke = _ptr(E)
        pF, mF, kF = _ptr(F)
        pt, mt, kt = _ptr(T)
        pr, mr, kr = _ptr(rho_cv)
        mem = _check_mem(me, mF, mt if pt else None, mr if pr else None)
        self._call("m1_set_state", pe, pF, pt, pr, mem)

    def set_boundary(self, axis, side, E, F, mask=None):
        """m1_set_boundary: Dirichlet ghost data (E, F) of one face and its mask (1: given, 0: zero-gradient)."""
        pe, me, ke = _ptr(E)
        pF, mF, kF = _ptr(F)
        pm, mm, km = _ptr(mask, dtype=np.uint8)
        self._call("m1_set_boundary", axis, side, pe, pF, pm, _check_mem(me, mF, mm if pm else None))

    def set_emission(self, B):
        """m1_set_emission: the frozen emission B = a_r T_g^4 of the radiation-only model (N values)."""
        p, m, k = _ptr(B)
        self._call("m1_set_emission", p, m)

    def set_source(self, S):
        """m1_set_source: the point-source term S added to the energy equation (N values)."""
        p, m, k = _ptr(S)
        self._call("m1_set_source", p, m)

    # ---------------------------------------------------------------- outputs
    def get_state(self, out=None):
        """(E, F, T) as numpy arrays (or into device tensors given in ``out``)."""
        if out is None:
            E = np.empty(self.N)
            F = np.empty(self.dim * self.N)
            T = np.empty(self.N) if self.nu == 2 + self.dim else None
            self._call("m1_get_state", E.ctypes.data, F.ctypes.data, T.ctypes.data if T is not None else None,
                       MEM_HOST)
            return E, F, T
        E, F, T = out
        pe, me, _ = _ptr(E)
        pF, mF, _ = _ptr(F)
        pt, mt, _ = _ptr(T)
        self._call("m1_get_state", pe, pF, pt, _check_mem(me, mF, mt if pt else None))
        return out

    def get_state_vector(self, out):
        """The current state as one unknown vector [E, F_0.., (T)] written into ``out``
        (a contiguous float64 numpy array or device tensor of n_u N values)."""
        p, m, k = _ptr(out)
        N = self.N
        pT = p + 8 * (1 + self.dim) * N if self.nu == 2 + self.dim else None
        self._call("m1_get_state", p, p + 8 * N, pT, m)
        return out

    def get_solution(self, out=None):
        """m1_get_solution: the last implicit step's U^{n+1} as [E, F_0.., (T)] (n_u N values)."""
        if out is None:
            out = np.empty(self.nu * self.N)
        p, m, k = _ptr(out)
        self._call("m1_get_solution", p, m)
        return out

    # ---------------------------------------------------------------- steps
    def explicit_step(self, dt: float):
        """m1_explicit_step: one semi-implicit step of size dt (Sect. 3.1); advances the state."""
        self._call("m1_explicit_step", C.c_double(dt))

    def implicit_step(self, dt: float, opts: Optional[SolverOpts] = None, raise_on_fail: bool = True):
        """m1_implicit_step: one backward-Euler step by Newton + Krylov; returns (status, StepInfo)."""
        info = StepInfo()
        o = opts if opts is not None else default_opts()
        st = self.lib.m1_implicit_step(self.h, C.c_double(dt), C.byref(o), C.byref(info))
        if st != M1_OK and raise_on_fail:
            raise M1Error(st, self.last_error())
        return st, info

    def get_fallback(self, out=None):
        """m1_get_fallback: the cells the admissibility fallback flagged in the last implicit step
        (N bytes, x fastest; 1 = flagged)."""
        if out is None:
            out = np.empty(self.N, dtype=np.uint8)
        p, m, k = _ptr(out, dtype=np.uint8)
        self._call("m1_get_fallback", p, m)
        return out

    def residual(self, dt: float, U, out=None):
        """m1_residual: the FP64 backward-Euler residual R(U) for step dt (time-n data from the state)."""
        pu, mu, ku = _ptr(U)
        if out is None:
            out = np.empty(self.nu * self.N) if mu == MEM_HOST else None
        po, mo, ko = _ptr(out)
        self._call("m1_residual", C.c_double(dt), pu, po, _check_mem(mu, mo))
        return out

    def jv(self, dt: float, U, v, out=None, precision: int = PREC_FP64):
        """m1_jv: J(U) v of the residual, in FP64 or with the mixed path's FP32 operator."""
        pu, mu, ku = _ptr(U)
        pv, mv, kv = _ptr(v)
        if out is None:
            out = np.empty(self.nu * self.N)
        po, mo, ko = _ptr(out)
        self._call("m1_jv", C.c_double(dt), pu, pv, po, precision, _check_mem(mu, mv, mo))
        return out

    def diag_blocks(self, dt: float, U, out=None):
        """m1_diag_blocks: the point blocks dR_i/dU_i of J(U), n_u^2 N values component-major."""
        pu, mu, ku = _ptr(U)
        if out is None:
            out = np.empty(self.nu * self.nu * self.N)
        po, mo, ko = _ptr(out)
        self._call("m1_diag_blocks", C.c_double(dt), pu, po, _check_mem(mu, mo))
        return out

    def mg_apply(self, dt: float, r, U=None, out=None):
        """One multigrid cycle z ~ J(U)^-1 r, the hierarchy built at U (None: time-n state)."""
        pu, mu, ku = _ptr(U)
        pr, mr, kr = _ptr(r)
        if out is None:
            out = np.empty(self.nu * self.N)
        po, mo, ko = _ptr(out)
        self._call("m1_mg_apply", C.c_double(dt), pu, pr, po, _check_mem(mu, mr, mo))
        return out

    def mg_levels(self) -> int:
        """Number of levels of the multigrid hierarchy last built."""
        n = C.c_int(0)
        self._call("m1_mg_blocks", 0, C.byref(n), None, MEM_HOST)
        return n.value

    def mg_blocks(self, level: int, nx: int, ny: int):
        """Stencil of one level after mg_apply, shaped (5, n_u, n_u, nx * ny)."""
        out = np.empty(5 * self.nu * self.nu * nx * ny)
        n = C.c_int(0)
        self._call("m1_mg_blocks", level, C.byref(n), out.ctypes.data, MEM_HOST)
        return out.reshape(5, self.nu, self.nu, nx * ny)

    def gmres_solve(self, dt: float, b, U=None, out=None, opts: Optional[SolverOpts] = None,
                    raise_on_fail: bool = True):
        """m1_gmres_solve: solve J(U) x = b with the solver options; returns (x, SolveInfo)."""
        pu, mu, ku = _ptr(U)
        pb, mb, kb = _ptr(b)
        if out is None:
            out = np.empty(self.nu * self.N)
        po, mo, ko = _ptr(out)
        info = SolveInfo()
        o = opts if opts is not None else default_opts()
        st = self.lib.m1_gmres_solve(self.h, C.c_double(dt), pu, pb, po, C.byref(o), C.byref(info),
                                     _check_mem(mu if pu else None, mb, mo))
        if st != M1_OK and raise_on_fail:
            raise M1Error(st, self.last_error())
        return out, info

    def set_velocity(self, ux, uy=None, uz=None):
        """m1_set_velocity: prescribed face velocities of the gas, one array per axis."""
        ps = [_ptr(u) for u in (ux, uy, uz)]
        self._call("m1_set_velocity", ps[0][0], ps[1][0], ps[2][0],
                   _check_mem(*[q[1] for q in ps if q[0] is not None]))

    def advect(self, dt: float):
        """m1_advect: explicit upwind transport of rho c_v T by the prescribed velocities over dt."""
        self._call("m1_advect", C.c_double(dt))

    def velocity_sources(self, dt: float):
        """Apply the explicit velocity-dependent radiation sources over dt to the state."""
        self._call("m1_velocity_sources", C.c_double(dt))

    def set_preconditioner(self, net):
        """m1_set_preconditioner: attach a trained U-Net (Net) as the learned preconditioner."""
        self._call("m1_set_preconditioner", net.h if net is not None else None)
        self._net = net  # keep the network alive while attached

    def set_learned_form(self, form: int):
        """m1_set_learned_form: LEARNED_ADDITIVE (default), LEARNED_TWO_STAGE (a point-block
        Jacobi stage, then the network on the residual it leaves, on odd Arnoldi steps) or
        LEARNED_TWO_STAGE_ALL (the two-stage form on every step)."""
        self._call("m1_set_learned_form", int(form))

    def make_pair(self, dt: float, e, U=None, out=None):
        """(x, t) NHWC float32 training pair from this context's Jacobian."""
        pe, me, ke = _ptr(e)
        pu, mu, ku = _ptr(U)
        if out is None:
            x = np.empty(7 * self.N, dtype=np.float32)
            t = np.empty(3 * self.N, dtype=np.float32)
        else:
            x, t = out
        px, mx, kx = _ptr(x, dtype=np.float32)
        pt, mt, kt = _ptr(t, dtype=np.float32)
        self._call("m1_nn_make_pair", C.c_double(dt), pu, pe, px, pt, _check_mem(me, mu if pu else None, mx, mt))
        return x, t

    def profile(self, enable: bool = True):
        """m1_profile: switch the per-kernel-class event timers on or off."""
        self._call("m1_profile", int(bool(enable)))

    def set_fp64_arithmetic(self, mode: int):
        """m1_set_fp64_arithmetic: FP64_AUTO, FP64_NATIVE or FP64_DOUBLE_WORD."""
        self._call("m1_set_fp64_arithmetic", int(mode))

    def fp64_arithmetic(self):
        """m1_get_fp64_arithmetic: (the arithmetic in use, range fallbacks so far)."""
        m, f = C.c_int(), C.c_longlong()
        self._call("m1_get_fp64_arithmetic", C.byref(m), C.byref(f))
        return m.value, f.value

    def stats(self) -> dict:
        """m1_stats: counters, kernel times per class and algorithmic bytes as a dict."""
        s = Stats()
        self._call("m1_stats", C.byref(s))
        return s.as_dict()


def grid_desc(dim, n, lo=None, hi=None, bc=None, c=1.0, a_r=1.0, gas=False, well_balanced=True,
              ap_correction=True, fixed_eigs=False, lambda_floor=0.0, wb_boundary=True,
              implicit_eigs=True) -> GridDesc:
    d = GridDesc()
    d.dim = dim
    n3 = list(n) + [1] * (3 - len(n))
    lo = list(lo or [0.0] * dim) + [0.0] * (3 - dim)
    hi = list(hi or [1.0] * dim) + [1.0] * (3 - dim)
    bc = list(bc or [("outflow", "outflow")] * dim) + [("outflow", "outflow")] * (3 - dim)
    for a in range(3):
        d.n[a] = int(n3[a])
        d.lo[a] = float(lo[a])
        d.hi[a] = float(hi[a])
        for s in range(2):
            d.bc[a][s] = BC[bc[a][s]] if isinstance(bc[a][s], str) else int(bc[a][s])
    d.c, d.a_r = float(c), float(a_r)
    d.gas_coupling = int(bool(gas))
    d.well_balanced = int(bool(well_balanced))
    d.ap_correction = int(bool(ap_correction))
    d.fixed_eigs = int(bool(fixed_eigs))
    d.lambda_floor = float(lambda_floor)
    d.wb_boundary = int(bool(wb_boundary))
    d.implicit_eigs = int(bool(implicit_eigs))
    return d


def context_from_problem(p, stream: Optional[int] = None, device: bool = False) -> Context:
    """Context for a problem object with the attributes of seeded_inputs.Problem
    (duck-typed: dim, n, lo, hi, bc, c, a_r, flags, fields, boundary)."""
    d = grid_desc(p.dim, p.n[:p.dim], p.lo[:p.dim], p.hi[:p.dim], p.bc, p.c, p.a_r, p.gas, p.well_balanced,
                  p.ap_correction, p.fixed_eigs, p.lambda_floor, p.wb_boundary, p.implicit_eigs)
    ctx = Context(d, stream)

    def put(x):
        if x is None:
            return None
        a = np.ascontiguousarray(x, dtype=np.float64).ravel()
        if device:
            import torch
            return torch.from_numpy(a).cuda()
        return a

    ctx.set_opacity(put(p.sigma_a), put(p.sigma_f))
    ctx.set_state(put(p.E), put(p.F), put(p.T) if p.gas else None, put(p.rho_cv) if p.gas else None)
    if not p.gas and p.B is not None:
        ctx.set_emission(put(p.B))
    if p.S is not None:
        ctx.set_source(put(p.S))
    for (a, side), (Eg, Fg, mask) in p.boundary.items():
        M = ctx.N // p.n[a]
        Eg = np.broadcast_to(np.asarray(Eg, float), (M,)) if np.ndim(Eg) == 0 else np.asarray(Eg, float).ravel()
        Fg = np.asarray(Fg, float).reshape(p.dim, -1)
        Fg = np.broadcast_to(Fg, (p.dim, M)) if Fg.shape[1] == 1 else Fg
        mask = None if mask is None else np.broadcast_to(np.asarray(mask, np.uint8).ravel(), (M,))
        ctx.set_boundary(a, side, np.ascontiguousarray(Eg), np.ascontiguousarray(Fg),
                         None if mask is None else np.ascontiguousarray(mask))
    return ctx


def residual_noalloc(desc: GridDesc, dt: float, fields: DeviceFields, U: int, R: int, norm2: int = 0,
                     stream: int = 0) -> int:
    """m1_residual_noalloc with raw device pointers; returns the status code
    (asynchronous on ``stream``)."""
    return load().m1_residual_noalloc(C.byref(desc), C.c_double(dt), C.byref(fields), C.c_void_p(U),
                                      C.c_void_p(R), C.c_void_p(norm2 or None), C.c_void_p(stream or None))


class Net:
    """m1_nn: the learned preconditioner network (batches of H x W images)."""

    def __init__(self, H: int, W: int, batch: int = 1, stream: int = 0):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.m1_nn_create(H, W, batch, C.c_void_p(stream or None), C.byref(h))
        if st != M1_OK:
            raise M1Error(st, "m1_nn_create failed")
        self.h, self.H, self.W, self.B = h, H, W, batch
        self.nparams = int(self.lib.m1_nn_num_params())

    def close(self):
        if getattr(self, "h", None):
            self.lib.m1_nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        st = getattr(self.lib, name)(self.h, *args)
        if st != M1_OK:
            raise M1Error(st, self.lib.m1_nn_last_error(self.h).decode())

    def set_tensor_cores(self, on: bool = True):
        """m1_nn_set_tensor_cores: BF16 tensor-core convolutions (default) or FP32 CUDA-core ones."""
        self._call("m1_nn_set_tensor_cores", int(bool(on)))

    def set_params(self, theta):
        p, m, k = _ptr(theta, dtype=np.float32)
        self._call("m1_nn_set_params", p, m)

    def get_params(self):
        out = np.empty(self.nparams, dtype=np.float32)
        self._call("m1_nn_get_params", out.ctypes.data, MEM_HOST)
        return out

    def forward(self, x, bf16: bool = False):
        px, mx, kx = _ptr(x, dtype=np.float32)
        y = np.empty(self.B * self.H * self.W * 3, dtype=np.float32)
        if mx == MEM_DEVICE:
            import torch
            y = torch.empty(y.size, dtype=torch.float32, device="cuda")
        py, my, ky = _ptr(y, dtype=np.float32)
        self._call("m1_nn_forward", px, py, int(bf16), _check_mem(mx, my))
        return y

    def loss_grad(self, x, t):
        px, mx, kx = _ptr(x, dtype=np.float32)
        pt, mt, kt = _ptr(t, dtype=np.float32)
        g = np.empty(self.nparams, dtype=np.float32)
        loss = C.c_double()
        if mx == MEM_DEVICE:
            import torch
            g = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        pg, mg, kg = _ptr(g, dtype=np.float32)
        self._call("m1_nn_loss_grad", px, pt, C.byref(loss), pg, _check_mem(mx, mt, mg))
        return loss.value, g

    def train(self, X, T, npairs: int, epochs: int = 1, lr: float = 1e-3, lr_decay: float = 1.0, seed: int = 1):
        px, mx, kx = _ptr(X, dtype=np.float32)
        pt, mt, kt = _ptr(T, dtype=np.float32)
        o = TrainOpts(epochs, lr, lr_decay, seed)
        info = TrainInfo()
        self._call("m1_nn_train", px, pt, int(npairs), C.byref(o), C.byref(info), _check_mem(mx, mt))
        return info.as_dict()


class Batch:
    """m1_batch: many independent 2D radiation-only problems per launch."""

    def __init__(self, problems, stream: int = 0):
        self.lib = load()
        descs = (GridDesc * len(problems))()
        for k, p in enumerate(problems):
            descs[k] = grid_desc(p.dim, p.n[:p.dim], p.lo[:p.dim], p.hi[:p.dim], p.bc, p.c, p.a_r, p.gas,
                                 p.well_balanced, p.ap_correction, p.fixed_eigs, p.lambda_floor, p.wb_boundary,
                                 p.implicit_eigs)
        h = C.c_void_p()
        st = self.lib.m1_batch_create(len(problems), C.cast(descs, C.c_void_p), C.c_void_p(stream or None),
                                      C.byref(h))
        if st != M1_OK:
            raise M1Error(st, "m1_batch_create failed")
        self.h = h
        self.problems = problems
        for k, p in enumerate(problems):
            arrs = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (p.sigma_a, p.sigma_f, p.E, p.F)]
            Bm = np.ascontiguousarray(p.B, dtype=np.float64).ravel() if p.B is not None else None
            self._call("m1_batch_set_problem", k, *[a.ctypes.data for a in arrs],
                       Bm.ctypes.data if Bm is not None else None, MEM_HOST)

    def close(self):
        """m1_batch_destroy."""
        if getattr(self, "h", None):
            self.lib.m1_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        st = getattr(self.lib, name)(self.h, *args)
        if st != M1_OK:
            raise M1Error(st, self.lib.m1_batch_last_error(self.h).decode())

    def num_classes(self) -> int:
        """m1_batch_num_classes: the number of size classes (distinct cell counts)."""
        return int(self.lib.m1_batch_num_classes(self.h))

    def set_class(self, c: int, threads: int):
        """Class c on persistent CTAs of `threads` (128, 256, 512), or 0: the single-grid path."""
        self._call("m1_batch_set_class", int(c), int(threads))

    def tune(self, dts, opts=None):
        """m1_batch_tune: per class the fastest of the single-grid path (0) and CTA sizes 128/256/512."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        chosen = np.zeros(self.num_classes(), dtype=np.int32)
        o = opts if opts is not None else default_opts()
        self._call("m1_batch_tune", d.ctypes.data, C.byref(o), chosen.ctypes.data)
        return chosen

    def implicit_step(self, dts, opts=None):
        """m1_batch_implicit_step: one step of every problem; returns (per-problem info, elapsed ms)."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        info = (BatchProblemInfo * len(self.problems))()
        ms = C.c_double()
        o = opts if opts is not None else default_opts()
        self._call("m1_batch_implicit_step", d.ctypes.data, C.byref(o), C.cast(info, C.c_void_p), C.byref(ms))
        return [{k: getattr(i, k) for k, _ in i._fields_} for i in info], ms.value

    def get_solution(self, k: int):
        """m1_batch_get_solution: problem k's U^{n+1} (3 N values)."""
        p = self.problems[k]
        out = np.empty(p.n_u * p.ncell)
        self._call("m1_batch_get_solution", int(k), out.ctypes.data, MEM_HOST)
        return out
